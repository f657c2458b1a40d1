// Batched COCG frequency-response solver in one persistent cooperative launch.
//
// Paper Sec. 4 solves the complex double-precision Helmholtz system with Krylov methods on
// the GPU. For the complex symmetric matrix of the eliminated FE system (A == A^T) the
// conjugate orthogonal CG (COCG: CG with the unconjugated bilinear form x^T y) is used:
//   q = A p, alpha = rho / p^T q, x += alpha p, r -= alpha q, rho' = r^T r, beta = rho'/rho,
//   p = r + beta p;
// stop when ||r|| / ||b|| <= tol, confirm with the true residual b - A x, restart from x with
// p = r if it misses tol. Optional stagnation rule: if the estimate has not halved its best
// value within `stall_window` steps, the same check-and-restart is taken.
//
// Mixed precision (FP64 iterative refinement, complex64 inner solve): r = b - A x in FP64,
// inner COCG on A d = r / ||r|| with complex64 matrix, vectors and SpMV accumulation, stopped at
// an inner reduction inner_tol, then x += ||r|| d in FP64. The true residual, the refinement
// update and the convergence test stay FP64; the inner dot products accumulate in FP64. A system
// whose refinement step fails to halve the FP64 residual (complex64 COCG stalls on strongly
// indefinite systems) is restarted as FP64 COCG from x = 0 in the same launch; an inner solve
// that did not reduce its own residual contributes no correction.
//
// Matrices are stored slot-major (27 values per row, val[k * n + row], columns implicit from
// the lattice offsets), one thread per row.
//
// Every system of the batch (its own lattice, frequency and matrix) is cut into row tiles.
// One launch runs all systems in lockstep super-steps of three phases (A: SpMV + dot, B: axpys
// + dots, C: direction update or true residual), separated by bounded grid barriers. Each
// tile writes its dot-product partials; the last block to finish a system's tiles (atomic
// arrival count) sums the partials in tile order -- a fixed order, so results do not depend
// on timing -- and takes that system's scalar decisions. Decisions that end a system take
// effect only in phase C, so the loop-control values every block reads at the top of a step
// are stable. Converged systems drop out of a compacted tile list.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "krylov_engine.cuh"

namespace helm {
namespace {
using namespace eng;

// ------------------------------- FP64 COCG phases ---------------------------------------------

__device__ void init_tile(const KParams& P, int t, double* sh, bool mixed) {
  const KTile T = P.tiles[t];
  KState* S = P.st + T.sys;
  const KSys Y = P.sys[T.sys];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = T.row0 + threadIdx.x; i < T.row1; i += kBlock) {
    const cd bi = Y.b[i];
    Y.x[i] = cd(0.0, 0.0);
    Y.r[i] = bi;
    v[0] += bi.re * bi.re - bi.im * bi.im;
    v[1] += 2.0 * bi.re * bi.im;
    v[2] += wnorm(Y, i) * (bi.re * bi.re + bi.im * bi.im);
  }
  block_sum<4>(v, sh);
  write_parts(P.part, t, v);
  if (arrive_last(S, Y.ntiles)) {
    cd rho, rr;
    sum_parts(P.part, Y.tile0, Y.ntiles, rho, rr, sh);
    if (threadIdx.x == 0) {
      S->bnorm = sqrt(rr.re);
      S->rnorm = S->bnorm;
      S->rho = rho;
      S->amode = 1;
      S->mode = MODE_RESID;
      S->prev_rel = 1.0;
      S->best_est = 1.0;
      S->best_it = 0;
      if (S->bnorm == 0.0) finish(P, S, HELM_OK, 0.0);
    }
  }
}

__device__ void phaseA_fp64(const KParams& P, int t, double* sh) {
  const KTile T = P.tiles[t];
  KState* S = P.st + T.sys;
  if (!vload(&S->act)) return;
  const KSys Y = P.sys[T.sys];
  const int amode = vload(&S->amode);
  const cd* src = amode ? Y.r : Y.p;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  tile_spmv<double>(
      Y.val, Y.cflag, src, Y.n, Y.Nx, Y.NxNy, T.row0, T.row1,
      [&](int64_t row, cd q, int) {
        Y.q[row] = q;
        const cd pi = src[row];
        if (amode) Y.p[row] = pi;
        v[0] += pi.re * q.re - pi.im * q.im;
        v[1] += pi.re * q.im + pi.im * q.re;
      },
      [&](int64_t row, cd qi) {
        const cd q0 = Y.q[row];
        Y.q[row] = cd(q0.re + qi.re, q0.im + qi.im);
        const cd pi = src[row];
        v[0] += pi.re * qi.re - pi.im * qi.im;
        v[1] += pi.re * qi.im + pi.im * qi.re;
      });
  block_sum<4>(v, sh);
  write_parts(P.part, t, v);
  if (arrive_last(S, Y.ntiles)) {
    cd mu, unused;
    sum_parts(P.part, Y.tile0, Y.ntiles, mu, unused, sh);
    if (threadIdx.x == 0) {
      S->it += 1;
      const cd rho = S->rho;
      if ((mu.re == 0.0 && mu.im == 0.0) || (rho.re == 0.0 && rho.im == 0.0)) {
        S->bd = 1;
        S->alpha = cd(0.0, 0.0);
      } else {
        S->alpha = cdiv(rho, mu);
      }
    }
  }
}

__device__ void phaseB_fp64(const KParams& P, int t, double* sh) {
  const KTile T = P.tiles[t];
  KState* S = P.st + T.sys;
  if (!vload(&S->act)) return;
  const KSys Y = P.sys[T.sys];
  const cd al = S->alpha;
  const cd mal(-al.re, -al.im);
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  constexpr int U = HELM_VEC_UNROLL;  // rows per thread per pass: all loads issued before the arithmetic
  for (int64_t i0 = T.row0 + threadIdx.x; i0 < T.row1; i0 += U * kBlock) {
    cd pv[U], qv[U], xv[U], rv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + (int64_t)u * kBlock;
      if (i < T.row1) {
        pv[u] = Y.p[i];
        qv[u] = Y.q[i];
        xv[u] = Y.x[i];
        rv[u] = Y.r[i];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + (int64_t)u * kBlock;
      if (i < T.row1) {
        cfma(xv[u], al, pv[u]);
        cfma(rv[u], mal, qv[u]);
        Y.x[i] = xv[u];
        Y.r[i] = rv[u];
        const cd ri = rv[u];
        v[0] += ri.re * ri.re - ri.im * ri.im;
        v[1] += 2.0 * ri.re * ri.im;
        v[2] += wnorm(Y, i) * (ri.re * ri.re + ri.im * ri.im);
      }
    }
  }
  block_sum<4>(v, sh);
  write_parts(P.part, t, v);
  if (arrive_last(S, Y.ntiles)) {
    cd rho_new, rr;
    sum_parts(P.part, Y.tile0, Y.ntiles, rho_new, rr, sh);
    if (threadIdx.x == 0) {
      const double est = sqrt(rr.re) / S->bnorm;
      S->est = est;
      S->amode = 0;
      S->save_best = 0;
      if (est < 0.5 * S->best_est) {
        S->best_est = est;
        S->best_it = S->it;
        S->save_best = 1;
      }
      if (!(est > P.tol) || S->it >= P.maxit || S->bd || (P.stall > 0 && S->it - S->best_it >= P.stall)) {
        // converged estimate, step cap, breakdown, or stagnation: true residual -- of the saved
        // best iterate if the estimate halved since the last restart and is above that value now
        // (restarting from the same point again would repeat the run)
        const bool best = est > P.tol && S->best_est < est && S->best_it > S->start_it && !S->bd;
        S->cmode = best ? C_CHECK_BEST : C_CHECK;
        S->save_best = 0;
      } else {
        S->beta = cdiv(rho_new, S->rho);
        S->rho = rho_new;
        S->cmode = C_PUPDATE;
      }
    }
  }
}

__device__ void phaseC_fp64(const KParams& P, int t, double* sh) {
  const KTile T = P.tiles[t];
  KState* S = P.st + T.sys;
  if (!vload(&S->act)) return;
  const KSys Y = P.sys[T.sys];
  const int cmode = vload(&S->cmode);
  if (cmode == C_PUPDATE) {
    const cd be = S->beta;
    if (vload(&S->save_best))
      for (int64_t i = T.row0 + threadIdx.x; i < T.row1; i += kBlock) Y.xb[i] = Y.x[i];
    constexpr int U = HELM_VEC_UNROLL;
    for (int64_t i0 = T.row0 + threadIdx.x; i0 < T.row1; i0 += U * kBlock) {
      cd rv[U], pv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t i = i0 + (int64_t)u * kBlock;
        if (i < T.row1) {
          rv[u] = Y.r[i];
          pv[u] = Y.p[i];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t i = i0 + (int64_t)u * kBlock;
        if (i < T.row1) {
          cfma(rv[u], be, pv[u]);
          Y.p[i] = rv[u];
        }
      }
    }
    return;
  }
  // true residual r = b - A x (x replaced by the saved best iterate first for C_CHECK_BEST: the
  // product reads xb, and each thread copies its own rows into x, which nothing reads here)
  const bool from_best = cmode == C_CHECK_BEST;
  const cd* xs = from_best ? Y.xb : Y.x;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  auto add = [&](int64_t row, cd ri) {
    v[0] += ri.re * ri.re - ri.im * ri.im;
    v[1] += 2.0 * ri.re * ri.im;
    v[2] += wnorm(Y, row) * (ri.re * ri.re + ri.im * ri.im);
  };
  tile_spmv<double>(
      Y.val, Y.cflag, xs, Y.n, Y.Nx, Y.NxNy, T.row0, T.row1,
      [&](int64_t row, cd s, int c) {
        if (from_best) Y.x[row] = Y.xb[row];
        const cd bi = Y.b[row];
        const cd ri(bi.re - s.re, bi.im - s.im);
        Y.r[row] = ri;
        if (!c) add(row, ri);
      },
      [&](int64_t row, cd si) {
        const cd r0 = Y.r[row];
        const cd ri(r0.re - si.re, r0.im - si.im);
        Y.r[row] = ri;
        add(row, ri);
      });
  block_sum<4>(v, sh);
  write_parts(P.part, t, v);
  if (arrive_last(S, Y.ntiles)) {
    cd rho, rr;
    sum_parts(P.part, Y.tile0, Y.ntiles, rho, rr, sh);
    if (threadIdx.x == 0) {
      const double rel = sqrt(rr.re) / S->bnorm;
      S->relres = rel;
      if (rel <= P.tol) finish(P, S, HELM_OK, rel);
      else if (!(rel == rel)) finish(P, S, HELM_NAN, rel);
      else if (S->it >= P.maxit) finish(P, S, HELM_NOT_CONVERGED, rel);
      else if (S->bd) finish(P, S, HELM_BREAKDOWN, rel);
      else {
        S->rho = rho;
        S->amode = 1;
        S->restarts += 1;
        S->best_est = rel;
        S->best_it = S->it;
        S->start_it = S->it;
      }
    }
  }
}

// ------------------------------- mixed-precision phases ---------------------------------------

// FP64 true residual of a refinement step (both mixed variants), phase A.
__device__ void resid_phaseA(const KParams& P, int t, double* sh, const KTile& T, KState* S, const KSys& Y) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  // FP64 true residual of the refinement (norm, and r^T r for a switch to FP64 COCG)
  auto add = [&](int64_t row, cd ri) {
    v[0] += ri.re * ri.re - ri.im * ri.im;
    v[1] += 2.0 * ri.re * ri.im;
    v[2] += wnorm(Y, row) * (ri.re * ri.re + ri.im * ri.im);
  };
  tile_spmv<double>(
      Y.val, Y.cflag, Y.x, Y.n, Y.Nx, Y.NxNy, T.row0, T.row1,
      [&](int64_t row, cd s, int c) {
        const cd bi = Y.b[row];
        const cd ri(bi.re - s.re, bi.im - s.im);
        Y.r[row] = ri;
        if (!c) add(row, ri);
      },
      [&](int64_t row, cd si) {
        const cd r0 = Y.r[row];
        const cd ri(r0.re - si.re, r0.im - si.im);
        Y.r[row] = ri;
        add(row, ri);
      });
  block_sum<4>(v, sh);
  write_parts(P.part, t, v);
  if (arrive_last(S, Y.ntiles)) {
    cd rho, rr;
    sum_parts(P.part, Y.tile0, Y.ntiles, rho, rr, sh);
    if (threadIdx.x == 0) {
      const double rel = sqrt(rr.re) / S->bnorm;
      S->relres = rel;
      S->pend = 0;
      S->to_fp64 = 0;
      if (rel <= P.tol) { S->pend = 1; S->status = HELM_OK; }
      else if (!(rel == rel)) { S->pend = 1; S->status = HELM_NAN; }
      else if (S->outer >= P.max_outer || S->it >= P.maxit) { S->pend = 1; S->status = HELM_NOT_CONVERGED; }
      else if (S->outer >= 1 && rel > 0.5 * S->prev_rel) {
        // complex64 refinement stalls on this system: restart it as FP64 COCG from x = 0
        // (phase B sets x = 0, r = b). COCG's path on these indefinite systems depends on its
        // starting vector; from zero the fallback runs exactly the plain FP64 iteration.
        S->to_fp64 = 1;
        S->reset_x = 1;
        S->best_est = 1.0;
        S->best_it = S->it;
        S->start_it = S->it;
        S->rho = rho;
        S->amode = 1;
        S->bd = 0;
      } else { S->rnorm = sqrt(rr.re); S->outer += 1; }
      S->prev_rel = rel;
    }
  }
}

__device__ void phaseA_mixed(const KParams& P, int t, double* sh) {
  const KTile T = P.tiles[t];
  KState* S = P.st + T.sys;
  if (!vload(&S->act)) return;
  const KSys Y = P.sys[T.sys];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  if (vload(&S->mode) == MODE_RESID) {
    resid_phaseA(P, t, sh, T, S, Y);
    return;
  }
  // inner complex64 step: q32 = A32 src
  const int amode = vload(&S->amode);
  const cf* src = amode ? Y.r32 : Y.p32;
  float a0 = 0.f, a1 = 0.f;  // per-thread FP32 partial over its rows, FP64 from the block sum on
  tile_spmv<float>(
      Y.val32, Y.cflag, src, Y.n, Y.Nx, Y.NxNy, T.row0, T.row1,
      [&](int64_t row, cf q, int) {
        Y.q32[row] = q;
        const cf pi = src[row];
        if (amode) Y.p32[row] = pi;
        a0 += pi.re * q.re - pi.im * q.im;
        a1 += pi.re * q.im + pi.im * q.re;
      },
      [&](int64_t row, cf qi) {
        const cf q0 = Y.q32[row];
        Y.q32[row] = cf(q0.re + qi.re, q0.im + qi.im);
        const cf pi = src[row];
        a0 += pi.re * qi.re - pi.im * qi.im;
        a1 += pi.re * qi.im + pi.im * qi.re;
      });
  v[0] = a0;
  v[1] = a1;
  block_sum<4>(v, sh);
  write_parts(P.part, t, v);
  if (arrive_last(S, Y.ntiles)) {
    cd mu, unused;
    sum_parts(P.part, Y.tile0, Y.ntiles, mu, unused, sh);
    if (threadIdx.x == 0) {
      S->it += 1;
      S->it32 += 1;
      S->inner_it += 1;
      const cd rho = S->rho;
      if ((mu.re == 0.0 && mu.im == 0.0) || (rho.re == 0.0 && rho.im == 0.0)) {
        S->bd = 1;
        S->alpha = cd(0.0, 0.0);
      } else {
        S->alpha = cdiv(rho, mu);
      }
    }
  }
}

// Fallback of a mixed system to FP64 COCG from x = 0: r = b, rho = b^T b (phase B).
__device__ void fallback_phaseB(const KParams& P, int t, double* sh, const KTile& T, KState* S, const KSys& Y) {
  if (!vload(&S->reset_x)) return;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  // restart from x = 0: r = b, rho = b^T b
  for (int64_t i = T.row0 + threadIdx.x; i < T.row1; i += kBlock) {
    const cd bi = Y.b[i];
    Y.x[i] = cd(0.0, 0.0);
    Y.r[i] = bi;
    v[0] += bi.re * bi.re - bi.im * bi.im;
    v[1] += 2.0 * bi.re * bi.im;
  }
  block_sum<4>(v, sh);
  write_parts(P.part, t, v);
  if (arrive_last(S, Y.ntiles)) {
    cd rho, unused;
    sum_parts(P.part, Y.tile0, Y.ntiles, rho, unused, sh);
    if (threadIdx.x == 0) S->rho = rho;
  }
}

__device__ void phaseB_mixed(const KParams& P, int t, double* sh) {
  const KTile T = P.tiles[t];
  KState* S = P.st + T.sys;
  if (!vload(&S->act)) return;
  const KSys Y = P.sys[T.sys];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  if (vload(&S->mode) == MODE_RESID) {
    if (vload(&S->pend)) return;
    if (vload(&S->to_fp64)) {
      fallback_phaseB(P, t, sh, T, S, Y);
      return;
    }
    // start an inner solve on r / ||r|| (complex64), x32 = 0
    const double sc = 1.0 / S->rnorm;
    float a0 = 0.f, a1 = 0.f;
    for (int64_t i = T.row0 + threadIdx.x; i < T.row1; i += kBlock) {
      const cd ri = Y.r[i];
      const cf r32(__double2float_rn(ri.re * sc), __double2float_rn(ri.im * sc));
      Y.r32[i] = r32;
      Y.x32[i] = cf(0.f, 0.f);
      a0 += r32.re * r32.re - r32.im * r32.im;
      a1 += 2.f * r32.re * r32.im;
    }
    v[0] = a0;
    v[1] = a1;
    block_sum<4>(v, sh);
    write_parts(P.part, t, v);
    if (arrive_last(S, Y.ntiles)) {
      cd rho, unused;
      sum_parts(P.part, Y.tile0, Y.ntiles, rho, unused, sh);
      if (threadIdx.x == 0) {
        S->rho = rho;
        S->amode = 1;
        S->inner_it = 0;
        S->best_est = 1.0;
        S->best_it = 0;
        S->bd = 0;  // the mode itself changes in phase C (phase C of this step still reads it)
      }
    }
    return;
  }
  const cd al = S->alpha;
  const cf a32((float)al.re, (float)al.im);
  const cf ma32(-a32.re, -a32.im);
  float acc[3] = {0.f, 0.f, 0.f};
  constexpr int U = HELM_VEC_UNROLL;
  for (int64_t i0 = T.row0 + threadIdx.x; i0 < T.row1; i0 += U * kBlock) {
    cf pv[U], qv[U], xv[U], rv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + (int64_t)u * kBlock;
      if (i < T.row1) {
        pv[u] = Y.p32[i];
        qv[u] = Y.q32[i];
        xv[u] = Y.x32[i];
        rv[u] = Y.r32[i];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + (int64_t)u * kBlock;
      if (i < T.row1) {
        cfma(xv[u], a32, pv[u]);
        cfma(rv[u], ma32, qv[u]);
        Y.x32[i] = xv[u];
        Y.r32[i] = rv[u];
        const cf ri = rv[u];
        acc[0] += ri.re * ri.re - ri.im * ri.im;
        acc[1] += 2.f * ri.re * ri.im;
        acc[2] += wnorm32(Y, i) * (ri.re * ri.re + ri.im * ri.im);
      }
    }
  }
  v[0] = acc[0];
  v[1] = acc[1];
  v[2] = acc[2];
  block_sum<4>(v, sh);
  write_parts(P.part, t, v);
  if (arrive_last(S, Y.ntiles)) {
    cd rho_new, rr;
    sum_parts(P.part, Y.tile0, Y.ntiles, rho_new, rr, sh);
    if (threadIdx.x == 0) {
      const double est = sqrt(rr.re);  // relative to ||r / ||r|| || = 1
      S->est = est;
      S->amode = 0;
      if (est < 0.5 * S->best_est) {
        S->best_est = est;
        S->best_it = S->inner_it;
      }
      if (!(est > inner_stop(P, S)) || S->inner_it >= P.inner_maxit || S->it >= P.maxit || S->bd ||
          (P.stall > 0 && S->inner_it - S->best_it >= P.stall)) {
        S->cmode = C_XUPDATE;
        S->discard = !(est < 1.0);  // no reduction (or NaN): keep x, the residual test switches
      } else {
        S->beta = cdiv(rho_new, S->rho);
        S->rho = rho_new;
        S->cmode = C_PUPDATE;
      }
    }
  }
}

// End of a refinement residual step (both mixed variants), phase C: finish, fall back to FP64
// COCG, or start the next inner solve.
__device__ void resid_phaseC(const KParams& P, KState* S, const KSys& Y) {
  const int pend = vload(&S->pend), to64 = vload(&S->to_fp64);
  if (arrive_last(S, Y.ntiles) && threadIdx.x == 0) {
    if (pend) finish(P, S, S->status, S->relres);
    else if (to64) { S->mode = MODE_FP64; S->fell_back = 1; }
    else S->mode = MODE_INNER;
  }
}

__device__ void phaseC_mixed(const KParams& P, int t, double* sh) {
  const KTile T = P.tiles[t];
  KState* S = P.st + T.sys;
  if (!vload(&S->act)) return;
  const KSys Y = P.sys[T.sys];
  if (vload(&S->mode) == MODE_RESID) {
    resid_phaseC(P, S, Y);
    return;
  }
  if (vload(&S->cmode) == C_PUPDATE) {
    const cd be = S->beta;
    const cf b32((float)be.re, (float)be.im);
    constexpr int U = HELM_VEC_UNROLL;
    for (int64_t i0 = T.row0 + threadIdx.x; i0 < T.row1; i0 += U * kBlock) {
      cf rv[U], pv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t i = i0 + (int64_t)u * kBlock;
        if (i < T.row1) {
          rv[u] = Y.r32[i];
          pv[u] = Y.p32[i];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t i = i0 + (int64_t)u * kBlock;
        if (i < T.row1) {
          cfma(rv[u], b32, pv[u]);
          Y.p32[i] = rv[u];
        }
      }
    }
    return;
  }
  // refinement update x += ||r|| * d (FP64)
  const double sc = vload(&S->discard) ? 0.0 : S->rnorm;
  for (int64_t i = T.row0 + threadIdx.x; i < T.row1; i += kBlock) {
    const cf d = Y.x32[i];
    cd xi = Y.x[i];
    xi.re = fma(sc, (double)d.re, xi.re);
    xi.im = fma(sc, (double)d.im, xi.im);
    Y.x[i] = xi;
  }
  if (arrive_last(S, Y.ntiles) && threadIdx.x == 0) S->mode = MODE_RESID;
}

// ------------------------------- double-word mixed phases -------------------------------------
// Same refinement as above; the inner COCG runs in double-word arithmetic (dw.cuh): matrix,
// vectors and every inner product and update carried as pairs of floats on the FP32 pipe, the
// real and imaginary components of each complex value advanced together by the paired FP32
// instructions (dacc2), the per-thread dot-product partials converted to FP64 once per phase.
// Refinement residuals, the correction x += ||r|| d and all scalar decisions stay FP64.

// Real-part product of one row in double-word arithmetic: matrix parts (slot stride ns) and x
// by cached loads, three accumulators per component (one per stencil line dj), planes in order.
// CLAMP: gather indices clamped into [0, n) (rows within one stencil reach of either end; the
// entries there are zero); interior rows skip the clamps.
template <bool CLAMP>
__device__ __forceinline__ cw dia_row_re_dw2(const float2* __restrict__ vre, const cw* x, int64_t n, int64_t ns,
                                             int64_t Nx, int64_t NxNy, int64_t row) {
  dacc2 acc[3];
#pragma unroll
  for (int dl = -1; dl <= 1; ++dl) {
    float2 a[9];
    cw xv[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {  // all loads of one lattice plane first
      const int di = q % 3 - 1, dj = q / 3 - 1;
      const int k = q + 9 * (dl + 1);
      int64_t c = row + di + Nx * dj + NxNy * dl;
      if (CLAMP) c = c < 0 ? 0 : (c >= n ? n - 1 : c);
      a[q] = __ldcs(vre + (int64_t)k * ns + row);
      xv[q] = x[c];
    }
#pragma unroll
    for (int q = 0; q < 9; ++q)
      acc[q / 3].mac(make_float2(a[q].x, a[q].x), make_float2(a[q].y, a[q].y), cw_hi(xv[q]), cw_lo(xv[q]));
  }
  acc[0].add(acc[1]);
  acc[0].add(acc[2]);
  float2 hi, lo;
  acc[0].get(hi, lo);
  return cw_from(hi, lo);
}

// Product of the tile's rows with x: first(row, q, complex_row_flag) with the real-part product
// of every row, then, if any row of the tile is flagged complex, fix(row, imaginary part) for the
// flagged rows. With `pf` = d > 0 each thread prefetches into L2 the matrix parts of the row it
// reaches d iterations later.
template <typename F1, typename F2>
__device__ __forceinline__ void tile_spmv_dw(const KSys& Y, const cw* x, int64_t row0, int64_t row1, F1 first, F2 fix,
                                             int pf) {
  const int64_t n = Y.n, ns = Y.nsw, Nx = Y.Nx, NxNy = Y.NxNy;
  const int64_t reach = NxNy + Nx + 1;  // largest |column - row| of the stencil
  int has_c = 0;
  const int64_t ahead = (int64_t)pf * kBlock;
  for (int64_t r0 = row0 + threadIdx.x; r0 < row1; r0 += kBlock) {
    if (pf && r0 + ahead < row1) {
#pragma unroll
      for (int k = 0; k < 27; ++k) prefetch_l2(Y.valw + (int64_t)k * ns + r0 + ahead);
      const int64_t up = r0 + ahead + NxNy;  // x of the plane above, first touched by this tile
      if (up < n) prefetch_l2(x + up);
    }
    const cw s0 = (r0 >= reach && r0 + reach < n) ? dia_row_re_dw2<false>(Y.valw, x, n, ns, Nx, NxNy, r0)
                                                  : dia_row_re_dw2<true>(Y.valw, x, n, ns, Nx, NxNy, r0);
    const int c0 = Y.cflag[r0];
    first(r0, s0, c0);
    has_c |= c0;
  }
  if (__syncthreads_or(has_c)) {
    const float2* vim = Y.valw + 27 * ns;
    for (int64_t row = row0 + threadIdx.x; row < row1; row += kBlock)
      if (Y.cflag[row]) fix(row, dia_row_im_dw2<true>(vim, x, n, ns, Nx, NxNy, row));
  }
}

// Thread 0: bulk L2 prefetch of rows [r0, r0 + kBlock) of the given vectors (16 bytes per row).
template <int NV>
__device__ __forceinline__ void prefetch_rows(const cw* const (&v)[NV], int64_t r0, int64_t row1) {
  if (r0 >= row1) return;
  const uint32_t bytes = (uint32_t)((row1 - r0 < kBlock ? row1 - r0 : kBlock) * 16);
#pragma unroll
  for (int k = 0; k < NV; ++k) bulk_prefetch_l2(v[k] + r0, bytes);
}

__device__ __forceinline__ double2 dacc2_to_double(const dacc2& a) {
  return make_double2((double)a.s.x + (double)a.c.x, (double)a.s.y + (double)a.c.y);
}

__device__ void phaseA_dw(const KParams& P, int t, double* sh) {
  const KTile T = P.tiles[t];
  KState* S = P.st + T.sys;
  if (!vload(&S->act)) return;
  const KSys Y = P.sys[T.sys];
  if (vload(&S->mode) == MODE_RESID) {
    resid_phaseA(P, t, sh, T, S, Y);
    return;
  }
  const int amode = vload(&S->amode);
  const cw* src = amode ? Y.rw : Y.pw;
  dacc2 dot;  // p^T q
  auto first = [&](int64_t row, cw q, int c) {
    Y.qw[row] = q;
    const cw pi = src[row];
    if (amode) Y.pw[row] = pi;
    if (!c) cw_dotu_acc2(dot, pi, q);
  };
  auto fix = [&](int64_t row, cw qi) {
    const cw q = cw_add(Y.qw[row], qi);
    Y.qw[row] = q;
    cw_dotu_acc2(dot, src[row], q);
  };
  tile_spmv_dw(Y, src, T.row0, T.row1, first, fix, P.prefetch);
  const double2 d2 = dacc2_to_double(dot);
  double v[4] = {d2.x, d2.y, 0.0, 0.0};
  block_sum<4>(v, sh);
  write_parts(P.part, t, v);
  if (arrive_last(S, Y.ntiles)) {
    cd mu, unused;
    sum_parts(P.part, Y.tile0, Y.ntiles, mu, unused, sh);
    if (threadIdx.x == 0) {
      S->it += 1;
      S->it32 += 1;
      S->inner_it += 1;
      const cd rho = S->rho;
      if ((mu.re == 0.0 && mu.im == 0.0) || (rho.re == 0.0 && rho.im == 0.0)) {
        S->bd = 1;
        S->alpha = cd(0.0, 0.0);
      } else {
        S->alpha = cdiv(rho, mu);
      }
    }
  }
}

__device__ void phaseB_dw(const KParams& P, int t, double* sh) {
  const KTile T = P.tiles[t];
  KState* S = P.st + T.sys;
  if (!vload(&S->act)) return;
  const KSys Y = P.sys[T.sys];
  if (vload(&S->mode) == MODE_RESID) {
    if (vload(&S->pend)) return;
    if (vload(&S->to_fp64)) {
      fallback_phaseB(P, t, sh, T, S, Y);
      return;
    }
    // start an inner solve on r / ||r|| (double-word), d = 0
    const double sc = 1.0 / S->rnorm;
    dacc2 rr;
    for (int64_t i = T.row0 + threadIdx.x; i < T.row1; i += kBlock) {
      const cd ri = Y.r[i];
      cw w;
      split_double(ri.re * sc, w.rh, w.rl);
      split_double(ri.im * sc, w.ih, w.il);
      Y.rw[i] = w;
      Y.xw[i] = cw{0.f, 0.f, 0.f, 0.f};
      cw_dotu_acc2(rr, w, w);
    }
    const double2 r2 = dacc2_to_double(rr);
    double v[4] = {r2.x, r2.y, 0.0, 0.0};
    block_sum<4>(v, sh);
    write_parts(P.part, t, v);
    if (arrive_last(S, Y.ntiles)) {
      cd rho, unused;
      sum_parts(P.part, Y.tile0, Y.ntiles, rho, unused, sh);
      if (threadIdx.x == 0) {
        S->rho = rho;
        S->amode = 1;
        S->inner_it = 0;
        S->best_est = 1.0;
        S->best_it = 0;
        S->bd = 0;  // the mode itself changes in phase C
      }
    }
    return;
  }
  // r -= alpha q here; x += alpha p is left to phase C, which reads p anyway (same values)
  const cd al = S->alpha;
  const cws ma = to_cws(-al.re, -al.im);
  dacc2 rr;
  float nrm = 0.f;  // ||r||^2 for the stopping estimate (FP32 is enough for a threshold test)
  // thread 0 keeps the block's next `pf_chunks` row chunks of q, r on their way into L2
  const int d = P.pf_chunks;
  const cw* const vecs[2] = {Y.qw, Y.rw};
  if (threadIdx.x == 0)
    for (int j = 0; j < d; ++j) prefetch_rows(vecs, T.row0 + (int64_t)j * kBlock, T.row1);
  // four rows per thread per pass, all of their loads issued before the arithmetic (the phase
  // streams only q and r, so the rows' loads fit in registers; the rows are still taken, and
  // their dot-product terms added, in the same order as one row per pass)
  constexpr int U = 4;
  for (int64_t i0 = T.row0; i0 < T.row1; i0 += U * kBlock) {
    if (threadIdx.x == 0 && d > 0)
#pragma unroll
      for (int u = 0; u < U; ++u) prefetch_rows(vecs, i0 + (int64_t)(d + u) * kBlock, T.row1);
    cw qv[U], rv[U];
    float wv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + (int64_t)u * kBlock + threadIdx.x;
      if (i < T.row1) {
        qv[u] = Y.qw[i];
        rv[u] = Y.rw[i];
        wv[u] = wnorm32(Y, i);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + (int64_t)u * kBlock + threadIdx.x;
      if (i < T.row1) {
        const cw rn = cw_axpy2(rv[u], ma, qv[u]);
        Y.rw[i] = rn;
        cw_dotu_acc2(rr, rn, rn);
        nrm = fmaf(wv[u], fmaf(rn.rh, rn.rh, rn.ih * rn.ih), nrm);
      }
    }
  }
  const double2 r2 = dacc2_to_double(rr);
  double v[4] = {r2.x, r2.y, (double)nrm, 0.0};
  block_sum<4>(v, sh);
  write_parts(P.part, t, v);
  if (arrive_last(S, Y.ntiles)) {
    cd rho_new, rrn;
    sum_parts(P.part, Y.tile0, Y.ntiles, rho_new, rrn, sh);
    if (threadIdx.x == 0) {
      const double est = sqrt(rrn.re);  // relative to ||r / ||r|| || = 1
      S->est = est;
      S->amode = 0;
      if (est < 0.5 * S->best_est) {
        S->best_est = est;
        S->best_it = S->inner_it;
      }
      if (!(est > inner_stop(P, S)) || S->inner_it >= P.inner_maxit || S->it >= P.maxit || S->bd ||
          (P.stall > 0 && S->inner_it - S->best_it >= P.stall)) {
        S->cmode = C_XUPDATE;
        S->discard = !(est < 1.0);
      } else {
        S->beta = cdiv(rho_new, S->rho);
        S->rho = rho_new;
        S->cmode = C_PUPDATE;
      }
    }
  }
}

__device__ void phaseC_dw(const KParams& P, int t, double* sh) {
  const KTile T = P.tiles[t];
  KState* S = P.st + T.sys;
  if (!vload(&S->act)) return;
  const KSys Y = P.sys[T.sys];
  if (vload(&S->mode) == MODE_RESID) {
    resid_phaseC(P, S, Y);
    return;
  }
  // the step's x += alpha p (deferred from phase B), then p = r + beta p -- or, when the inner
  // solve ends, the refinement update with the finished correction
  const cd al = S->alpha;
  const cws a = to_cws(al.re, al.im);
  if (vload(&S->cmode) == C_PUPDATE) {
    const cd be = S->beta;
    const cws b = to_cws(be.re, be.im);
    const int d = P.pf_chunks;
    const cw* const vecs[3] = {Y.rw, Y.pw, Y.xw};
    if (threadIdx.x == 0)
      for (int j = 0; j < d; ++j) prefetch_rows(vecs, T.row0 + (int64_t)j * kBlock, T.row1);
    constexpr int U = HELM_VEC_UNROLL;
    for (int64_t i0 = T.row0; i0 < T.row1; i0 += U * kBlock) {
      if (threadIdx.x == 0 && d > 0)
#pragma unroll
        for (int u = 0; u < U; ++u) prefetch_rows(vecs, i0 + (int64_t)(d + u) * kBlock, T.row1);
      cw rv[U], pv[U], xv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t i = i0 + (int64_t)u * kBlock + threadIdx.x;
        if (i < T.row1) {
          rv[u] = Y.rw[i];
          pv[u] = Y.pw[i];
          xv[u] = Y.xw[i];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t i = i0 + (int64_t)u * kBlock + threadIdx.x;
        if (i < T.row1) {
          Y.xw[i] = cw_axpy2(xv[u], a, pv[u]);
          Y.pw[i] = cw_axpy2(rv[u], b, pv[u]);
        }
      }
    }
    return;
  }
  // refinement update x += ||r|| d (FP64), d the inner solution after its last step
  const double sc = vload(&S->discard) ? 0.0 : S->rnorm;
  for (int64_t i = T.row0 + threadIdx.x; i < T.row1; i += kBlock) {
    const cw d = cw_axpy2(Y.xw[i], a, Y.pw[i]);
    cd xi = Y.x[i];
    xi.re = fma(sc, join_double(d.rh, d.rl), xi.re);
    xi.im = fma(sc, join_double(d.ih, d.il), xi.im);
    Y.x[i] = xi;
  }
  if (arrive_last(S, Y.ntiles) && threadIdx.x == 0) S->mode = MODE_RESID;
}

// A mixed-precision system that fell back to FP64 COCG (its mode changes only in phase C, after
// every tile of the system has arrived, so all blocks see one mode per step).
__device__ __forceinline__ bool in_fp64(const KParams& P, int t) {
  return vload(&P.st[P.tiles[t].sys].mode) == MODE_FP64;
}

// PREC: 0 = FP64 COCG, 1 = complex64 inner + FP64 refinement, 2 = double-word inner + FP64
// refinement.
template <int PREC, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) cocg_persistent(KParams P) {
  constexpr bool MIXED = PREC != 0;
  __shared__ double sh[4 * (kBlock / 32)];
  __shared__ int sh_int[kBlock / 32];
  const unsigned nb = gridDim.x;
  int seen_fin = 0;
  for (int t = blockIdx.x; t < P.ntiles; t += nb) init_tile(P, t, sh, MIXED);
  if (!grid_barrier(P.bar, nb, P.bar_extra, P.bar_timeout)) return;
  for (int step = 0; step < P.max_steps; ++step) {
    if (vload(&P.ctrl[CTRL_NACT]) == 0) break;
    const int cur = vload(&P.ctrl[CTRL_CUR]);
    const int nat = vload(&P.ctrl[cur ? CTRL_CNT1 : CTRL_CNT0]);
    const int* list = cur ? P.list1 : P.list0;
    bool rebuilt = false;
    if (blockIdx.x == 0) rebuilt = rebuild_list(P, cur, seen_fin, sh_int);
    // phase A of the double-word solve (about 60 us per 4,096-row tile) requests its tiles one at a
    // time: on the 256-lattice sweep the barrier wait after it fell from 66 to 48 us per step
    for_tiles_dynamic(P, 3 * step, nat, list, [&](int t) {
      if (PREC == 1 && !in_fp64(P, t)) phaseA_mixed(P, t, sh);
      else if (PREC == 2 && !in_fp64(P, t)) phaseA_dw(P, t, sh);
      else phaseA_fp64(P, t, sh);
    }, PREC != 2);
    trace_mark(P, step, 0);
    trace_count(P, step, nat);
    if (!grid_barrier(P.bar, nb, P.bar_extra, P.bar_timeout)) return;
    trace_mark(P, step, 1);
    if (rebuilt && threadIdx.x == 0) P.ctrl[CTRL_CUR] = cur ^ 1;
    for_tiles_dynamic(P, 3 * step + 1, nat, list, [&](int t) {
      if (PREC == 1 && !in_fp64(P, t)) phaseB_mixed(P, t, sh);
      else if (PREC == 2 && !in_fp64(P, t)) phaseB_dw(P, t, sh);
      else phaseB_fp64(P, t, sh);
    });
    trace_mark(P, step, 2);
    if (!grid_barrier(P.bar, nb, P.bar_extra, P.bar_timeout)) return;
    trace_mark(P, step, 3);
    for_tiles_dynamic(P, 3 * step + 2, nat, list, [&](int t) {
      if (PREC == 1 && !in_fp64(P, t)) phaseC_mixed(P, t, sh);
      else if (PREC == 2 && !in_fp64(P, t)) phaseC_dw(P, t, sh);
      else phaseC_fp64(P, t, sh);
    });
    trace_mark(P, step, 4);
    if (!grid_barrier(P.bar, nb, P.bar_extra, P.bar_timeout)) return;
    trace_mark(P, step, 5);
  }
}

}  // namespace

namespace eng {
void* cocg_kernel(int prec, int minb) {
  if (prec == 2)
    return minb >= 4 ? (void*)cocg_persistent<2, 4>
         : minb == 3 ? (void*)cocg_persistent<2, 3>
         : minb == 2 ? (void*)cocg_persistent<2, 2> : (void*)cocg_persistent<2, 1>;
  if (prec == 1)
    return minb >= 4 ? (void*)cocg_persistent<1, 4>
         : minb == 3 ? (void*)cocg_persistent<1, 3>
         : minb == 2 ? (void*)cocg_persistent<1, 2> : (void*)cocg_persistent<1, 1>;
  return minb >= 4 ? (void*)cocg_persistent<0, 4>
       : minb == 3 ? (void*)cocg_persistent<0, 3>
       : minb == 2 ? (void*)cocg_persistent<0, 2> : (void*)cocg_persistent<0, 1>;
}
}  // namespace eng
}  // namespace helm
