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
// per-thread dot-product partials converted to FP64 once per phase. Refinement residuals,
// the correction x += ||r|| d and all scalar decisions stay FP64.

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
  dacc dr, di;  // p^T q
  tile_spmv_dw(
      Y.valw, Y.cflag, src, Y.n, Y.Nx, Y.NxNy, T.row0, T.row1,
      [&](int64_t row, cw q, int c) {
        Y.qw[row] = q;
        const cw pi = src[row];
        if (amode) Y.pw[row] = pi;
        if (!c) cw_dotu_acc(dr, di, pi, q);
      },
      [&](int64_t row, cw qi) {
        const cw q = cw_add(Y.qw[row], qi);
        Y.qw[row] = q;
        cw_dotu_acc(dr, di, src[row], q);
      });
  double v[4] = {dr.to_double(), di.to_double(), 0.0, 0.0};
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
    dacc rr_, ri_;
    for (int64_t i = T.row0 + threadIdx.x; i < T.row1; i += kBlock) {
      const cd ri = Y.r[i];
      cw w;
      split_double(ri.re * sc, w.rh, w.rl);
      split_double(ri.im * sc, w.ih, w.il);
      Y.rw[i] = w;
      Y.xw[i] = cw{0.f, 0.f, 0.f, 0.f};
      cw_dotu_acc(rr_, ri_, w, w);
    }
    double v[4] = {rr_.to_double(), ri_.to_double(), 0.0, 0.0};
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
  const cd al = S->alpha;
  const cws a = to_cws(al.re, al.im);
  const cws ma = to_cws(-al.re, -al.im);
  dacc rr_, ri_;
  float nrm = 0.f;  // ||r||^2 for the stopping estimate (FP32 is enough for a threshold test)
  for (int64_t i = T.row0 + threadIdx.x; i < T.row1; i += kBlock) {
    const cw pv = Y.pw[i], qv = Y.qw[i];
    const cw xn = cw_axpy(Y.xw[i], a, pv);
    const cw rn = cw_axpy(Y.rw[i], ma, qv);
    Y.xw[i] = xn;
    Y.rw[i] = rn;
    cw_dotu_acc(rr_, ri_, rn, rn);
    nrm = fmaf(wnorm32(Y, i), fmaf(rn.rh, rn.rh, rn.ih * rn.ih), nrm);
  }
  double v[4] = {rr_.to_double(), ri_.to_double(), (double)nrm, 0.0};
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
  if (vload(&S->cmode) == C_PUPDATE) {
    const cd be = S->beta;
    const cws b = to_cws(be.re, be.im);
    for (int64_t i = T.row0 + threadIdx.x; i < T.row1; i += kBlock) Y.pw[i] = cw_axpy(Y.rw[i], b, Y.pw[i]);
    return;
  }
  // refinement update x += ||r|| d (FP64)
  const double sc = vload(&S->discard) ? 0.0 : S->rnorm;
  for (int64_t i = T.row0 + threadIdx.x; i < T.row1; i += kBlock) {
    const cw d = Y.xw[i];
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
    for (int a = blockIdx.x; a < nat; a += nb) {
      if (PREC == 1 && !in_fp64(P, list[a])) phaseA_mixed(P, list[a], sh);
      else if (PREC == 2 && !in_fp64(P, list[a])) phaseA_dw(P, list[a], sh);
      else phaseA_fp64(P, list[a], sh);
    }
    trace_mark(P, step, 0);
    if (!grid_barrier(P.bar, nb, P.bar_extra, P.bar_timeout)) return;
    trace_mark(P, step, 1);
    if (rebuilt && threadIdx.x == 0) P.ctrl[CTRL_CUR] = cur ^ 1;
    for (int a = blockIdx.x; a < nat; a += nb) {
      if (PREC == 1 && !in_fp64(P, list[a])) phaseB_mixed(P, list[a], sh);
      else if (PREC == 2 && !in_fp64(P, list[a])) phaseB_dw(P, list[a], sh);
      else phaseB_fp64(P, list[a], sh);
    }
    trace_mark(P, step, 2);
    if (!grid_barrier(P.bar, nb, P.bar_extra, P.bar_timeout)) return;
    trace_mark(P, step, 3);
    for (int a = blockIdx.x; a < nat; a += nb) {
      if (PREC == 1 && !in_fp64(P, list[a])) phaseC_mixed(P, list[a], sh);
      else if (PREC == 2 && !in_fp64(P, list[a])) phaseC_dw(P, list[a], sh);
      else phaseC_fp64(P, list[a], sh);
    }
    trace_mark(P, step, 4);
    if (!grid_barrier(P.bar, nb, P.bar_extra, P.bar_timeout)) return;
    trace_mark(P, step, 5);
  }
}

// Simple bump allocator over one device allocation (256-byte aligned pieces).
struct Arena {
  char* base = nullptr;
  size_t off = 0, cap = 0;
  template <typename T> T* take(size_t count) {
    size_t bytes = ((count * sizeof(T)) + 255) & ~(size_t)255;
    T* p = reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};
inline size_t rnd(size_t bytes) { return (bytes + 255) & ~(size_t)255; }

}  // namespace

helm_status solve_cocg_batch(const BatchSystem* sys, int nsys, const helm_solve_opts& o, cudaStream_t s) {
  if (nsys <= 0) return HELM_OK;
  const int prec = o.mixed;  // 0 FP64, 1 complex64 inner, 2 double-word inner
  const bool mixed = prec != 0;
  int dev = 0, nsm = 1;
  HELM_CUDA(cudaGetDevice(&dev));
  HELM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  int coop = 0;
  HELM_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return set_error(HELM_ERR_CUDA, "device does not support cooperative launch");
  // Register budgets: 1 block per SM (255 registers, deep per-thread ILP) up to 4 (64
  // registers, more resident warps); HELM_PERSIST_BLOCKS_PER_SM selects one (tuning knob).
  const char* env = getenv("HELM_PERSIST_BLOCKS_PER_SM");
  const int want = env ? std::max(1, std::min(atoi(env), 4)) : HELM_DEFAULT_BLOCKS_PER_SM;
  const bool bicg = o.solver == HELM_SOLVER_BICGSTAB;
  const bool tfq = o.solver == HELM_SOLVER_TFQMR;
  const bool jac = o.precond == HELM_PRECOND_JACOBI && (bicg || tfq);   // right Jacobi A D^-1
  const bool sjac = o.precond == HELM_PRECOND_JACOBI && !(bicg || tfq);  // symmetric S A S (COCG)
  void (*kern)(KParams) = nullptr;
  if (bicg) kern = reinterpret_cast<void (*)(KParams)>(bicg_kernel(want));
  else if (tfq) kern = reinterpret_cast<void (*)(KParams)>(tfqmr_kernel(want));
  else if (prec == 2)
    kern = want >= 4 ? cocg_persistent<2, 4>
         : want == 3 ? cocg_persistent<2, 3>
         : want == 2 ? cocg_persistent<2, 2> : cocg_persistent<2, 1>;
  else if (want == 4) kern = mixed ? cocg_persistent<1, 4> : cocg_persistent<0, 4>;
  else if (want == 3) kern = mixed ? cocg_persistent<1, 3> : cocg_persistent<0, 3>;
  else if (want == 2) kern = mixed ? cocg_persistent<1, 2> : cocg_persistent<0, 2>;
  else kern = mixed ? cocg_persistent<1, 1> : cocg_persistent<0, 1>;
  int per_sm = 0;
  HELM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, 0));
  if (per_sm < 1) return set_error(HELM_ERR_CUDA, "persistent kernel cannot be resident");
  per_sm = std::min(per_sm, want);
  const int nblocks = nsm * per_sm;

  // tiles: about nblocks tiles for a system that fills the GPU, multiples of 2 * kBlock rows
  // (the SpMV phases give every thread a pair of rows)
  std::vector<KTile> tiles;
  std::vector<int> tile0(nsys), ntl(nsys);
  const int64_t TQ = 2 * kBlock;
  for (int k = 0; k < nsys; ++k) {
    const int64_t n = sys[k].ctx->n;
    const int64_t per = TQ * std::max<int64_t>(1, (n + TQ * nblocks - 1) / (TQ * nblocks));
    tile0[k] = (int)tiles.size();
    for (int64_t r0 = 0; r0 < n; r0 += per) tiles.push_back(KTile{k, 0, r0, std::min(n, r0 + per)});
    ntl[k] = (int)tiles.size() - tile0[k];
  }
  const int ntiles = (int)tiles.size();

  // one arena for every per-system buffer plus the control data
  size_t bytes = 0;
  for (int k = 0; k < nsys; ++k) {
    const size_t n = sys[k].ctx->n, nnz = 27 * n;  // slot-major 27-point values
    bytes += rnd(nnz * sizeof(cd)) + rnd(n * sizeof(cd)) * 2 + rnd(n);  // val, b, r, row flags
    if (prec == 1) bytes += rnd(nnz * sizeof(cf)) + 4 * rnd(n * sizeof(cf));
    if (prec == 2) bytes += rnd(nnz * 2 * sizeof(float2)) + 4 * rnd(n * sizeof(cw));
    bytes += 2 * rnd(n * sizeof(cd));  // p, q (FP64 COCG, also the fallback of the mixed solver)
    if (!(bicg || tfq)) bytes += rnd(n * sizeof(cd));  // best iterate of FP64 COCG
    if (bicg || tfq) bytes += 3 * rnd(n * sizeof(cd));  // rs, s, t (TFQMR: r0*, w, A u)
    if (tfq) bytes += rnd(n * sizeof(cd));              // TFQMR direction d
    if (jac) bytes += rnd(n * sizeof(cd));              // diag(A)
    if (sjac) bytes += rnd(n * sizeof(cd)) + rnd(n * sizeof(double)) + (mixed ? rnd(n * sizeof(float)) : 0);
  }
  const char* tenv = getenv("HELM_TRACE_STEPS");
  const int trace_steps = tenv ? std::max(0, std::min(atoi(tenv), 100000)) : 0;
  bytes += rnd((size_t)trace_steps * 6 * sizeof(unsigned long long));
  bytes += rnd(nsys * sizeof(KSys)) + rnd(nsys * sizeof(KState)) + rnd(ntiles * sizeof(KTile)) +
           2 * rnd(ntiles * sizeof(int)) + rnd(CTRL_N * sizeof(int)) + rnd(2 * (size_t)ntiles * sizeof(cd)) +
           rnd(sizeof(GridBar));
  Arena A;
  A.cap = bytes;
  helm_status st = dev_alloc(&A.base, bytes);
  if (st != HELM_OK) return st;

  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  for (int q = 0; q < 3; ++q) cudaEventCreate(&ev[q]);
  cudaEventRecord(ev[0], s);
  std::vector<KSys> hs(nsys);
  std::vector<KState> hst(nsys);
  for (int k = 0; k < nsys; ++k) {
    const helm_ctx* c = sys[k].ctx;
    KSys& Y = hs[k];
    memset(&Y, 0, sizeof(Y));
    Y.n = c->n;
    Y.Nx = c->mesh.nx + 1;
    Y.NxNy = Y.Nx * (c->mesh.ny + 1);
    cd* val = A.take<cd>(27 * (size_t)c->n);
    cd* b = A.take<cd>(c->n);
    uint8_t* cflag = A.take<uint8_t>(c->n);
    Y.cflag = cflag;
    Y.val = val;
    Y.b = b;
    Y.x = sys[k].p_out;
    Y.r = A.take<cd>(c->n);
    if (prec == 2) {
      Y.valw = A.take<float2>(54 * (size_t)c->n);
      Y.xw = A.take<cw>(c->n);
      Y.rw = A.take<cw>(c->n);
      Y.pw = A.take<cw>(c->n);
      Y.qw = A.take<cw>(c->n);
    }
    if (prec == 1) {
      cf* v32 = A.take<cf>(27 * (size_t)c->n);
      Y.val32 = v32;
      Y.x32 = A.take<cf>(c->n);
      Y.r32 = A.take<cf>(c->n);
      Y.p32 = A.take<cf>(c->n);
      Y.q32 = A.take<cf>(c->n);
    }
    Y.p = A.take<cd>(c->n);
    Y.q = A.take<cd>(c->n);
    if (!(bicg || tfq)) Y.xb = A.take<cd>(c->n);
    if (bicg || tfq) {
      Y.rs = A.take<cd>(c->n);
      Y.sv = A.take<cd>(c->n);
      Y.tv = A.take<cd>(c->n);
    }
    if (tfq) Y.dv = A.take<cd>(c->n);
    if (jac) Y.djac = A.take<cd>(c->n);
    double* wn = nullptr;
    float* wn32 = nullptr;
    if (sjac) {
      Y.jsc = A.take<cd>(c->n);
      wn = A.take<double>(c->n);
      if (mixed) wn32 = A.take<float>(c->n);
      Y.wn = wn;
      Y.wn32 = wn32;
    }
    Y.tile0 = tile0[k];
    Y.ntiles = ntl[k];
    st = assemble_values(c, sys[k].freq, val, b, s, true, /*dia=*/true, cflag);
    if (st == HELM_OK && sys[k].rhs) {
      cudaError_t ce = cudaMemcpyAsync(b, sys[k].rhs, c->n * sizeof(cd), cudaMemcpyDeviceToDevice, s);
      if (ce != cudaSuccess) st = cuda_error(ce, "rhs copy");
    }
    if (st == HELM_OK && sjac)
      st = sym_jacobi_prepare(reinterpret_cast<double*>(val), cflag, b, Y.jsc, wn, wn32, c->n, c->mesh.nx, c->mesh.ny, s);
    if (st == HELM_OK && jac)
      st = jacobi_prepare(reinterpret_cast<double*>(val), cflag, Y.djac, c->n, c->mesh.nx, c->mesh.ny, c->mesh.nz, s);
    if (st == HELM_OK && prec == 1) st = cast_values(val, const_cast<cf*>(Y.val32), 27 * c->n, s);
    if (st == HELM_OK && prec == 2)
      st = split_values(reinterpret_cast<const double*>(val), const_cast<float2*>(Y.valw), 54 * c->n, s);
    if (st != HELM_OK) {
      cudaFree(A.base);
      return st;
    }
    memset(&hst[k], 0, sizeof(KState));
    hst[k].act = 1;
  }
  KSys* d_sys = A.take<KSys>(nsys);
  KState* d_st = A.take<KState>(nsys);
  KTile* d_tiles = A.take<KTile>(ntiles);
  int* d_l0 = A.take<int>(ntiles);
  int* d_l1 = A.take<int>(ntiles);
  int* d_ctrl = A.take<int>(CTRL_N);
  cd* d_part = A.take<cd>(2 * (size_t)ntiles);
  GridBar* d_bar = A.take<GridBar>(1);
  unsigned long long* d_trace = trace_steps ? A.take<unsigned long long>((size_t)trace_steps * 6) : nullptr;
  std::vector<int> l0(ntiles);
  for (int t = 0; t < ntiles; ++t) l0[t] = t;
  int ctrl[CTRL_N] = {0};
  ctrl[CTRL_CUR] = 0;
  ctrl[CTRL_CNT0] = ntiles;
  ctrl[CTRL_NACT] = nsys;
  cudaError_t e = cudaSuccess;
  auto H2D = [&](void* d, const void* h, size_t nb) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(d, h, nb, cudaMemcpyHostToDevice, s);
  };
  H2D(d_sys, hs.data(), nsys * sizeof(KSys));
  H2D(d_st, hst.data(), nsys * sizeof(KState));
  H2D(d_tiles, tiles.data(), ntiles * sizeof(KTile));
  H2D(d_l0, l0.data(), ntiles * sizeof(int));
  H2D(d_ctrl, ctrl, sizeof(ctrl));
  if (e == cudaSuccess) e = cudaMemsetAsync(d_bar, 0, sizeof(GridBar), s);

  KParams P;
  P.sys = d_sys;
  P.st = d_st;
  P.tiles = d_tiles;
  P.ntiles = ntiles;
  P.list0 = d_l0;
  P.list1 = d_l1;
  P.ctrl = d_ctrl;
  P.part = d_part;
  P.bar = d_bar;
  P.tol = o.tol;
  P.maxit = o.maxit;
  P.inner_tol = o.inner_tol;
  P.inner_maxit = o.inner_maxit;
  P.max_outer = o.max_outer;
  P.stall = o.stall_window;
  P.trace = d_trace;
  P.trace_steps = trace_steps;
  // Host-side fault injection for tests (never set in normal use): the barriers wait for one
  // block that does not exist and give up after 200 ms, so the launch ends with HELM_TIMEOUT
  // without faulting or hanging the GPU.
  const FaultMode fm = fault_mode();
  P.bar_extra = fm == FAULT_BARRIER ? 1u : 0u;
  P.bar_timeout = fm == FAULT_BARRIER ? 200000000ull : kTimeoutNs;
  // each super-step advances every active system by one Krylov step (one BiCGSTAB iteration),
  // except refinement residual steps (at most max_outer + 1 of them) and residual checks
  P.max_steps = 2 * o.maxit + 2 * (o.max_outer + 2) + 16;
  if (tfq) P.max_steps = 6 * o.maxit + 16;  // one barrier per sub-step, at most 4 per restart cycle
  void* args[] = {&P};
  if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
  if (e == cudaSuccess)
    e = cudaLaunchCooperativeKernel((const void*)kern, dim3(nblocks), dim3(kBlock), args, 0, s);
  if (e == cudaSuccess) e = cudaEventRecord(ev[2], s);
  // back to the unknowns of A x = b (also for a system that did not converge: its best iterate)
  if (jac)  // x = D^-1 y
    for (int k = 0; k < nsys && e == cudaSuccess; ++k)
      if (jacobi_unscale(hs[k].x, hs[k].djac, hs[k].n, s) != HELM_OK) e = cudaGetLastError();
  if (sjac)  // x = S y
    for (int k = 0; k < nsys && e == cudaSuccess; ++k)
      if (jacobi_rescale(hs[k].x, hs[k].jsc, hs[k].n, s) != HELM_OK) e = cudaGetLastError();
  GridBar hb;
  memset(&hb, 0, sizeof(hb));
  if (e == cudaSuccess) e = cudaMemcpyAsync(hst.data(), d_st, nsys * sizeof(KState), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, d_bar, sizeof(GridBar), cudaMemcpyDeviceToHost, s);
  std::vector<unsigned long long> htrace((size_t)trace_steps * 6);
  if (e == cudaSuccess && trace_steps)
    e = cudaMemcpyAsync(htrace.data(), d_trace, htrace.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(A.base);
  if (e == cudaSuccess && trace_steps > 1) {
    // mean durations (us) over the traced steps: own work of A, wait at barrier A, B work, B
    // wait, C work, C wait (block 0's view)
    double acc[6] = {0, 0, 0, 0, 0, 0};
    int cnt = 0;
    for (int k = 1; k < trace_steps; ++k) {
      const unsigned long long* t = &htrace[(size_t)k * 6];
      const unsigned long long prev = htrace[(size_t)(k - 1) * 6 + 5];
      if (t[5] == 0 || prev == 0) break;
      acc[0] += (double)(t[0] - prev); acc[1] += (double)(t[1] - t[0]);
      acc[2] += (double)(t[2] - t[1]); acc[3] += (double)(t[3] - t[2]);
      acc[4] += (double)(t[4] - t[3]); acc[5] += (double)(t[5] - t[4]);
      ++cnt;
    }
    if (cnt)
      fprintf(stderr, "helm trace (%d steps, us): A work %.2f wait %.2f | B work %.2f wait %.2f | C work %.2f wait %.2f\n",
              cnt, acc[0] / cnt / 1e3, acc[1] / cnt / 1e3, acc[2] / cnt / 1e3, acc[3] / cnt / 1e3, acc[4] / cnt / 1e3,
              acc[5] / cnt / 1e3);
  }
  if (e == cudaSuccess) {
    float t_asm = 0.f, t_solve = 0.f;
    cudaEventElapsedTime(&t_asm, ev[0], ev[1]);
    cudaEventElapsedTime(&t_solve, ev[1], ev[2]);
    helm_profile& pr = last_profile();
    pr.assemble_ms += t_asm;
    pr.solve_ms += t_solve;
    pr.launches += (int64_t)nsys * (mixed ? 2 : 1) + 1;
    pr.grid_blocks = nblocks;
    pr.ntiles = ntiles;
  }
  for (int q = 0; q < 3; ++q) cudaEventDestroy(ev[q]);
  if (e != cudaSuccess) return cuda_error(e, "cocg persistent solve");

  helm_status overall = HELM_OK;
  const bool dbg = getenv("HELM_DEBUG_STATE") != nullptr;  // diagnosis aid: state of failed systems
  for (int k = 0; k < nsys; ++k) {
    helm_solve_stats& S = *sys[k].stats;
    const KState& K = hst[k];
    if (dbg && (K.act || K.status != HELM_OK))
      fprintf(stderr,
              "helm state sys %d: status %d it %d bd %d est %.3e relres %.3e rho (%.3e,%.3e) alpha (%.3e,%.3e) "
              "omega (%.3e,%.3e) beta (%.3e,%.3e) tau %.3e theta %.3e\n",
              k, K.status, K.it, K.bd, K.est, K.relres, K.rho.re, K.rho.im, K.alpha.re, K.alpha.im, K.omega.re,
              K.omega.im, K.beta.re, K.beta.im, K.tau, K.theta);
    S.status = K.act ? HELM_NOT_CONVERGED : K.status;
    if (hb.status & DEV_TIMEOUT) S.status = HELM_TIMEOUT;
    S.iterations = K.it;
    S.restarts = K.restarts;
    S.outer = K.fell_back ? -K.outer : K.outer;
    S.iterations_c64 = K.it32;
    S.pad = 0;
    S.relres = K.relres;
    S.bnorm = K.bnorm;
    if (S.status != HELM_OK && overall == HELM_OK) overall = (helm_status)S.status;
  }
  if (hb.status & DEV_TIMEOUT) return set_error(HELM_TIMEOUT, "persistent solver: grid barrier timed out");
  if (overall != HELM_OK) set_error(overall, "at least one system did not converge");
  return overall;
}

}  // namespace helm
