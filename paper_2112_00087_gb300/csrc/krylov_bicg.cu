// BiCGSTAB and TFQMR in the persistent batched engine (krylov_engine.cuh), the paper's own
// Sec. 4 solvers (Table 3: P-BiCGSTAB, P-tfQMR), with optional right Jacobi preconditioning
// ("P" is not named in the paper; Jacobi is the reading taken): the matrix is assembled as
// A D^-1 (columns scaled once), the solver runs on it unchanged, and x = D^-1 y at the end, so
// every residual the solver computes is the residual of A x = b.
#include <algorithm>

#include "krylov_engine.cuh"

namespace helm {
namespace {
using namespace eng;

// ------------------------------- BiCGSTAB phases (FP64) ---------------------------------------
// Paper Sec. 4 (Table 3: P-BiCGSTAB; the preconditioner "P" is not named, none is applied).
// (u, v) = v^H u; one iteration = phases A1 (v = A p, rs^H v -> alpha), B1 (s = r - alpha v),
// A2 (t = A s, t^H s, t^H t -> omega), B2 (x, r updates, rs^H r, ||r||^2 -> beta or check),
// C (p = r + beta (p - omega v), or the true residual and a restart with rs = p = r).

__device__ void bi_init(const KParams& P, int t, double* sh) {
  const KTile T = P.tiles[t];
  KState* S = P.st + T.sys;
  const KSys Y = P.sys[T.sys];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = T.row0 + threadIdx.x; i < T.row1; i += kBlock) {
    const cd bi = Y.b[i];
    Y.x[i] = cd(0.0, 0.0);
    Y.r[i] = bi;
    v[2] += bi.re * bi.re + bi.im * bi.im;
  }
  block_sum<4>(v, sh);
  write_parts(P.part, t, v);
  if (arrive_last(S, Y.ntiles)) {
    cd u, rr;
    sum_parts(P.part, Y.tile0, Y.ntiles, u, rr, sh);
    if (threadIdx.x == 0) {
      S->bnorm = sqrt(rr.re);
      S->rho = cd(rr.re, 0.0);  // (r, rs) with rs = r
      S->amode = 1;
      if (S->bnorm == 0.0) finish(P, S, HELM_OK, 0.0);
    }
  }
}

__device__ void bi_A1(const KParams& P, int t, double* sh) {
  const KTile T = P.tiles[t];
  KState* S = P.st + T.sys;
  if (!vload(&S->act)) return;
  const KSys Y = P.sys[T.sys];
  const int amode = vload(&S->amode);
  const cd* src = amode ? Y.r : Y.p;  // restart: p := r, rs := r
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  tile_spmv<double>(
      Y.val, Y.cflag, src, Y.n, Y.Nx, Y.NxNy, T.row0, T.row1,
      [&](int64_t row, cd q, int) {
        Y.q[row] = q;
        const cd ri = src[row];
        if (amode) { Y.p[row] = ri; Y.rs[row] = ri; }
        const cd rsi = amode ? ri : Y.rs[row];
        v[0] += rsi.re * q.re + rsi.im * q.im;  // conj(rs) v
        v[1] += rsi.re * q.im - rsi.im * q.re;
      },
      [&](int64_t row, cd qi) {
        const cd q0 = Y.q[row];
        Y.q[row] = cd(q0.re + qi.re, q0.im + qi.im);
        const cd rsi = Y.rs[row];  // written by this thread in the first pass when restarting
        v[0] += rsi.re * qi.re + rsi.im * qi.im;
        v[1] += rsi.re * qi.im - rsi.im * qi.re;
      });
  block_sum<4>(v, sh);
  write_parts(P.part, t, v);
  if (arrive_last(S, Y.ntiles)) {
    cd den, unused;
    sum_parts(P.part, Y.tile0, Y.ntiles, den, unused, sh);
    if (threadIdx.x == 0) {
      S->it += 1;
      const cd rho = S->rho;
      if ((den.re == 0.0 && den.im == 0.0) || (rho.re == 0.0 && rho.im == 0.0)) {
        S->bd = 1;
        S->alpha = cd(0.0, 0.0);
      } else {
        S->alpha = cdiv(rho, den);
      }
    }
  }
}

__device__ void bi_B1(const KParams& P, int t) {
  const KTile T = P.tiles[t];
  KState* S = P.st + T.sys;
  if (!vload(&S->act)) return;
  const KSys Y = P.sys[T.sys];
  const cd al = S->alpha;
  const cd mal(-al.re, -al.im);
  for (int64_t i = T.row0 + threadIdx.x; i < T.row1; i += kBlock) {
    cd si = Y.r[i];
    cfma(si, mal, Y.q[i]);
    Y.sv[i] = si;
  }
}

__device__ void bi_A2(const KParams& P, int t, double* sh) {
  const KTile T = P.tiles[t];
  KState* S = P.st + T.sys;
  if (!vload(&S->act)) return;
  const KSys Y = P.sys[T.sys];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  tile_spmv<double>(
      Y.val, Y.cflag, Y.sv, Y.n, Y.Nx, Y.NxNy, T.row0, T.row1,
      [&](int64_t row, cd q, int c) {
        Y.tv[row] = q;
        if (!c) {
          const cd si = Y.sv[row];
          v[0] += q.re * si.re + q.im * si.im;  // conj(t) s
          v[1] += q.re * si.im - q.im * si.re;
          v[2] += q.re * q.re + q.im * q.im;
        }
      },
      [&](int64_t row, cd qi) {
        const cd q0 = Y.tv[row];
        const cd q(q0.re + qi.re, q0.im + qi.im);
        Y.tv[row] = q;
        const cd si = Y.sv[row];
        v[0] += q.re * si.re + q.im * si.im;
        v[1] += q.re * si.im - q.im * si.re;
        v[2] += q.re * q.re + q.im * q.im;
      });
  block_sum<4>(v, sh);
  write_parts(P.part, t, v);
  if (arrive_last(S, Y.ntiles)) {
    cd ts, tt;
    sum_parts(P.part, Y.tile0, Y.ntiles, ts, tt, sh);
    if (threadIdx.x == 0) S->omega = tt.re == 0.0 ? cd(0.0, 0.0) : cd(ts.re / tt.re, ts.im / tt.re);
  }
}

__device__ void bi_B2(const KParams& P, int t, double* sh) {
  const KTile T = P.tiles[t];
  KState* S = P.st + T.sys;
  if (!vload(&S->act)) return;
  const KSys Y = P.sys[T.sys];
  const cd al = S->alpha, om = S->omega;
  const cd mom(-om.re, -om.im);
  const bool bd = S->bd;  // (rs, v) or rho vanished in A1: x and r stay as they are
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = T.row0 + threadIdx.x; i < T.row1 && !bd; i += kBlock) {
    cd xi = Y.x[i];
    const cd si = Y.sv[i];
    cfma(xi, al, Y.p[i]);
    cfma(xi, om, si);
    Y.x[i] = xi;
    cd ri = si;
    cfma(ri, mom, Y.tv[i]);
    Y.r[i] = ri;
    const cd rsi = Y.rs[i];
    v[0] += rsi.re * ri.re + rsi.im * ri.im;  // conj(rs) r
    v[1] += rsi.re * ri.im - rsi.im * ri.re;
    v[2] += ri.re * ri.re + ri.im * ri.im;
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
      const bool om0 = (om.re == 0.0 && om.im == 0.0);
      if (bd || !(est > P.tol) || S->it >= P.maxit || om0) {
        if (om0 && est > P.tol) S->bd = 1;
        S->cmode = C_CHECK;
      } else {
        S->beta = cdiv(rho_new, S->rho) * cdiv(al, om);
        S->rho = rho_new;
        S->cmode = C_PUPDATE;
      }
    }
  }
}

__device__ void bi_C(const KParams& P, int t, double* sh) {
  const KTile T = P.tiles[t];
  KState* S = P.st + T.sys;
  if (!vload(&S->act)) return;
  const KSys Y = P.sys[T.sys];
  if (vload(&S->cmode) == C_PUPDATE) {
    const cd be = S->beta, om = S->omega;
    const cd mom(-om.re, -om.im);
    for (int64_t i = T.row0 + threadIdx.x; i < T.row1; i += kBlock) {
      cd w = Y.p[i];  // p - omega v
      cfma(w, mom, Y.q[i]);
      cd pn = Y.r[i];
      cfma(pn, be, w);
      Y.p[i] = pn;
    }
    return;
  }
  // true residual; restart with rs = p = r, rho = ||r||^2
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  tile_spmv<double>(
      Y.val, Y.cflag, Y.x, Y.n, Y.Nx, Y.NxNy, T.row0, T.row1,
      [&](int64_t row, cd s, int c) {
        const cd bi = Y.b[row];
        const cd ri(bi.re - s.re, bi.im - s.im);
        Y.r[row] = ri;
        if (!c) v[2] += ri.re * ri.re + ri.im * ri.im;
      },
      [&](int64_t row, cd si) {
        const cd r0 = Y.r[row];
        const cd ri(r0.re - si.re, r0.im - si.im);
        Y.r[row] = ri;
        v[2] += ri.re * ri.re + ri.im * ri.im;
      });
  block_sum<4>(v, sh);
  write_parts(P.part, t, v);
  if (arrive_last(S, Y.ntiles)) {
    cd u, rr;
    sum_parts(P.part, Y.tile0, Y.ntiles, u, rr, sh);
    if (threadIdx.x == 0) {
      const double rel = sqrt(rr.re) / S->bnorm;
      S->relres = rel;
      if (rel <= P.tol) finish(P, S, HELM_OK, rel);
      else if (!(rel == rel)) finish(P, S, HELM_NAN, rel);
      else if (S->it >= P.maxit) finish(P, S, HELM_NOT_CONVERGED, rel);
      else if (S->bd) finish(P, S, HELM_BREAKDOWN, rel);
      else {
        S->rho = cd(rr.re, 0.0);
        S->amode = 1;
        S->restarts += 1;
      }
    }
  }
}

template <int MINB>
__global__ void __launch_bounds__(kBlock, MINB) bicg_persistent(KParams P) {
  __shared__ double sh[4 * (kBlock / 32)];
  __shared__ int sh_int[kBlock / 32];
  const unsigned nb = gridDim.x;
  int seen_fin = 0;
  for (int t = blockIdx.x; t < P.ntiles; t += nb) bi_init(P, t, sh);
  if (!grid_barrier(P.bar, nb, P.bar_extra, P.bar_timeout)) return;
  for (int step = 0; step < P.max_steps; ++step) {
    if (vload(&P.ctrl[CTRL_NACT]) == 0) break;
    const int cur = vload(&P.ctrl[CTRL_CUR]);
    const int nat = vload(&P.ctrl[cur ? CTRL_CNT1 : CTRL_CNT0]);
    const int* list = cur ? P.list1 : P.list0;
    bool rebuilt = false;
    if (blockIdx.x == 0) rebuilt = rebuild_list(P, cur, seen_fin, sh_int);
    for (int a = blockIdx.x; a < nat; a += nb) bi_A1(P, list[a], sh);
    if (!grid_barrier(P.bar, nb, P.bar_extra, P.bar_timeout)) return;
    if (rebuilt && threadIdx.x == 0) P.ctrl[CTRL_CUR] = cur ^ 1;
    for (int a = blockIdx.x; a < nat; a += nb) bi_B1(P, list[a]);
    if (!grid_barrier(P.bar, nb, P.bar_extra, P.bar_timeout)) return;
    for (int a = blockIdx.x; a < nat; a += nb) bi_A2(P, list[a], sh);
    if (!grid_barrier(P.bar, nb, P.bar_extra, P.bar_timeout)) return;
    for (int a = blockIdx.x; a < nat; a += nb) bi_B2(P, list[a], sh);
    if (!grid_barrier(P.bar, nb, P.bar_extra, P.bar_timeout)) return;
    for (int a = blockIdx.x; a < nat; a += nb) bi_C(P, list[a], sh);
    if (!grid_barrier(P.bar, nb, P.bar_extra, P.bar_timeout)) return;
  }
}


// ------------------------------- TFQMR (FP64) --------------------------------------------------
// Paper Sec. 4 (Table 3: P-tfQMR). Transpose-free QMR, (u, v) = v^H u, r0* = r0. Steps m = 0, 1,
// ...: even steps renew alpha = rho / (r0*, v) and u <- u - alpha v; every step
// w <- w - alpha A u, d <- u + (theta^2 / alpha) eta d, theta = ||w|| / tau,
// c = (1 + theta^2)^-1/2, tau <- tau theta c, eta = c^2 alpha, x <- x + eta d; odd steps renew
// rho = (w, r0*), beta, u <- w + beta u and v <- A u + beta (A u_old + beta v). The estimate
// tau sqrt(m + 1) / ||b|| stops the iteration, the true residual decides (a miss restarts from x).
//
// Engine layout: a per-system state machine with ONE grid barrier per super-step; each active
// system executes its current sub-step (T_*), its last arriving tile takes the scalar decisions
// and sets the next sub-step. The x update x += eta d of a step needs that step's eta (known
// only after its reduction), so it is applied by the following sub-step, row by row, before d
// changes. One pair of steps = T_EVEN, T_ODD, T_U, T_V: four super-steps, two SpMVs.
// Vectors: w = sv, u = p, v = q, A u = tv (A u_m of the current step), d = dv, r0* = rs.

enum : int { T_SETUP = 0, T_V0 = 1, T_EVEN = 2, T_ODD = 3, T_U = 4, T_V = 5, T_XC = 6, T_RES = 7 };

__device__ void tq_init(const KParams& P, int t, double* sh) {
  const KTile T = P.tiles[t];
  KState* S = P.st + T.sys;
  const KSys Y = P.sys[T.sys];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = T.row0 + threadIdx.x; i < T.row1; i += kBlock) {
    const cd bi = Y.b[i];
    Y.x[i] = cd(0.0, 0.0);
    Y.r[i] = bi;
    v[2] += bi.re * bi.re + bi.im * bi.im;
  }
  block_sum<4>(v, sh);
  write_parts(P.part, t, v);
  if (arrive_last(S, Y.ntiles)) {
    cd u, rr;
    sum_parts(P.part, Y.tile0, Y.ntiles, u, rr, sh);
    if (threadIdx.x == 0) {
      S->bnorm = sqrt(rr.re);
      S->tstate = T_SETUP;
      if (S->bnorm == 0.0) finish(P, S, HELM_OK, 0.0);
    }
  }
}

// (re) start from r: w = u = r0* = r, d = 0, tau = ||r||, rho = ||r||^2, theta = eta = 0
__device__ void tq_setup(const KParams& P, int t, double* sh, const KTile& T, KState* S, const KSys& Y) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = T.row0 + threadIdx.x; i < T.row1; i += kBlock) {
    const cd ri = Y.r[i];
    Y.sv[i] = ri;
    Y.p[i] = ri;
    Y.rs[i] = ri;
    Y.dv[i] = cd(0.0, 0.0);
    v[2] += ri.re * ri.re + ri.im * ri.im;
  }
  block_sum<4>(v, sh);
  write_parts(P.part, t, v);
  if (arrive_last(S, Y.ntiles)) {
    cd u, rr;
    sum_parts(P.part, Y.tile0, Y.ntiles, u, rr, sh);
    if (threadIdx.x == 0) {
      S->tau = sqrt(rr.re);
      S->rho = cd(rr.re, 0.0);
      S->theta = 0.0;
      S->eta = cd(0.0, 0.0);
      S->inner_it = 0;
      S->tstate = T_V0;
    }
  }
}

// v = A u (+ beta (A u_old + beta v) after an odd step), A u kept for the even step, then
// alpha = rho / (r0*, v)
__device__ void tq_v(const KParams& P, int t, double* sh, const KTile& T, KState* S, const KSys& Y, bool first) {
  const cd be = first ? cd(0.0, 0.0) : S->beta;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  auto row_done = [&](int64_t row, cd au) {
    cd vn = au;
    if (!first) {
      cd w = Y.tv[row];  // A u_old + beta v_old
      cfma(w, be, Y.q[row]);
      cfma(vn, be, w);
    }
    Y.tv[row] = au;  // A u of the coming even step
    Y.q[row] = vn;
    const cd rsi = Y.rs[row];
    v[0] += rsi.re * vn.re + rsi.im * vn.im;
    v[1] += rsi.re * vn.im - rsi.im * vn.re;
  };
  tile_spmv<double>(
      Y.val, Y.cflag, Y.p, Y.n, Y.Nx, Y.NxNy, T.row0, T.row1,
      [&](int64_t row, cd q, int c) {
        if (c) Y.r[row] = q;  // flagged rows finish in the second pass (r is free until the next check)
        else row_done(row, q);
      },
      [&](int64_t row, cd qi) {
        const cd q0 = Y.r[row];
        row_done(row, cd(q0.re + qi.re, q0.im + qi.im));
      });
  block_sum<4>(v, sh);
  write_parts(P.part, t, v);
  if (arrive_last(S, Y.ntiles)) {
    cd den, unused;
    sum_parts(P.part, Y.tile0, Y.ntiles, den, unused, sh);
    if (threadIdx.x == 0) {
      const cd rho = S->rho;
      if ((den.re == 0.0 && den.im == 0.0) || (rho.re == 0.0 && rho.im == 0.0)) {
        S->bd = 1;
        S->tstate = T_RES;  // x is current: no step pending
      } else {
        S->alpha = cdiv(rho, den);
        S->tstate = T_EVEN;
      }
    }
  }
}

// theta, c, tau, eta after a step whose ||w||^2 is ww; returns the stopping estimate
__device__ __forceinline__ double tq_scalars(KState* S, double ww) {
  const double th = sqrt(ww) / S->tau;
  const double c = 1.0 / sqrt(1.0 + th * th);
  S->theta = th;
  S->tau = S->tau * th * c;
  S->eta = cd(c * c * S->alpha.re, c * c * S->alpha.im);
  S->it += 1;
  return S->tau * sqrt((double)S->inner_it + 1.0) / S->bnorm;
}

__device__ void tq_even(const KParams& P, int t, double* sh, const KTile& T, KState* S, const KSys& Y) {
  const cd al = S->alpha, mal(-al.re, -al.im);
  const cd f = cdiv(cd(S->theta * S->theta * S->eta.re, S->theta * S->theta * S->eta.im), al);
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = T.row0 + threadIdx.x; i < T.row1; i += kBlock) {
    const cd ui = Y.p[i], vi = Y.q[i];
    cd di = ui;
    cfma(di, f, Y.dv[i]);  // d = u + (theta^2 / alpha) eta d
    Y.dv[i] = di;
    cd un = ui;
    cfma(un, mal, vi);     // u - alpha v
    Y.p[i] = un;
    cd wn = Y.sv[i];
    cfma(wn, mal, Y.tv[i]);  // w - alpha A u_m
    Y.sv[i] = wn;
    v[2] += wn.re * wn.re + wn.im * wn.im;
  }
  block_sum<4>(v, sh);
  write_parts(P.part, t, v);
  if (arrive_last(S, Y.ntiles)) {
    cd u, ww;
    sum_parts(P.part, Y.tile0, Y.ntiles, u, ww, sh);
    if (threadIdx.x == 0) {
      const double est = tq_scalars(S, ww.re);
      S->est = est;
      if (!(est > P.tol) || S->it >= P.maxit) {
        S->tstate = T_XC;
      } else {
        S->inner_it += 1;
        S->tstate = T_ODD;
      }
    }
  }
}

__device__ void tq_odd(const KParams& P, int t, double* sh, const KTile& T, KState* S, const KSys& Y) {
  const cd al = S->alpha, mal(-al.re, -al.im);
  const cd eta = S->eta;  // of the even step: its x update is applied here
  const cd f = cdiv(cd(S->theta * S->theta * eta.re, S->theta * S->theta * eta.im), al);
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  auto row_done = [&](int64_t row, cd au) {
    Y.tv[row] = au;
    const cd dold = Y.dv[row];
    cd xi = Y.x[row];
    cfma(xi, eta, dold);
    Y.x[row] = xi;
    cd di = Y.p[row];
    cfma(di, f, dold);
    Y.dv[row] = di;
    cd wn = Y.sv[row];
    cfma(wn, mal, au);
    Y.sv[row] = wn;
    const cd rsi = Y.rs[row];
    v[0] += rsi.re * wn.re + rsi.im * wn.im;  // (w, r0*) = r0*^H w
    v[1] += rsi.re * wn.im - rsi.im * wn.re;
    v[2] += wn.re * wn.re + wn.im * wn.im;
  };
  tile_spmv<double>(
      Y.val, Y.cflag, Y.p, Y.n, Y.Nx, Y.NxNy, T.row0, T.row1,
      [&](int64_t row, cd q, int c) {
        if (c) Y.tv[row] = q;
        else row_done(row, q);
      },
      [&](int64_t row, cd qi) {
        const cd q0 = Y.tv[row];
        row_done(row, cd(q0.re + qi.re, q0.im + qi.im));
      });
  block_sum<4>(v, sh);
  write_parts(P.part, t, v);
  if (arrive_last(S, Y.ntiles)) {
    cd rho_new, ww;
    sum_parts(P.part, Y.tile0, Y.ntiles, rho_new, ww, sh);
    if (threadIdx.x == 0) {
      const double est = tq_scalars(S, ww.re);
      S->est = est;
      const cd rho = S->rho;
      if (!(est > P.tol) || S->it >= P.maxit) {
        S->tstate = T_XC;
      } else if (rho.re == 0.0 && rho.im == 0.0) {
        S->bd = 1;
        S->tstate = T_XC;
      } else {
        S->beta = cdiv(rho_new, rho);
        S->rho = rho_new;
        S->inner_it += 1;
        S->tstate = T_U;
      }
    }
  }
}

// x += eta d (odd step), u = w + beta u
__device__ void tq_u(const KParams& P, const KTile& T, KState* S, const KSys& Y) {
  const cd eta = S->eta, be = S->beta;
  for (int64_t i = T.row0 + threadIdx.x; i < T.row1; i += kBlock) {
    cd xi = Y.x[i];
    cfma(xi, eta, Y.dv[i]);
    Y.x[i] = xi;
    cd un = Y.sv[i];
    cfma(un, be, Y.p[i]);
    Y.p[i] = un;
  }
  if (arrive_last(S, Y.ntiles) && threadIdx.x == 0) S->tstate = T_V;
}

// pending x += eta d before a true-residual check
__device__ void tq_xc(const KParams& P, const KTile& T, KState* S, const KSys& Y) {
  const cd eta = S->eta;
  for (int64_t i = T.row0 + threadIdx.x; i < T.row1; i += kBlock) {
    cd xi = Y.x[i];
    cfma(xi, eta, Y.dv[i]);
    Y.x[i] = xi;
  }
  if (arrive_last(S, Y.ntiles) && threadIdx.x == 0) S->tstate = T_RES;
}

__device__ void tq_res(const KParams& P, int t, double* sh, const KTile& T, KState* S, const KSys& Y) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  tile_spmv<double>(
      Y.val, Y.cflag, Y.x, Y.n, Y.Nx, Y.NxNy, T.row0, T.row1,
      [&](int64_t row, cd s, int c) {
        const cd bi = Y.b[row];
        const cd ri(bi.re - s.re, bi.im - s.im);
        Y.r[row] = ri;
        if (!c) v[2] += ri.re * ri.re + ri.im * ri.im;
      },
      [&](int64_t row, cd si) {
        const cd r0 = Y.r[row];
        const cd ri(r0.re - si.re, r0.im - si.im);
        Y.r[row] = ri;
        v[2] += ri.re * ri.re + ri.im * ri.im;
      });
  block_sum<4>(v, sh);
  write_parts(P.part, t, v);
  if (arrive_last(S, Y.ntiles)) {
    cd u, rr;
    sum_parts(P.part, Y.tile0, Y.ntiles, u, rr, sh);
    if (threadIdx.x == 0) {
      const double rel = sqrt(rr.re) / S->bnorm;
      S->relres = rel;
      if (rel <= P.tol) finish(P, S, HELM_OK, rel);
      else if (!(rel == rel)) finish(P, S, HELM_NAN, rel);
      else if (S->it >= P.maxit) finish(P, S, HELM_NOT_CONVERGED, rel);
      else if (S->bd) finish(P, S, HELM_BREAKDOWN, rel);
      else {
        S->restarts += 1;
        S->tstate = T_SETUP;
      }
    }
  }
}

__device__ void tq_step(const KParams& P, int t, double* sh) {
  const KTile T = P.tiles[t];
  KState* S = P.st + T.sys;
  if (!vload(&S->act)) return;
  const KSys Y = P.sys[T.sys];
  switch (vload(&S->tstate)) {
    case T_SETUP: tq_setup(P, t, sh, T, S, Y); break;
    case T_V0: tq_v(P, t, sh, T, S, Y, true); break;
    case T_EVEN: tq_even(P, t, sh, T, S, Y); break;
    case T_ODD: tq_odd(P, t, sh, T, S, Y); break;
    case T_U: tq_u(P, T, S, Y); break;
    case T_V: tq_v(P, t, sh, T, S, Y, false); break;
    case T_XC: tq_xc(P, T, S, Y); break;
    default: tq_res(P, t, sh, T, S, Y); break;
  }
}

// One grid barrier per super-step. The tile list for step s is list[ctrl[CTRL_P0 + (s & 1)]]:
// block 0 writes the choice for step s + 1 during step s (before the barrier), and the slot it
// writes is never the one any block reads during the same step.
template <int MINB>
__global__ void __launch_bounds__(kBlock, MINB) tfqmr_persistent(KParams P) {
  __shared__ double sh[4 * (kBlock / 32)];
  __shared__ int sh_int[kBlock / 32];
  const unsigned nb = gridDim.x;
  int seen_fin = 0;
  for (int t = blockIdx.x; t < P.ntiles; t += nb) tq_init(P, t, sh);
  if (!grid_barrier(P.bar, nb, P.bar_extra, P.bar_timeout)) return;
  for (int step = 0; step < P.max_steps; ++step) {
    if (vload(&P.ctrl[CTRL_NACT]) == 0) break;
    const int cur = vload(&P.ctrl[CTRL_P0 + (step & 1)]);
    const int nat = vload(&P.ctrl[cur ? CTRL_CNT1 : CTRL_CNT0]);
    const int* list = cur ? P.list1 : P.list0;
    if (blockIdx.x == 0) {
      const bool rebuilt = rebuild_list(P, cur, seen_fin, sh_int);
      if (threadIdx.x == 0) P.ctrl[CTRL_P0 + ((step + 1) & 1)] = rebuilt ? cur ^ 1 : cur;
    }
    for (int a = blockIdx.x; a < nat; a += nb) tq_step(P, list[a], sh);
    if (!grid_barrier(P.bar, nb, P.bar_extra, P.bar_timeout)) return;
  }
}

// ------------------------------- right Jacobi ---------------------------------------------------

__global__ void jacobi_diag_kernel(const double* __restrict__ val, cd* __restrict__ djac, int64_t n) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row < n) djac[row] = cd(val[13 * n + row], val[27 * n + 13 * n + row]);
}

// column scaling A D^-1: entry (row, c) divided by djac[c]; row flag = any non-zero imaginary part
__global__ void jacobi_scale_kernel(double* __restrict__ val, uint8_t* __restrict__ cflag,
                                    const cd* __restrict__ djac, int64_t n, int64_t Nx, int64_t NxNy) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= n) return;
  int cplx_row = 0;
  for (int k = 0; k < 27; ++k) {
    const int di = k % 3 - 1, dj = (k / 3) % 3 - 1, dl = k / 9 - 1;
    int64_t c = row + di + Nx * dj + NxNy * dl;
    c = c < 0 ? 0 : (c >= n ? n - 1 : c);  // padded slots hold 0 and stay 0
    const int64_t e = (int64_t)k * n + row;
    const cd a(val[e], val[27 * n + e]);
    const cd q = cdiv(a, djac[c]);
    val[e] = q.re;
    val[27 * n + e] = q.im;
    cplx_row |= (q.im != 0.0);
  }
  cflag[row] = (uint8_t)cplx_row;
}

__global__ void jacobi_unscale_kernel(cd* __restrict__ x, const cd* __restrict__ djac, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] = cdiv(x[i], djac[i]);
}

// ------------------------------- symmetric Jacobi (COCG) ---------------------------------------

// principal square root of a + ib: for a >= 0, t = sqrt((|z| + a) / 2) and sqrt(z) = t + i b/(2t);
// for a < 0, t = sqrt((|z| - a) / 2) and sqrt(z) = |b|/(2t) + i sign(b) t (no cancellation)
__device__ __forceinline__ cd csqrt_principal(cd z) {
  const double r = hypot(z.re, z.im);
  if (r == 0.0) return cd(0.0, 0.0);
  if (z.re >= 0.0) {
    const double t = sqrt(0.5 * (r + z.re));
    return cd(t, z.im / (2.0 * t));
  }
  const double t = sqrt(0.5 * (r - z.re));
  return cd(fabs(z.im) / (2.0 * t), copysign(t, z.im));
}

__global__ void sym_jacobi_diag_kernel(const double* __restrict__ val, cd* __restrict__ jsc, double* __restrict__ wn,
                                       float* __restrict__ wn32, int64_t n) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= n) return;
  const cd d(val[13 * n + row], val[27 * n + 13 * n + row]);
  jsc[row] = cdiv(cd(1.0, 0.0), csqrt_principal(d));
  const double m = hypot(d.re, d.im);
  wn[row] = m;
  if (wn32) wn32[row] = (float)m;
}

__global__ void sym_jacobi_scale_kernel(double* __restrict__ val, uint8_t* __restrict__ cflag, cd* __restrict__ b,
                                        const cd* __restrict__ jsc, int64_t n, int64_t Nx, int64_t NxNy) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= n) return;
  const cd sr = jsc[row];
  int cplx_row = 0;
  for (int k = 0; k < 27; ++k) {
    const int di = k % 3 - 1, dj = (k / 3) % 3 - 1, dl = k / 9 - 1;
    int64_t c = row + di + Nx * dj + NxNy * dl;
    c = c < 0 ? 0 : (c >= n ? n - 1 : c);  // padded slots hold 0 and stay 0
    const int64_t e = (int64_t)k * n + row;
    const cd a(val[e], val[27 * n + e]);
    const cd q = (sr * a) * jsc[c];
    val[e] = q.re;
    val[27 * n + e] = q.im;
    cplx_row |= (q.im != 0.0);
  }
  cflag[row] = (uint8_t)cplx_row;
  b[row] = sr * b[row];
}

__global__ void jacobi_rescale_kernel(cd* __restrict__ x, const cd* __restrict__ jsc, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] = jsc[i] * x[i];
}

}  // namespace

namespace eng {
void* bicg_kernel(int minb) {
  return minb >= 2 ? (void*)bicg_persistent<2> : (void*)bicg_persistent<1>;
}

void* tfqmr_kernel(int minb) {
  return minb >= 2 ? (void*)tfqmr_persistent<2> : (void*)tfqmr_persistent<1>;
}

helm_status jacobi_prepare(double* val, uint8_t* cflag, cd* djac, int64_t n, int64_t nx, int64_t ny, int64_t nz,
                           cudaStream_t s) {
  if (n == 0) return HELM_OK;
  const int64_t Nx = nx + 1, NxNy = Nx * (ny + 1);
  (void)nz;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  jacobi_diag_kernel<<<blocks, 256, 0, s>>>(val, djac, n);
  jacobi_scale_kernel<<<blocks, 256, 0, s>>>(val, cflag, djac, n, Nx, NxNy);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

helm_status sym_jacobi_prepare(double* val, uint8_t* cflag, cd* b, cd* jsc, double* wn, float* wn32, int64_t n,
                               int64_t nx, int64_t ny, cudaStream_t s) {
  if (n == 0) return HELM_OK;
  const int64_t Nx = nx + 1, NxNy = Nx * (ny + 1);
  const unsigned blocks = (unsigned)((n + 255) / 256);
  sym_jacobi_diag_kernel<<<blocks, 256, 0, s>>>(val, jsc, wn, wn32, n);
  sym_jacobi_scale_kernel<<<blocks, 256, 0, s>>>(val, cflag, b, jsc, n, Nx, NxNy);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

helm_status jacobi_rescale(cd* x, const cd* jsc, int64_t n, cudaStream_t s) {
  if (n == 0) return HELM_OK;
  jacobi_rescale_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, jsc, n);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

helm_status jacobi_unscale(cd* x, const cd* djac, int64_t n, cudaStream_t s) {
  if (n == 0) return HELM_OK;
  jacobi_unscale_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, djac, n);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}
}  // namespace eng
}  // namespace helm
