// Restarted, right-preconditioned GMRES(m) for the complex FE Helmholtz system (paper Sec. 4:
// Krylov solve in complex double precision on the GPU).
//
// One restart cycle runs entirely on the device: x0 = 0; v_0 = r / ||r||; for j < m:
//   z = M^-1 v_j (right preconditioner, identity or restricted additive Schwarz), w = A z,
//   classical Gram-Schmidt applied twice (h = V^H w, w -= V h, h2 = V^H w, w -= V h2),
//   h_{j+1,j} = ||w||, complex Givens rotations on the Hessenberg column (c = |a|/r,
//   s = (a/|a|) b/r, r = sqrt(|a|^2 + b^2); c = 0, s = 1 when a = 0), residual estimate
//   |g_{j+1}| / ||b||; the cycle stops at the estimate <= tol, a zero h_{j+1,j} or maxit.
// Cycle end: R y = g (back substitution), x += M^-1 V y, true residual r = b - A x decides
// convergence or restart. Every kernel reads its step index from its launch arguments and a
// "cycle done" flag from device memory, so the whole cycle is captured once as a CUDA graph
// and replayed; the host reads one status word per cycle.
//
// Reductions: every tile (block) writes its partial sums; the last block of a reduction
// (atomic arrival count) adds them in tile order, so results do not depend on timing.
#include <algorithm>
#include <cstring>
#include <vector>

#include "kernels.cuh"
#include "ras.cuh"

namespace helm {
namespace {

struct GmCtl {
  int it, j_end, done_cycle, stop, status, restarts, bd, pad;
  unsigned arrive;
  unsigned pad2;
  double bnorm, rnorm, est, relres, hn;
};

struct GmArgs {
  int64_t n;
  int ntiles;
  int64_t tile_rows;
  int m;
  const int32_t* rowptr;
  const int32_t* col;
  const cd* val;
  const cd* b;
  cd* x;
  cd* r;
  cd* V;     // [(m+1)][n]
  cd* w;     // [n]
  cd* z;     // [n] preconditioned vector (or null)
  cd* u;     // [n] V y
  cd* H;     // [(m+1) * m], column j at H + j*(m+1)
  cd* g;     // [m+1]
  double* cs;
  cd* sn;
  cd* y;     // [m]
  cd* h1;    // [m+1]
  cd* part;  // [ntiles][m+1]
  GmCtl* ctl;
  double tol;
  int maxit;
};

__device__ __forceinline__ int vld(const int* p) { return *((volatile const int*)p); }

__device__ __forceinline__ bool last_block(GmCtl* c, int ntiles) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned old = atomicAdd(&c->arrive, 1u);
    s_last = (old + 1u == (unsigned)ntiles);
    if (s_last) {
      c->arrive = 0u;
      __threadfence();
    }
  }
  __syncthreads();
  return s_last != 0;
}

// ---- init: x = 0, r = b, ||b|| ----
__global__ void __launch_bounds__(kBlock) gm_init(GmArgs a) {
  __shared__ double sh[kBlock / 32];
  const int64_t r0 = blockIdx.x * a.tile_rows, r1 = min(a.n, r0 + a.tile_rows);
  double v[1] = {0.0};
  for (int64_t i = r0 + threadIdx.x; i < r1; i += kBlock) {
    const cd bi = a.b[i];
    a.x[i] = cd(0.0, 0.0);
    a.r[i] = bi;
    v[0] += bi.re * bi.re + bi.im * bi.im;
  }
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) a.part[blockIdx.x] = cd(v[0], 0.0);
  if (last_block(a.ctl, a.ntiles)) {
    double s[1] = {0.0};
    for (int t = threadIdx.x; t < a.ntiles; t += kBlock) s[0] += ld_l2(a.part + t).re;
    block_sum<1>(s, sh);
    if (threadIdx.x == 0) {
      GmCtl* c = a.ctl;
      c->bnorm = sqrt(s[0]);
      c->rnorm = c->bnorm;
      c->relres = 1.0;
      if (c->bnorm == 0.0) {
        c->stop = 1;
        c->status = HELM_OK;
        c->relres = 0.0;
      }
    }
  }
}

// ---- cycle start: v_0 = r / ||r||, g = (||r||, 0, ...) ----
__global__ void __launch_bounds__(kBlock) gm_start(GmArgs a) {
  if (vld(&a.ctl->stop)) return;
  const double s = 1.0 / a.ctl->rnorm;
  const int64_t r0 = blockIdx.x * a.tile_rows, r1 = min(a.n, r0 + a.tile_rows);
  for (int64_t i = r0 + threadIdx.x; i < r1; i += kBlock) {
    const cd ri = a.r[i];
    a.V[i] = cd(ri.re * s, ri.im * s);
  }
  if (blockIdx.x == 0 && threadIdx.x <= a.m) a.g[threadIdx.x] = cd(threadIdx.x == 0 ? a.ctl->rnorm : 0.0, 0.0);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ctl->done_cycle = 0;
    a.ctl->j_end = 0;
  }
}

// ---- w = A src ----
__global__ void __launch_bounds__(kBlock) gm_spmv(GmArgs a, const cd* src, int j) {
  if (vld(&a.ctl->done_cycle) || vld(&a.ctl->stop)) return;
  constexpr int G = 4;
  const int gid = threadIdx.x / G, g = threadIdx.x % G;
  const int64_t r0 = blockIdx.x * a.tile_rows, r1 = min(a.n, r0 + a.tile_rows);
  for (int64_t base = r0; base < r1; base += kBlock / G) {
    const int64_t row = base + gid;
    const bool valid = row < r1;
    const cd s = csr_row27<G, double>(a.rowptr, a.col, a.val, src, row, valid, g);
    if (valid && g == 0) a.w[row] = s;
  }
}

// Partial dots h_i = V_i^H w over the tile's rows for i <= j (warp k takes i = k, k+8, ...),
// then, in the last block, h[i] = sum over tiles in order (warp per i).
__device__ void dots_and_reduce(const GmArgs& a, int j, cd* h_out, double* sh) {
  const int64_t r0 = blockIdx.x * a.tile_rows, r1 = min(a.n, r0 + a.tile_rows);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i <= j; i += kBlock / 32) {
    const cd* Vi = a.V + (int64_t)i * a.n;
    double re = 0.0, im = 0.0;
    for (int64_t k = r0 + lane; k < r1; k += 32) {
      const cd v = Vi[k], ww = a.w[k];
      re += v.re * ww.re + v.im * ww.im;  // conj(v) * w
      im += v.re * ww.im - v.im * ww.re;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) a.part[(int64_t)blockIdx.x * (a.m + 1) + i] = cd(re, im);
  }
  if (last_block(a.ctl, a.ntiles)) {
    for (int i = warp; i <= j; i += kBlock / 32) {
      double re = 0.0, im = 0.0;
      for (int t = lane; t < a.ntiles; t += 32) {
        const cd p = ld_l2(a.part + (int64_t)t * (a.m + 1) + i);
        re += p.re;
        im += p.im;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
      }
      if (lane == 0) h_out[i] = cd(re, im);
    }
    __threadfence();
  }
}

__global__ void __launch_bounds__(kBlock) gm_dots1(GmArgs a, int j) {
  if (vld(&a.ctl->done_cycle) || vld(&a.ctl->stop)) return;
  __shared__ double sh[kBlock / 32];
  dots_and_reduce(a, j, a.h1, sh);
}

// w -= V h for the tile's rows (h in shared memory)
__device__ void subtract_Vh(const GmArgs& a, int j, const cd* h, cd* hs) {
  for (int i = threadIdx.x; i <= j; i += kBlock) hs[i] = ld_l2(h + i);
  __syncthreads();
  const int64_t r0 = blockIdx.x * a.tile_rows, r1 = min(a.n, r0 + a.tile_rows);
  for (int64_t k = r0 + threadIdx.x; k < r1; k += kBlock) {
    cd acc = a.w[k];
    for (int i = 0; i <= j; ++i) {
      const cd v = a.V[(int64_t)i * a.n + k];
      const cd hi = hs[i];
      acc.re -= v.re * hi.re - v.im * hi.im;
      acc.im -= v.re * hi.im + v.im * hi.re;
    }
    a.w[k] = acc;
  }
  __syncthreads();
}

// second Gram-Schmidt pass: w -= V h1, then h2 = V^H w (into part -> g scratch h2 = y buffer)
__global__ void __launch_bounds__(kBlock) gm_update_dots2(GmArgs a, int j, cd* h2) {
  if (vld(&a.ctl->done_cycle) || vld(&a.ctl->stop)) return;
  __shared__ double sh[kBlock / 32];
  __shared__ cd hs[129];
  subtract_Vh(a, j, a.h1, hs);
  dots_and_reduce(a, j, h2, sh);
}

// w -= V h2, ||w||, Hessenberg column, Givens, residual estimate (last block)
__global__ void __launch_bounds__(kBlock) gm_update_norm(GmArgs a, int j, const cd* h2) {
  if (vld(&a.ctl->done_cycle) || vld(&a.ctl->stop)) return;
  __shared__ double sh[kBlock / 32];
  __shared__ cd hs[129];
  subtract_Vh(a, j, h2, hs);
  const int64_t r0 = blockIdx.x * a.tile_rows, r1 = min(a.n, r0 + a.tile_rows);
  double v[1] = {0.0};
  for (int64_t k = r0 + threadIdx.x; k < r1; k += kBlock) {
    const cd ww = a.w[k];
    v[0] += ww.re * ww.re + ww.im * ww.im;
  }
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) a.part[(int64_t)blockIdx.x * (a.m + 1)] = cd(v[0], 0.0);
  if (last_block(a.ctl, a.ntiles)) {
    double s[1] = {0.0};
    for (int t = threadIdx.x; t < a.ntiles; t += kBlock) s[0] += ld_l2(a.part + (int64_t)t * (a.m + 1)).re;
    block_sum<1>(s, sh);
    if (threadIdx.x == 0) {
      GmCtl* c = a.ctl;
      const int m1 = a.m + 1;
      cd* Hj = a.H + (int64_t)j * m1;
      const double hn = sqrt(s[0]);
      for (int i = 0; i <= j; ++i) {
        const cd x1 = ld_l2(a.h1 + i), x2 = ld_l2(h2 + i);
        Hj[i] = cd(x1.re + x2.re, x1.im + x2.im);
      }
      Hj[j + 1] = cd(hn, 0.0);
      for (int i = 0; i < j; ++i) {  // previous rotations
        const double ci = a.cs[i];
        const cd si = a.sn[i];
        const cd xa = Hj[i], xb = Hj[i + 1];
        Hj[i] = cd(ci * xa.re + (si.re * xb.re - si.im * xb.im), ci * xa.im + (si.re * xb.im + si.im * xb.re));
        // -conj(s) xa + c xb
        Hj[i + 1] = cd(-(si.re * xa.re + si.im * xa.im) + ci * xb.re, -(si.re * xa.im - si.im * xa.re) + ci * xb.im);
      }
      const cd aj = Hj[j];
      const double bj = hn;
      double cj;
      cd sj;
      const double aa = sqrt(aj.re * aj.re + aj.im * aj.im);
      if (aa == 0.0) {
        cj = 0.0;
        sj = cd(1.0, 0.0);
      } else {
        const double rr = sqrt(aa * aa + bj * bj);
        cj = aa / rr;
        sj = cd((aj.re / aa) * (bj / rr), (aj.im / aa) * (bj / rr));
      }
      a.cs[j] = cj;
      a.sn[j] = sj;
      Hj[j] = cd(cj * aj.re + sj.re * bj, cj * aj.im + sj.im * bj);
      Hj[j + 1] = cd(0.0, 0.0);
      const cd gj = a.g[j];
      a.g[j] = cd(cj * gj.re, cj * gj.im);
      const cd gn(-(sj.re * gj.re + sj.im * gj.im), -(sj.re * gj.im - sj.im * gj.re));  // -conj(s) g_j
      a.g[j + 1] = gn;
      const double est = sqrt(gn.re * gn.re + gn.im * gn.im) / c->bnorm;
      c->est = est;
      c->hn = hn;
      c->it += 1;
      c->j_end = j + 1;
      if (hn == 0.0) c->bd = 1;
      if (!(est > a.tol) || hn == 0.0 || c->it >= a.maxit || j + 1 == a.m) c->done_cycle = 1;
      __threadfence();
    }
  }
}

// v_{j+1} = w / h_{j+1,j}
__global__ void __launch_bounds__(kBlock) gm_scale(GmArgs a, int j) {
  if (vld(&a.ctl->done_cycle) || vld(&a.ctl->stop)) return;
  const double s = 1.0 / a.ctl->hn;
  cd* Vn = a.V + (int64_t)(j + 1) * a.n;
  const int64_t r0 = blockIdx.x * a.tile_rows, r1 = min(a.n, r0 + a.tile_rows);
  for (int64_t k = r0 + threadIdx.x; k < r1; k += kBlock) {
    const cd ww = a.w[k];
    Vn[k] = cd(ww.re * s, ww.im * s);
  }
}

// cycle end 1: R y = g (back substitution, one thread), then u = V y (all blocks)
__global__ void gm_lsq(GmArgs a) {
  if (vld(&a.ctl->stop)) return;
  if (threadIdx.x != 0) return;
  const int je = a.ctl->j_end, m1 = a.m + 1;
  for (int i = je - 1; i >= 0; --i) {
    cd s = a.g[i];
    for (int k = i + 1; k < je; ++k) {
      const cd hk = a.H[(int64_t)k * m1 + i], yk = a.y[k];
      s.re -= hk.re * yk.re - hk.im * yk.im;
      s.im -= hk.re * yk.im + hk.im * yk.re;
    }
    a.y[i] = cdiv(s, a.H[(int64_t)i * m1 + i]);
  }
}

__global__ void __launch_bounds__(kBlock) gm_combine(GmArgs a, int add_to_x) {
  if (vld(&a.ctl->stop)) return;
  __shared__ cd ys[128];
  const int je = a.ctl->j_end;
  for (int i = threadIdx.x; i < je; i += kBlock) ys[i] = a.y[i];
  __syncthreads();
  const int64_t r0 = blockIdx.x * a.tile_rows, r1 = min(a.n, r0 + a.tile_rows);
  for (int64_t k = r0 + threadIdx.x; k < r1; k += kBlock) {
    cd acc(0.0, 0.0);
    for (int i = 0; i < je; ++i) cfma(acc, a.V[(int64_t)i * a.n + k], ys[i]);
    if (add_to_x) {
      cd xi = a.x[k];
      a.x[k] = cd(xi.re + acc.re, xi.im + acc.im);
    } else {
      a.u[k] = acc;
    }
  }
}

__global__ void __launch_bounds__(kBlock) gm_add(GmArgs a, const cd* zz) {
  if (vld(&a.ctl->stop)) return;
  const int64_t r0 = blockIdx.x * a.tile_rows, r1 = min(a.n, r0 + a.tile_rows);
  for (int64_t k = r0 + threadIdx.x; k < r1; k += kBlock) {
    const cd xi = a.x[k], d = zz[k];
    a.x[k] = cd(xi.re + d.re, xi.im + d.im);
  }
}

// cycle end 2: r = b - A x, relres, decision
__global__ void __launch_bounds__(kBlock) gm_residual(GmArgs a) {
  if (vld(&a.ctl->stop)) return;
  __shared__ double sh[kBlock / 32];
  constexpr int G = 4;
  const int gid = threadIdx.x / G, g = threadIdx.x % G;
  const int64_t r0 = blockIdx.x * a.tile_rows, r1 = min(a.n, r0 + a.tile_rows);
  double v[1] = {0.0};
  for (int64_t base = r0; base < r1; base += kBlock / G) {
    const int64_t row = base + gid;
    const bool valid = row < r1;
    const cd s = csr_row27<G, double>(a.rowptr, a.col, a.val, a.x, row, valid, g);
    if (valid && g == 0) {
      const cd bi = a.b[row];
      const cd ri(bi.re - s.re, bi.im - s.im);
      a.r[row] = ri;
      v[0] += ri.re * ri.re + ri.im * ri.im;
    }
  }
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) a.part[(int64_t)blockIdx.x * (a.m + 1)] = cd(v[0], 0.0);
  if (last_block(a.ctl, a.ntiles)) {
    double s[1] = {0.0};
    for (int t = threadIdx.x; t < a.ntiles; t += kBlock) s[0] += ld_l2(a.part + (int64_t)t * (a.m + 1)).re;
    block_sum<1>(s, sh);
    if (threadIdx.x == 0) {
      GmCtl* c = a.ctl;
      const double rn = sqrt(s[0]);
      const double rel = rn / c->bnorm;
      c->relres = rel;
      if (rel <= a.tol) { c->stop = 1; c->status = HELM_OK; }
      else if (!(rel == rel)) { c->stop = 1; c->status = HELM_NAN; }
      else if (c->it >= a.maxit) { c->stop = 1; c->status = HELM_NOT_CONVERGED; }
      else if (c->bd) { c->stop = 1; c->status = HELM_BREAKDOWN; }
      else { c->rnorm = rn; c->restarts += 1; }
      __threadfence();
    }
  }
}

}  // namespace

helm_status solve_gmres_system(const helm_ctx* ctx, const int32_t* rowptr, const int32_t* col, const cd* val,
                               double freq, const cd* b, const helm_solve_opts& o, cd* x, helm_solve_stats* st) {
  // The cycle is captured as a CUDA graph, which the legacy default stream does not allow: run
  // the solve on a private stream ordered after the context stream.
  cudaStream_t s = nullptr;
  HELM_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  {
    cudaEvent_t ev = nullptr;
    cudaError_t e0 = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e0 == cudaSuccess) e0 = cudaEventRecord(ev, ctx->stream);
    if (e0 == cudaSuccess) e0 = cudaStreamWaitEvent(s, ev, 0);
    if (ev) cudaEventDestroy(ev);
    if (e0 != cudaSuccess) {
      cudaStreamDestroy(s);
      return cuda_error(e0, "gmres stream");
    }
  }
  const int64_t n = ctx->n;
  const int m = o.restart;
  int dev = 0, nsm = 1;
  HELM_CUDA(cudaGetDevice(&dev));
  HELM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int64_t tile_rows = 256 * std::max<int64_t>(1, (n + 256LL * 4 * nsm - 1) / (256LL * 4 * nsm));
  const int ntiles = (int)((n + tile_rows - 1) / tile_rows);

  // workspace
  const size_t nV = (size_t)(m + 1) * n;
  cd* ws = nullptr;
  const size_t ncd = 3 * (size_t)n /*r,w,u*/ + nV + (size_t)(m + 1) * m + 3 * (m + 1) + 2 * m +
                     (size_t)ntiles * (m + 1) +
                     (o.precond == HELM_PRECOND_RAS || o.precond == HELM_PRECOND_ORAS || o.precond == HELM_PRECOND_ORAS2 ? n : 0);
  helm_status stt = dev_alloc(&ws, ncd + 2 * m /*cs*/ + 8);
  if (stt != HELM_OK) return stt;
  GmCtl* dctl = nullptr;
  stt = dev_alloc(&dctl, 1);
  if (stt != HELM_OK) {
    cudaFree(ws);
    return stt;
  }
  GmArgs a;
  memset(&a, 0, sizeof(a));
  a.n = n;
  a.ntiles = ntiles;
  a.tile_rows = tile_rows;
  a.m = m;
  a.rowptr = rowptr;
  a.col = col;
  a.val = val;
  a.b = b;
  a.x = x;
  cd* p = ws;
  a.r = p; p += n;
  a.w = p; p += n;
  a.u = p; p += n;
  a.V = p; p += nV;
  a.H = p; p += (size_t)(m + 1) * m;
  a.g = p; p += m + 1;
  a.h1 = p; p += m + 1;
  cd* h2 = p; p += m + 1;
  a.sn = p; p += m;
  a.y = p; p += m;
  a.part = p; p += (size_t)ntiles * (m + 1);
  a.z = nullptr;
  if (o.precond == HELM_PRECOND_RAS || o.precond == HELM_PRECOND_ORAS || o.precond == HELM_PRECOND_ORAS2) {
    a.z = p;
    p += n;
  }
  a.cs = reinterpret_cast<double*>(p);
  a.ctl = dctl;
  a.tol = o.tol;
  a.maxit = o.maxit;

  RasPrecond* ras = nullptr;
  helm_status result = HELM_OK;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  GmCtl* hctl = nullptr;
  cudaError_t e = cudaMallocHost((void**)&hctl, sizeof(GmCtl));
  if (e != cudaSuccess) result = cuda_error(e, "cudaMallocHost");
  if (result == HELM_OK &&
      (o.precond == HELM_PRECOND_RAS || o.precond == HELM_PRECOND_ORAS || o.precond == HELM_PRECOND_ORAS2)) {
    // optimized Schwarz: Robin coefficient i k on every interface face (the matched impedance of
    // the wall term), or the two-sided pair (robin_lo, robin_hi) / h_normal
    const double k = 2.0 * 3.14159265358979323846 * freq / ctx->phys.c;
    RasRobin rb;
    if (o.precond == HELM_PRECOND_ORAS) rb.lo = rb.hi = cd(0.0, k);
    if (o.precond == HELM_PRECOND_ORAS2) {
      rb.lo = cd(o.robin_lo[0], o.robin_lo[1]);
      rb.hi = cd(o.robin_hi[0], o.robin_hi[1]);
      rb.per_h = true;
    }
    result = ras_create(ctx, rowptr, col, val, o.ras_parts, o.ras_overlap, rb, &ras, s);
  }
  if (result == HELM_OK) {
    e = cudaMemsetAsync(dctl, 0, sizeof(GmCtl), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.H, 0, sizeof(cd) * (m + 1) * m, s);
    if (e != cudaSuccess) result = cuda_error(e, "gmres init");
  }
  if (result == HELM_OK) {
    gm_init<<<ntiles, kBlock, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) result = cuda_error(e, "gm_init");
  }
  // capture one restart cycle
  if (result == HELM_OK) {
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) result = cuda_error(e, "begin capture");
  }
  if (result == HELM_OK) {
    gm_start<<<ntiles, kBlock, 0, s>>>(a);
    for (int j = 0; j < m && result == HELM_OK; ++j) {
      const cd* vj = a.V + (size_t)j * n;
      const cd* src = vj;
      if (ras) {
        result = ras_apply(ras, vj, a.z, &dctl->done_cycle, &dctl->stop, s);
        src = a.z;
      }
      gm_spmv<<<ntiles, kBlock, 0, s>>>(a, src, j);
      gm_dots1<<<ntiles, kBlock, 0, s>>>(a, j);
      gm_update_dots2<<<ntiles, kBlock, 0, s>>>(a, j, h2);
      gm_update_norm<<<ntiles, kBlock, 0, s>>>(a, j, h2);
      gm_scale<<<ntiles, kBlock, 0, s>>>(a, j);
    }
    gm_lsq<<<1, 32, 0, s>>>(a);
    if (ras) {
      gm_combine<<<ntiles, kBlock, 0, s>>>(a, 0);
      if (result == HELM_OK) result = ras_apply(ras, a.u, a.z, nullptr, &dctl->stop, s);
      gm_add<<<ntiles, kBlock, 0, s>>>(a, a.z);
    } else {
      gm_combine<<<ntiles, kBlock, 0, s>>>(a, 1);
    }
    gm_residual<<<ntiles, kBlock, 0, s>>>(a);
    e = cudaStreamEndCapture(s, &graph);
    if (e != cudaSuccess && result == HELM_OK) result = cuda_error(e, "end capture");
  }
  if (result == HELM_OK) {
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) result = cuda_error(e, "graph instantiate");
  }
  // host loop: one graph launch + one status read per cycle
  if (result == HELM_OK) {
    e = cudaMemcpyAsync(hctl, dctl, sizeof(GmCtl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) result = cuda_error(e, "gmres status");
    const int max_cycles = o.maxit / 1 + 2;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    int cycles = 0;
    for (int cyc = 0; result == HELM_OK && !hctl->stop && cyc < max_cycles; ++cyc) {
      e = cudaGraphLaunch(exec, s);
      ++cycles;
      if (e == cudaSuccess) e = cudaMemcpyAsync(hctl, dctl, sizeof(GmCtl), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) result = cuda_error(e, "gmres cycle");
    }
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    helm_profile& pr = last_profile();
    pr.solve_ms += ms;
    pr.launches += 1 + (int64_t)cycles * (m * (5 + (ras ? 1 : 0)) + 4 + (ras ? 2 : 0));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  if (result == HELM_OK && ras) result = ras_status(ras);
  if (result == HELM_OK) {
    st->status = hctl->stop ? hctl->status : HELM_NOT_CONVERGED;
    st->iterations = hctl->it;
    st->restarts = hctl->restarts;
    st->outer = 0;
    st->relres = hctl->relres;
    st->bnorm = hctl->bnorm;
    st->iterations_c64 = 0;
    st->pad = 0;
    result = (helm_status)st->status;
  } else {
    st->status = result;
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (ras) ras_destroy(ras);
  cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (hctl) cudaFreeHost(hctl);
  cudaFree(dctl);
  cudaFree(ws);
  (void)freq;
  return result;
}

helm_status solve_gmres(const helm_ctx* ctx, double freq, const helm_solve_opts& o, cd* p_out, helm_solve_stats* st) {
  cd* val = nullptr;
  cd* b = nullptr;
  helm_status r = dev_alloc(&val, ctx->nnz);
  if (r == HELM_OK) r = dev_alloc(&b, ctx->n);
  if (r == HELM_OK) r = assemble_values(ctx, freq, val, b, ctx->stream);
  if (r == HELM_OK) r = solve_gmres_system(ctx, ctx->rowptr, ctx->col, val, freq, b, o, p_out, st);
  cudaStreamSynchronize(ctx->stream);
  cudaFree(val);
  cudaFree(b);
  return r;
}

}  // namespace helm
