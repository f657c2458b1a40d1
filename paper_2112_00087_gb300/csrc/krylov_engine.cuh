// Shared pieces of the persistent batched Krylov engine: per-system descriptors, the state each
// system carries between super-steps, the tile / launch parameters, and the device helpers
// every solver's phases use (arrival counting, tile-ordered partial sums, the compacted tile
// list, the two-pass tile SpMV). The solvers themselves live in krylov_cocg.cu (COCG, FP64 and
// mixed) and krylov_bicg.cu (BiCGSTAB, TFQMR); krylov_host.cu launches them.
#pragma once

#include "bulk.cuh"
#include "kernels.cuh"

namespace helm {
namespace eng {

struct KSys {
  int64_t n;
  int64_t Nx, NxNy;   // lattice strides of the slot-major 27-point layout
  const cd* val;      // slot-major split layout: 27 n real parts, then 27 n imaginary (FP64)
  const cf* val32;    // the same in FP32 (mixed)
  const uint8_t* cflag;  // [n] 1 for rows with a non-zero imaginary entry
  const cd* b;
  cd* x;
  cd* r;
  cd* p;
  cd* q;
  cf* x32;
  cf* r32;
  cf* p32;
  cf* q32;
  const float2* valw;  // double-word mixed mode: (hi, lo) pairs, slot-major split layout, slot stride nsw
  int64_t nsw;         // slot stride of valw: n rounded up to even (16-byte aligned slot starts)
  cw* xw;
  cw* rw;
  cw* pw;
  cw* qw;
  cd* xb;   // FP64 COCG: iterate at the last halving of the best residual estimate
  cd* dv;   // TFQMR: direction d
  cd* djac; // right Jacobi: diag(A) of the unscaled matrix, or null
  cd* jsc;  // symmetric Jacobi (COCG): s_i = a_ii^-1/2, the system solved is S A S y = S b, x = S y
  const double* wn;   // symmetric Jacobi: norm weights |a_ii| (residual of A x = b), or null
  const float* wn32;  // the same in FP32 for the inner solves of the mixed modes
  cd* rs;   // BiCGSTAB: shadow residual r0*
  cd* sv;   // BiCGSTAB: s = r - alpha v
  cd* tv;   // BiCGSTAB: t = A s
  int tile0, ntiles;
};

enum : int { MODE_RESID = 0, MODE_INNER = 1, MODE_FP64 = 2 };
// phase C actions: direction update; true residual of x; true residual of the saved best
// iterate (which becomes x); refinement update of the mixed modes
enum : int { C_PUPDATE = 0, C_CHECK = 1, C_XUPDATE = 2, C_CHECK_BEST = 3 };

struct KState {
  int act;       // 1 while iterating
  int amode;     // phase A source: 0 = p, 1 = r (and p := r)
  int cmode;     // phase C action
  int mode;      // mixed: MODE_RESID / MODE_INNER
  int it;        // Krylov steps (complex64 inner and FP64 steps)
  int it32;      // complex64 inner steps
  int inner_it;
  int outer;
  int restarts;
  int status;
  int bd;        // breakdown seen
  int pend;      // mixed: finish pending (status in `status`)
  int to_fp64;   // mixed: switch to FP64 COCG at the end of this step
  int discard;   // mixed: the inner solve did not reduce its residual; skip its correction
  int fell_back; // mixed: the system finished in FP64 COCG
  int reset_x;   // mixed: the fallback restarts from x = 0 (refinement left x worse than zero)
  int best_it;   // step of the last halving of the best residual estimate
  int start_it;  // step count at the last (re)start of FP64 COCG
  int save_best; // phase C copies x to the best iterate (the estimate just halved)
  unsigned arrive;
  double bnorm, rnorm, relres, est, prev_rel, best_est;
  cd rho, alpha, beta, omega;
  cd eta;         // TFQMR
  double theta, tau;
  int tstate;     // TFQMR: sub-step of the state machine
  int pad2;
};

struct KTile {
  int sys;
  int pad;
  int64_t row0, row1;
};

// CTRL_P0 / CTRL_P1: tile list used on even / odd super-steps (engines with one barrier per step);
// CTRL_Q0 .. CTRL_Q0 + 5: tile counters of the dynamically scheduled phases (one per phase, six
// in rotation)
enum : int { CTRL_CUR = 0, CTRL_CNT0 = 1, CTRL_CNT1 = 2, CTRL_NACT = 3, CTRL_FIN = 4, CTRL_P0 = 5, CTRL_P1 = 6,
             CTRL_Q0 = 8, CTRL_NQ = 6, CTRL_N = 16 };

struct KParams {
  const KSys* sys;
  KState* st;
  const KTile* tiles;
  int ntiles;
  int* list0;
  int* list1;
  int* ctrl;
  cd* part;  // [ntiles][2]
  GridBar* bar;
  double tol;
  int maxit;
  double inner_tol;
  int inner_maxit;
  int max_outer;
  int max_steps;
  int stall;
  unsigned bar_extra;             // fault injection: arrivals the barriers wait for in addition
  unsigned long long bar_timeout;  // barrier give-up time (ns)
  unsigned long long* trace;       // optional phase trace of block 0 (HELM_TRACE_STEPS), or null
  int trace_steps;
  int prefetch;                    // double-word SpMV: each thread prefetches into L2 the matrix parts of
                                   // the row it reaches this many block rows later (0 = off)
  int pf_chunks;                   // double-word vector phases: thread 0 bulk-prefetches into L2 the
                                   // vectors of the block's chunk of 256 rows this many chunks ahead
};


// Kernel entry points of the solver translation units (host function pointers of the persistent
// kernels, for the cooperative launch in krylov_host.cu).
void* cocg_kernel(int prec, int blocks_per_sm);  // prec: 0 FP64, 1 complex64 inner, 2 double-word inner
void* bicg_kernel(int blocks_per_sm);
void* tfqmr_kernel(int blocks_per_sm);
// Right Jacobi preconditioning of a slot-major split matrix: djac = diag(A), then every column c
// scaled by 1 / djac[c] (row flags recomputed); after the solve x = y / djac.
helm_status jacobi_prepare(double* val, uint8_t* cflag, cd* djac, int64_t n, int64_t nx, int64_t ny, int64_t nz,
                           cudaStream_t s);
helm_status jacobi_unscale(cd* x, const cd* djac, int64_t n, cudaStream_t s);
// Symmetric Jacobi scaling for COCG: s_i = a_ii^-1/2 (principal root) into jsc, weights |a_ii|
// into wn (and wn32 if not null), entries a_ij <- s_i a_ij s_j, b <- S b (row flags recomputed);
// after the solve x <- S y (jacobi_rescale).
helm_status sym_jacobi_prepare(double* val, uint8_t* cflag, cd* b, cd* jsc, double* wn, float* wn32, int64_t n,
                               int64_t nx, int64_t ny, cudaStream_t s);
helm_status jacobi_rescale(cd* x, const cd* jsc, int64_t n, cudaStream_t s);

}  // namespace eng

namespace {
using namespace eng;

// Weight of row i in residual norms: 1, or |a_ii| under symmetric Jacobi scaling.
__device__ __forceinline__ double wnorm(const KSys& Y, int64_t i) { return Y.wn ? Y.wn[i] : 1.0; }
__device__ __forceinline__ float wnorm32(const KSys& Y, int64_t i) { return Y.wn32 ? Y.wn32[i] : 1.f; }

// Phase trace (tracing aid, off unless HELM_TRACE_STEPS is set): block 0 records %globaltimer
// after its own work of each phase and after each grid barrier, for the first trace_steps steps
// (kTraceStride slots per step: six times, then the number of active tiles of the step).
constexpr int kTraceStride = 8;
__device__ __forceinline__ void trace_mark(const KParams& P, int step, int k) {
  if (P.trace != nullptr && blockIdx.x == 0 && threadIdx.x == 0 && step < P.trace_steps)
    P.trace[(size_t)step * kTraceStride + k] = globaltimer();
}
__device__ __forceinline__ void trace_count(const KParams& P, int step, int nat) {
  if (P.trace != nullptr && blockIdx.x == 0 && threadIdx.x == 0 && step < P.trace_steps)
    P.trace[(size_t)step * kTraceStride + 6] = (unsigned long long)nat;
}


__device__ __forceinline__ int vload(const int* p) { return *((volatile const int*)p); }

// Dynamic tile scheduling of one phase: blocks take the entries of the active tile list in order
// from the phase's counter, one atomic per tile, so a block that finishes early takes more tiles
// and every block reaches the grid barrier at about the same time. While the list holds more
// than two tiles per block (and may_look_ahead) the next entry is requested as the current tile
// starts (hiding the atomic's latency); with fewer it is requested after the tile, so no block
// holds a tile that an idle block could have taken. A phase whose tiles are long next to the
// atomic's latency passes may_look_ahead = false: a request made as a tile starts can leave a
// block holding one more tile at the end of the phase while others already wait at the barrier.
// Results do not depend on which block processes a tile (partial
// sums are combined in tile order). Counter g % CTRL_NQ of phase g (three phases per super-step)
// is zeroed by block 0 in phase g + 3, between two barriers on either side of its uses; the host
// starts them at zero.
template <typename F>
__device__ __forceinline__ void for_tiles_dynamic(const KParams& P, int phase_g, int nat, const int* list, F f,
                                                  bool may_look_ahead = true) {
  __shared__ int s_a;
  int* ctr = P.ctrl + CTRL_Q0 + phase_g % CTRL_NQ;
  const bool ahead = may_look_ahead && nat > 2 * (int)gridDim.x;
  if (blockIdx.x == 0 && threadIdx.x == 0) P.ctrl[CTRL_Q0 + (phase_g + 3) % CTRL_NQ] = 0;
  if (threadIdx.x == 0) s_a = atomicAdd(ctr, 1);
  __syncthreads();
  int a = s_a;
  while (a < nat) {
    int next = 0;
    if (ahead && threadIdx.x == 0) next = atomicAdd(ctr, 1);
    f(list[a]);
    __syncthreads();
    if (threadIdx.x == 0) s_a = ahead ? next : atomicAdd(ctr, 1);
    __syncthreads();
    a = s_a;
  }
}

// Arrival of this block's tile for system s; true (block-uniform) for the last arriver.
__device__ __forceinline__ bool arrive_last(KState* S, int ntiles_s) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned old = atomicAdd(&S->arrive, 1u);
    s_last = (old + 1u == (unsigned)ntiles_s);
    if (s_last) {
      S->arrive = 0u;
      __threadfence();
    }
  }
  __syncthreads();
  return s_last != 0;
}

// Sum of the two complex partials of tiles [tile0, tile0 + nt), tile order, every thread.
__device__ __forceinline__ void sum_parts(const cd* part, int tile0, int nt, cd& a, cd& b, double* sh) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int t = threadIdx.x; t < nt; t += kBlock) {
    const cd u = ld_l2(part + 2 * (int64_t)(tile0 + t));
    const cd w = ld_l2(part + 2 * (int64_t)(tile0 + t) + 1);
    v[0] += u.re; v[1] += u.im; v[2] += w.re; v[3] += w.im;
  }
  block_sum<4>(v, sh);
  a = cd(v[0], v[1]);
  b = cd(v[2], v[3]);
}

__device__ __forceinline__ void write_parts(cd* part, int t, const double (&v)[4]) {
  if (threadIdx.x == 0) {
    part[2 * (int64_t)t] = cd(v[0], v[1]);
    part[2 * (int64_t)t + 1] = cd(v[2], v[3]);
  }
}

__device__ __forceinline__ void finish(const KParams& P, KState* S, int status, double relres) {
  S->status = status;
  S->relres = relres;
  S->act = 0;
  __threadfence();
  atomicAdd(&P.ctrl[CTRL_FIN], 1);
  atomicSub(&P.ctrl[CTRL_NACT], 1);
}

// Block 0, phase A: rebuild the other tile list from the act flags (only when a system
// finished since the last rebuild). Act flags change only in phase C, so the snapshot is
// exact. The list index is flipped by the caller in phase B, after every block has read the
// current index for this step; the new list is consumed from the next step on.
__device__ bool rebuild_list(const KParams& P, int cur, int& seen_fin, int* sh_int) {
  const int fin = vload(&P.ctrl[CTRL_FIN]);
  if (fin == seen_fin) return false;  // block-uniform: every thread read the same stable value
  seen_fin = fin;
  int* dst = cur ? P.list0 : P.list1;
  int base = 0;
  for (int t0 = 0; t0 < P.ntiles; t0 += kBlock) {
    const int t = t0 + threadIdx.x;
    const int keep = (t < P.ntiles) ? vload(&P.st[P.tiles[t].sys].act) : 0;
    // block exclusive scan of keep (warp ballots, then warp counts in order)
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh_int[w] = __popc(m);
    __syncthreads();
    int off = base;
    for (int i = 0; i < w; ++i) off += sh_int[i];
    int tot = 0;
    for (int i = 0; i < kBlock / 32; ++i) tot += sh_int[i];
    if (keep) dst[off + __popc(m & ((1u << lane) - 1u))] = t;
    base += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    P.ctrl[cur ? CTRL_CNT0 : CTRL_CNT1] = base;
    __threadfence();
  }
  return true;
}

// Product of the tile's rows with x in two passes: first(row, s_re, complex_flag) for every
// row with the real-part product (two rows per thread, so their loads overlap), then, if any
// row of the tile is flagged complex (block-uniform), fix(row, s_im) for each flagged row with
// its imaginary-part product. Thread t handles rows row0 + t + m kBlock in both passes, so a
// thread reads back only what it wrote itself.
#ifndef HELM_ROWS_PER_THREAD
#define HELM_ROWS_PER_THREAD 1
#endif
#ifndef HELM_VEC_UNROLL
#define HELM_VEC_UNROLL 1
#endif
#ifndef HELM_DEFAULT_BLOCKS_PER_SM
#define HELM_DEFAULT_BLOCKS_PER_SM 2
#endif

template <typename T, typename F1, typename F2>
__device__ __forceinline__ void tile_spmv(const cplx<T>* val, const uint8_t* cflag, const cplx<T>* x, int64_t n,
                                          int64_t Nx, int64_t NxNy, int64_t row0, int64_t row1, F1 first,
                                          F2 fix) {
  const T* vre = reinterpret_cast<const T*>(val);  // split layout: real parts, then imaginary
  const T* vim = vre + 27 * n;
  int has_c = 0;
  if (HELM_ROWS_PER_THREAD == 2) {
    for (int64_t r0 = row0 + threadIdx.x; r0 < row1; r0 += 2 * kBlock) {
      const int64_t r1 = r0 + kBlock < row1 ? r0 + kBlock : r0;  // clamped only in a ragged tail
      const cplx<T> s0 = dia_row_re<T>(vre, x, n, Nx, NxNy, r0);
      const cplx<T> s1 = dia_row_re<T>(vre, x, n, Nx, NxNy, r1);
      const int c0 = cflag[r0], c1 = cflag[r1];
      first(r0, s0, c0);
      if (r1 != r0) first(r1, s1, c1);
      has_c |= c0 | c1;
    }
  } else {
    for (int64_t r0 = row0 + threadIdx.x; r0 < row1; r0 += kBlock) {
      const cplx<T> s0 = dia_row_re<T>(vre, x, n, Nx, NxNy, r0);
      const int c0 = cflag[r0];
      first(r0, s0, c0);
      has_c |= c0;
    }
  }
  if (__syncthreads_or(has_c)) {
    for (int64_t row = row0 + threadIdx.x; row < row1; row += kBlock)
      if (cflag[row]) fix(row, dia_row_im<T>(vim, x, n, Nx, NxNy, row));
  }
}


__device__ __forceinline__ cw cw_add(const cw& a, const cw& b) {
  dacc2 acc;
  acc.s = cw_hi(a);
  acc.c = cw_lo(a);
  acc.add(cw_hi(b), cw_lo(b));
  float2 hi, lo;
  acc.get(hi, lo);
  return cw_from(hi, lo);
}

// L2 prefetch of one address (no register result, nothing waits for it)
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Inner stop of a refinement step: the inner estimate is relative to ||r_outer||; stop at the
// requested reduction, or once the outer target (half of tol ||b||) is reached.
__device__ __forceinline__ double inner_stop(const KParams& P, const KState* S) {
  return fmax(P.inner_tol, 0.5 * P.tol * S->bnorm / S->rnorm);
}

}  // namespace
}  // namespace helm
