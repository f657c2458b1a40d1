// Device building blocks shared by the SpMV, reduction and Krylov kernels.
#pragma once

#include "common.cuh"
#include "dw.cuh"

namespace helm {

constexpr int kBlock = 256;  // threads per block of every row-parallel kernel

// Streaming (evict-first) loads for matrix data read once per product.
__device__ __forceinline__ cd ld_stream(const cd* p) {
  double2 v = __ldcs(reinterpret_cast<const double2*>(p));
  return cd(v.x, v.y);
}
__device__ __forceinline__ cf ld_stream(const cf* p) {
  float2 v = __ldcs(reinterpret_cast<const float2*>(p));
  return cf(v.x, v.y);
}
// L2-only loads for values other blocks wrote during the same launch (partials).
__device__ __forceinline__ cd ld_l2(const cd* p) {
  double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return cd(v.x, v.y);
}

// One CSR row times a vector, computed by a group of G consecutive lanes (G | 32): lane g of
// the group takes entries k = start + g, start + g + G, ...; the G partial sums are combined
// by xor shuffles, so every lane of the group returns the row sum. Entries with a zero
// imaginary part (all rows away from admittance walls) skip the two imaginary products --
// the result is identical to the full complex product for finite x. `x` is read with
// ordinary (coherent) loads because persistent kernels rewrite it between phases.
// All 32 lanes of the warp must call this together (valid = false rows contribute zero).
template <int G, typename T>
__device__ __forceinline__ cplx<T> csr_row(const int32_t* __restrict__ rowptr,
                                           const int32_t* __restrict__ col,
                                           const cplx<T>* __restrict__ val, const cplx<T>* x,
                                           int64_t row, bool valid, int g) {
  cplx<T> acc(T(0), T(0));
  if (valid) {
    const int k0 = __ldg(rowptr + row), k1 = __ldg(rowptr + row + 1);
    for (int k = k0 + g; k < k1; k += G) {
      const cplx<T> a = ld_stream(val + k);
      const int c = __ldcs(col + k);
      const cplx<T> xv = x[c];
      acc.re = fma(a.re, xv.re, acc.re);
      acc.im = fma(a.re, xv.im, acc.im);
      if (a.im != T(0)) {
        acc.re = fma(-a.im, xv.im, acc.re);
        acc.im = fma(a.im, xv.re, acc.im);
      }
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
    acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
  }
  return acc;
}

// Same product for rows of at most kMaxRow entries (the 27-point lattice pattern): every lane
// issues all of its value / column loads, then all of its x gathers, then the multiply-adds,
// so each lane has up to ceil(kMaxRow / G) independent loads in flight instead of one
// load -> gather -> FMA chain per entry. Result identical to csr_row (same per-lane order).
constexpr int kMaxRow = 27;

template <int G, typename T>
__device__ __forceinline__ cplx<T> csr_row27(const int32_t* __restrict__ rowptr,
                                             const int32_t* __restrict__ col,
                                             const cplx<T>* __restrict__ val, const cplx<T>* x,
                                             int64_t row, bool valid, int g) {
  constexpr int S = (kMaxRow + G - 1) / G;
  int k0 = 0, k1 = 0;
  if (valid) {
    k0 = __ldg(rowptr + row);
    k1 = __ldg(rowptr + row + 1);
  }
  cplx<T> a[S];
  int c[S];
#pragma unroll
  for (int q = 0; q < S; ++q) {
    const int k = k0 + g + q * G;
    if (k < k1) {
      a[q] = ld_stream(val + k);
      c[q] = __ldcs(col + k);
    } else {
      a[q] = cplx<T>(T(0), T(0));
      c[q] = -1;
    }
  }
  cplx<T> xv[S];
#pragma unroll
  for (int q = 0; q < S; ++q) xv[q] = (c[q] >= 0) ? x[c[q]] : cplx<T>(T(0), T(0));
  cplx<T> acc(T(0), T(0));
#pragma unroll
  for (int q = 0; q < S; ++q) {
    if (c[q] >= 0) {
      acc.re = fma(a[q].re, xv[q].re, acc.re);
      acc.im = fma(a[q].re, xv[q].im, acc.im);
      if (a[q].im != T(0)) {
        acc.re = fma(-a[q].im, xv[q].im, acc.re);
        acc.im = fma(a[q].im, xv[q].re, acc.im);
      }
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
    acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
  }
  return acc;
}

// ---------------------------------------------------------------------------------------------
// Slot-major 27-point layout ("DIA-27"), real and imaginary parts in separate arrays:
// vre[k * n + row] / vim[k * n + row] hold the entry of `row` for lattice offset
// k = (di+1) + 3 (dj+1) + 9 (dl+1), column row + di + Nx (dj + Ny dl); entries whose neighbour
// lies outside the lattice are stored as zero. The two arrays are contiguous: vim = vre + 27 n. One thread per row: the value loads
// and the x gathers of a warp are contiguous, no column indices are read, and no lanes are
// idle. Gather indices are clamped into [0, n) so that padded slots (value 0) read a valid
// address; 0 * x adds nothing for finite x, so the clamp never changes a result. A per-row
// byte flag (set at assembly) marks rows with a non-zero imaginary entry.
// ---------------------------------------------------------------------------------------------
// Real-part product of one row: sum_k Re(a_k) x_{c_k}, real parts stored slot-major in vre
// (vre[k * n + row]). Three independent accumulation chains per component (one per stencil line
// dj = -1, 0, 1), so consecutive multiply-adds do not wait on each other. Complex entries occur
// only next to admittance walls; their imaginary parts (vim, same layout) are added by
// dia_row_im in a second pass that only rows flagged at assembly take -- on GB300 the FP64 pipe
// is the bottleneck, so the common real rows must not issue any imaginary FMA, and the real pass
// streams 8 bytes per entry instead of 16.
template <typename T>
__device__ __forceinline__ cplx<T> dia_row_re(const T* __restrict__ vre, const cplx<T>* x, int64_t n, int64_t Nx,
                                              int64_t NxNy, int64_t row) {
  cplx<T> acc[3] = {cplx<T>(T(0), T(0)), cplx<T>(T(0), T(0)), cplx<T>(T(0), T(0))};
#pragma unroll
  for (int dl = -1; dl <= 1; ++dl) {
    T a[9];
    cplx<T> xv[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {  // all loads of one lattice plane first
      const int di = q % 3 - 1, dj = q / 3 - 1;
      const int k = q + 9 * (dl + 1);
      int64_t c = row + di + Nx * dj + NxNy * dl;
      c = c < 0 ? 0 : (c >= n ? n - 1 : c);
      a[q] = __ldcs(vre + (int64_t)k * n + row);
      xv[q] = x[c];
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      cplx<T>& s = acc[q / 3];
      s.re = fma(a[q], xv[q].re, s.re);
      s.im = fma(a[q], xv[q].im, s.im);
    }
  }
  return cplx<T>((acc[0].re + acc[1].re) + acc[2].re, (acc[0].im + acc[1].im) + acc[2].im);
}

// Imaginary-part product of one row: sum_k i Im(a_k) x_{c_k}.
template <typename T>
__device__ __forceinline__ cplx<T> dia_row_im(const T* __restrict__ vim, const cplx<T>* x, int64_t n, int64_t Nx,
                                              int64_t NxNy, int64_t row) {
  cplx<T> acc(T(0), T(0));
#pragma unroll
  for (int k = 0; k < 27; ++k) {
    const int di = k % 3 - 1, dj = (k / 3) % 3 - 1, dl = k / 9 - 1;
    int64_t c = row + di + Nx * dj + NxNy * dl;
    c = c < 0 ? 0 : (c >= n ? n - 1 : c);
    const T b = vim[(int64_t)k * n + row];
    const cplx<T> xv = x[c];
    acc.re = fma(-b, xv.im, acc.re);
    acc.im = fma(b, xv.re, acc.im);
  }
  return acc;
}

// Double-word i Im(a) x part of a row flagged complex (imaginary matrix parts as (hi, lo) float
// pairs, slot-major with slot stride ns >= n): re -= Im(a) x.im, im += Im(a) x.re, Dot2-style
// accumulation on the FP32 pipe, both components in one packed accumulator.
// CLAMP: gather indices clamped into [0, n) (needed for rows within one stencil reach of
// either end).
template <bool CLAMP>
__device__ __forceinline__ cw dia_row_im_dw2(const float2* __restrict__ vim, const cw* x, int64_t n, int64_t ns,
                                             int64_t Nx, int64_t NxNy, int64_t row) {
  dacc2 acc;
#pragma unroll
  for (int k = 0; k < 27; ++k) {
    const int di = k % 3 - 1, dj = (k / 3) % 3 - 1, dl = k / 9 - 1;
    int64_t c = row + di + Nx * dj + NxNy * dl;
    if (CLAMP) c = c < 0 ? 0 : (c >= n ? n - 1 : c);
    const float2 b = vim[(int64_t)k * ns + row];
    const cw xv = x[c];
    acc.mac(make_float2(-b.x, b.x), make_float2(-b.y, b.y), make_float2(xv.ih, xv.rh), make_float2(xv.il, xv.rl));
  }
  float2 hi, lo;
  acc.get(hi, lo);
  return cw_from(hi, lo);
}

// Deterministic block sum of NV doubles per thread (fixed shuffle tree, then warps in order).
// Every thread gets the result. `sh` must hold NV * (kBlock/32) doubles.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh) {
#pragma unroll
  for (int q = 0; q < NV; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[q * (kBlock / 32) + w] = v[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kBlock / 32; ++i) s += sh[q * (kBlock / 32) + i];
    v[q] = s;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------------
// Bounded grid barrier for cooperative (co-resident) launches. Arrival: fence, then one atomic
// per block; the last arriver resets the count and bumps the generation. Waiters spin on the
// generation with an acquire load (no sleep between polls: one polling thread per block, and a
// sleep's wake-up granularity would add to every barrier), give up after kSpinLimit polls or
// kTimeoutNs nanoseconds,
// record DEV_TIMEOUT in the status word and return false so the kernel can unwind.
// ---------------------------------------------------------------------------------------------
struct GridBar {
  unsigned count;
  unsigned gen;
  int status;  // DEV_* bits
  int pad;
};

constexpr unsigned long long kTimeoutNs = 4000000000ull;  // 4 s
constexpr unsigned kSpinLimit = 1000000000u;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// `extra` adds arrivals the barrier waits for (0 in normal operation; the fault-injection test
// sets 1, so no generation bump ever happens and every block gives up after `timeout_ns`).
__device__ __forceinline__ bool grid_barrier(GridBar* bar, unsigned nblocks, unsigned extra = 0,
                                             unsigned long long timeout_ns = kTimeoutNs) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned g = ld_acquire(&bar->gen);
    __threadfence();
    const unsigned arrived = atomicAdd(&bar->count, 1u) + 1u;
    if (arrived == nblocks + extra) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      const unsigned long long t0 = globaltimer();
      unsigned spins = 0;
      while (ld_acquire(&bar->gen) == g) {
        ++spins;
        if (spins > kSpinLimit || ((spins & 1023u) == 0 && globaltimer() - t0 > timeout_ns)) {
          atomicOr(&bar->status, DEV_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    if (*((volatile int*)&bar->status) != 0) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace helm
