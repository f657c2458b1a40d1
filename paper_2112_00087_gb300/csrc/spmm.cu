// Shared-mesh multi-frequency SpMV ("SpMM"): Y_f = A(k_f) X_f for several wavenumbers on one
// lattice, with A(k) = K - k^2 M + i k rho c B (paper Sec. 3.2 Helmholtz operator; the FRF of
// Sec. 3.1 evaluates it at many frequencies on the same mesh). K, M and B do not depend on the
// frequency, so one pass reads each row's K and M entries once and applies them to every
// frequency of the batch; B (the wall term) is read only on the rows that carry it. Per entry
// and frequency the value a = K - k^2 M - k rho c Im B + i k rho c Re B costs one multiply-add
// more than a pre-assembled value, and the matrix bytes per frequency shrink by the batch size.
#include <algorithm>

#include "kernels.cuh"

namespace helm {
namespace {

constexpr int kFB = 8;  // frequencies per pass (accumulators per thread)

template <typename T>
struct FreqBatch {
  T k2[kFB];
  T krc[kFB];
  int nf;
};

// One thread per row; comp = [K | M | Re B | Im B] slot-major (27 n each), X / Y frequency-major
// ([nf][n]). The 27 slots are taken plane by plane (9 at a time, offsets known at compile time):
// the plane's K and M values are loaded once, then every frequency gathers its 9 x values and
// accumulates (K - k^2 M) x. Rows with a wall term add (-k rho c Im B + i k rho c Re B) x in a
// second pass (the same value as the assembled entry, summed in two parts). Gather indices are
// clamped into [0, n) so that padded slots (value 0) read a valid address.
template <typename T>
__global__ void __launch_bounds__(kBlock) spmm_kernel(const T* __restrict__ comp, const uint8_t* __restrict__ bflag,
                                                      const cplx<T>* X, cplx<T>* Y, FreqBatch<T> fb, int64_t n,
                                                      int64_t Nx, int64_t NxNy) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const T* Kc = comp;
  const T* Mc = comp + 27 * n;
  const T* Br = comp + 54 * n;
  const T* Bi = comp + 81 * n;
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < n; row += stride) {
    cplx<T> acc[kFB];
#pragma unroll
    for (int f = 0; f < kFB; ++f) acc[f] = cplx<T>(T(0), T(0));
#pragma unroll
    for (int dl = -1; dl <= 1; ++dl) {
      T kv[9], mv[9];
      int64_t cc[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const int di = q % 3 - 1, dj = q / 3 - 1;
        const int64_t e = (int64_t)(q + 9 * (dl + 1)) * n + row;
        int64_t c = row + di + Nx * dj + NxNy * dl;
        cc[q] = c < 0 ? 0 : (c >= n ? n - 1 : c);
        kv[q] = __ldcs(Kc + e);
        mv[q] = __ldcs(Mc + e);
      }
#pragma unroll
      for (int f = 0; f < kFB; ++f) {
        if (f < fb.nf) {
          const T mk2 = -fb.k2[f];
          const cplx<T>* Xf = X + (int64_t)f * n;
#pragma unroll
          for (int q = 0; q < 9; ++q) {
            const cplx<T> xv = Xf[cc[q]];
            const T a = fma(mk2, mv[q], kv[q]);
            acc[f].re = fma(a, xv.re, acc[f].re);
            acc[f].im = fma(a, xv.im, acc[f].im);
          }
        }
      }
    }
    if (bflag[row]) {
      for (int k = 0; k < 27; ++k) {
        const int di = k % 3 - 1, dj = (k / 3) % 3 - 1, dl = k / 9 - 1;
        int64_t c = row + di + Nx * dj + NxNy * dl;
        c = c < 0 ? 0 : (c >= n ? n - 1 : c);
        const int64_t e = (int64_t)k * n + row;
        const T br = Br[e], bi = Bi[e];
        if (br == T(0) && bi == T(0)) continue;
#pragma unroll
        for (int f = 0; f < kFB; ++f) {
          if (f < fb.nf) {
            const cplx<T> xv = X[(int64_t)f * n + c];
            const T are = -fb.krc[f] * bi, aim = fb.krc[f] * br;
            acc[f].re = fma(are, xv.re, fma(-aim, xv.im, acc[f].re));
            acc[f].im = fma(are, xv.im, fma(aim, xv.re, acc[f].im));
          }
        }
      }
    }
#pragma unroll
    for (int f = 0; f < kFB; ++f)
      if (f < fb.nf) Y[(int64_t)f * n + row] = acc[f];
  }
}

// Frequency-interleaved form: X and Y node-major ([n][F], the F <= kFB frequencies of a node
// contiguous), so each neighbour's F values arrive in one contiguous F * sizeof(complex) block
// (16-byte vector loads) instead of F separate gathers, and the matrix row (K, M) is read once
// for all F frequencies. Same arithmetic per frequency as spmm_kernel (the wall term in a second
// pass on flagged rows).
// 16-byte vector loads / stores of a node's F complex values (F * sizeof(complex) is a multiple of 16)
template <int F>
__device__ __forceinline__ void load_block(const cplx<float>* p, cplx<float> (&z)[F]) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int u = 0; u < F / 2; ++u) {
    const float4 v = q[u];
    z[2 * u] = cplx<float>(v.x, v.y);
    z[2 * u + 1] = cplx<float>(v.z, v.w);
  }
}
template <int F>
__device__ __forceinline__ void load_block(const cplx<double>* p, cplx<double> (&z)[F]) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int u = 0; u < F; ++u) {
    const double2 v = q[u];
    z[u] = cplx<double>(v.x, v.y);
  }
}
template <int F>
__device__ __forceinline__ void store_block(cplx<float>* p, const cplx<float> (&z)[F]) {
  float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
  for (int u = 0; u < F / 2; ++u) q[u] = make_float4(z[2 * u].re, z[2 * u].im, z[2 * u + 1].re, z[2 * u + 1].im);
}
template <int F>
__device__ __forceinline__ void store_block(cplx<double>* p, const cplx<double> (&z)[F]) {
  double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
  for (int u = 0; u < F; ++u) q[u] = make_double2(z[u].re, z[u].im);
}

// Frequency-interleaved form: X and Y node-major ([n][F], the F <= kFB frequencies of a node
// contiguous), so each neighbour's F values arrive in one contiguous F * sizeof(complex) block
// (16-byte vector loads) instead of F separate gathers, and the matrix row (K, M) is read once
// for all F frequencies. Same arithmetic per frequency as spmm_kernel (the wall term in a second
// pass on flagged rows).
template <typename T, int F>
__global__ void __launch_bounds__(kBlock) spmm_il_kernel(const T* __restrict__ comp, const uint8_t* __restrict__ bflag,
                                                         const cplx<T>* X, cplx<T>* Y, FreqBatch<T> fb, int64_t n,
                                                         int64_t Nx, int64_t NxNy) {
  static_assert((F * sizeof(cplx<T>)) % 16 == 0, "16-byte vector loads of a node's F values");
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const T* Kc = comp;
  const T* Mc = comp + 27 * n;
  const T* Br = comp + 54 * n;
  const T* Bi = comp + 81 * n;
  T mk2[F];
#pragma unroll
  for (int f = 0; f < F; ++f) mk2[f] = -fb.k2[f];
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < n; row += stride) {
    cplx<T> acc[F];
#pragma unroll
    for (int f = 0; f < F; ++f) acc[f] = cplx<T>(T(0), T(0));
#pragma unroll
    for (int k = 0; k < 27; ++k) {
      const int di = k % 3 - 1, dj = (k / 3) % 3 - 1, dl = k / 9 - 1;
      const int64_t e = (int64_t)k * n + row;
      int64_t c = row + di + Nx * dj + NxNy * dl;
      c = c < 0 ? 0 : (c >= n ? n - 1 : c);
      const T kv = __ldcs(Kc + e), mv = __ldcs(Mc + e);
      cplx<T> xz[F];
      load_block<F>(X + c * F, xz);
#pragma unroll
      for (int f = 0; f < F; ++f) {
        const T a = fma(mk2[f], mv, kv);
        acc[f].re = fma(a, xz[f].re, acc[f].re);
        acc[f].im = fma(a, xz[f].im, acc[f].im);
      }
    }
    if (bflag[row]) {
      for (int k = 0; k < 27; ++k) {
        const int di = k % 3 - 1, dj = (k / 3) % 3 - 1, dl = k / 9 - 1;
        int64_t c = row + di + Nx * dj + NxNy * dl;
        c = c < 0 ? 0 : (c >= n ? n - 1 : c);
        const int64_t e = (int64_t)k * n + row;
        const T br = Br[e], bi = Bi[e];
        if (br == T(0) && bi == T(0)) continue;
#pragma unroll
        for (int f = 0; f < F; ++f) {
          const cplx<T> xv = X[c * F + f];
          const T are = -fb.krc[f] * bi, aim = fb.krc[f] * br;
          acc[f].re = fma(are, xv.re, fma(-aim, xv.im, acc[f].re));
          acc[f].im = fma(are, xv.im, fma(aim, xv.re, acc[f].im));
        }
      }
    }
    store_block<F>(Y + row * F, acc);
  }
}

template <typename T, int F>
helm_status spmm_il_launch(const helm_shared* S, const double* freqs, const cplx<T>* X, cplx<T>* Y, const T* comp,
                           cudaStream_t s) {
  const helm_ctx* c = S->ctx;
  const int64_t n = S->n, Nx = c->mesh.nx + 1, NxNy = Nx * (c->mesh.ny + 1);
  int dev = 0, nsm = 1;
  HELM_CUDA(cudaGetDevice(&dev));
  HELM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int64_t blocks = std::min<int64_t>((n + kBlock - 1) / kBlock, (int64_t)nsm * 8);
  FreqBatch<T> fb;
  fb.nf = F;
  for (int f = 0; f < kFB; ++f) {
    const double k = f < F ? 2.0 * 3.14159265358979323846 * freqs[f] / c->phys.c : 0.0;
    fb.k2[f] = (T)(k * k);
    fb.krc[f] = (T)(k * c->phys.rho * c->phys.c);
  }
  spmm_il_kernel<T, F><<<(unsigned)blocks, kBlock, 0, s>>>(comp, S->bflag, X, Y, fb, n, Nx, NxNy);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

template <typename T>
helm_status spmm_run(const helm_shared* S, const double* freqs, int nfreq, const cplx<T>* X, cplx<T>* Y,
                     const T* comp, cudaStream_t s) {
  const helm_ctx* c = S->ctx;
  const int64_t n = S->n, Nx = c->mesh.nx + 1, NxNy = Nx * (c->mesh.ny + 1);
  int dev = 0, nsm = 1;
  HELM_CUDA(cudaGetDevice(&dev));
  HELM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int64_t blocks = std::min<int64_t>((n + kBlock - 1) / kBlock, (int64_t)nsm * 8);
  for (int f0 = 0; f0 < nfreq; f0 += kFB) {
    FreqBatch<T> fb;
    fb.nf = std::min(kFB, nfreq - f0);
    for (int f = 0; f < kFB; ++f) {
      const double k = f < fb.nf ? 2.0 * 3.14159265358979323846 * freqs[f0 + f] / c->phys.c : 0.0;
      fb.k2[f] = (T)(k * k);
      fb.krc[f] = (T)(k * c->phys.rho * c->phys.c);
    }
    spmm_kernel<T><<<(unsigned)blocks, kBlock, 0, s>>>(comp, S->bflag, X + (int64_t)f0 * n, Y + (int64_t)f0 * n, fb,
                                                       n, Nx, NxNy);
    HELM_CUDA(cudaGetLastError());
  }
  return HELM_OK;
}

}  // namespace
}  // namespace helm

using namespace helm;

extern "C" {

helm_status helm_assemble_shared(helm_ctx* ctx, int32_t precision, helm_shared** out) {
  if (!ctx || !out) return set_error(HELM_ERR_ARG, "helm_assemble_shared: null argument");
  *out = nullptr;
  if (precision != HELM_C128 && precision != HELM_C64)
    return set_error(HELM_ERR_ARG, "helm_assemble_shared: precision must be HELM_C128 or HELM_C64");
  if (!ctx->has_boundary) return set_error(HELM_ERR_ARG, "helm_assemble_shared: call helm_set_boundary first");
  helm_shared* S = new helm_shared;
  S->ctx = ctx;
  S->n = ctx->n;
  S->precision = precision;
  S->comp = nullptr;
  S->comp32 = nullptr;
  S->bflag = nullptr;
  helm_status st = dev_alloc(&S->comp, (size_t)108 * ctx->n);
  if (st == HELM_OK && precision == HELM_C64) st = dev_alloc(&S->comp32, (size_t)108 * ctx->n);
  if (st == HELM_OK) st = dev_alloc(&S->bflag, (size_t)ctx->n);
  if (st == HELM_OK) st = assemble_components(ctx, S->comp, S->comp32, S->bflag, ctx->stream);
  if (st != HELM_OK) {
    helm_shared_free(S);
    return st;
  }
  *out = S;
  return HELM_OK;
}

helm_status helm_spmv_multi(const helm_shared* S, const double* freqs_hz, int32_t nfreq, const void* X, void* Y,
                            void* stream) {
  if (!S || !freqs_hz || nfreq < 0 || (nfreq > 0 && (!X || !Y)))
    return set_error(HELM_ERR_ARG, "helm_spmv_multi: bad argument");
  if (nfreq > 0) {
    // byte ranges [X, X + nfreq n vb) and [Y, Y + nfreq n vb) must be disjoint
    const size_t vb = S->precision == HELM_C64 ? 8 : 16;
    const uintptr_t x0 = (uintptr_t)X, y0 = (uintptr_t)Y, len = (uintptr_t)((size_t)nfreq * (size_t)S->n * vb);
    if (len > 0 && x0 < y0 + len && y0 < x0 + len)
      return set_error(HELM_ERR_ARG, "helm_spmv_multi: X and Y must not overlap");
  }
  for (int f = 0; f < nfreq; ++f)
    if (!(freqs_hz[f] >= 0.0)) return set_error(HELM_ERR_ARG, "helm_spmv_multi: negative or NaN frequency");
  if (nfreq == 0 || S->n == 0) return HELM_OK;
  cudaStream_t s = stream ? (cudaStream_t)stream : S->ctx->stream;
  if (S->precision == HELM_C64)
    return spmm_run<float>(S, freqs_hz, nfreq, (const cf*)X, (cf*)Y, S->comp32, s);
  return spmm_run<double>(S, freqs_hz, nfreq, (const cd*)X, (cd*)Y, S->comp, s);
}

helm_status helm_spmv_multi_interleaved(const helm_shared* S, const double* freqs_hz, int32_t nfreq, const void* X,
                                        void* Y, void* stream) {
  if (!S || !freqs_hz || !X || !Y) return set_error(HELM_ERR_ARG, "helm_spmv_multi_interleaved: null argument");
  const bool c64 = S->precision == HELM_C64;
  const bool ok_nf = c64 ? (nfreq == 2 || nfreq == 4 || nfreq == 8) : (nfreq == 1 || nfreq == 2 || nfreq == 4 || nfreq == 8);
  if (!ok_nf) return set_error(HELM_ERR_ARG, "helm_spmv_multi_interleaved: nfreq must be 2, 4 or 8 (complex64) or 1, 2, 4, 8");
  if (((uintptr_t)X | (uintptr_t)Y) & 15u)
    return set_error(HELM_ERR_ARG, "helm_spmv_multi_interleaved: X and Y must be 16-byte aligned");
  const size_t vb = c64 ? 8 : 16;
  const uintptr_t x0 = (uintptr_t)X, y0 = (uintptr_t)Y, len = (uintptr_t)((size_t)nfreq * (size_t)S->n * vb);
  if (len > 0 && x0 < y0 + len && y0 < x0 + len)
    return set_error(HELM_ERR_ARG, "helm_spmv_multi_interleaved: X and Y must not overlap");
  for (int f = 0; f < nfreq; ++f)
    if (!(freqs_hz[f] >= 0.0)) return set_error(HELM_ERR_ARG, "helm_spmv_multi_interleaved: negative or NaN frequency");
  if (S->n == 0) return HELM_OK;
  cudaStream_t s = stream ? (cudaStream_t)stream : S->ctx->stream;
  if (c64) {
    const cf* x = (const cf*)X;
    cf* y = (cf*)Y;
    if (nfreq == 2) return spmm_il_launch<float, 2>(S, freqs_hz, x, y, S->comp32, s);
    if (nfreq == 4) return spmm_il_launch<float, 4>(S, freqs_hz, x, y, S->comp32, s);
    return spmm_il_launch<float, 8>(S, freqs_hz, x, y, S->comp32, s);
  }
  const cd* x = (const cd*)X;
  cd* y = (cd*)Y;
  if (nfreq == 1) return spmm_il_launch<double, 1>(S, freqs_hz, x, y, S->comp, s);
  if (nfreq == 2) return spmm_il_launch<double, 2>(S, freqs_hz, x, y, S->comp, s);
  if (nfreq == 4) return spmm_il_launch<double, 4>(S, freqs_hz, x, y, S->comp, s);
  return spmm_il_launch<double, 8>(S, freqs_hz, x, y, S->comp, s);
}

void helm_shared_free(helm_shared* S) {
  if (!S) return;
  cudaFree(S->comp);
  cudaFree(S->comp32);
  cudaFree(S->bflag);
  delete S;
}

}  // extern "C"
