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

void helm_shared_free(helm_shared* S) {
  if (!S) return;
  cudaFree(S->comp);
  cudaFree(S->comp32);
  cudaFree(S->bflag);
  delete S;
}

}  // extern "C"
