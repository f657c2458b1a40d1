// Standalone SpMV (paper Sec. 4: CSR storage; the SpMV dominates the Krylov iteration cost) and
// deterministic FP64 reductions (dot products / norms of the Krylov methods).
#include <algorithm>
#include <mutex>
#include <cstdlib>
#include <string>

#include "kernels.cuh"

namespace helm {
namespace {

int g_num_sms = 0;
int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

// y = A x, groups of G lanes per row, grid-stride over row groups (uniform per block).
template <int G, typename T>
__global__ void __launch_bounds__(kBlock) spmv_kernel(const int32_t* __restrict__ rowptr,
                                                      const int32_t* __restrict__ col,
                                                      const cplx<T>* __restrict__ val,
                                                      const cplx<T>* __restrict__ x,
                                                      cplx<T>* __restrict__ y, int64_t n) {
  constexpr int RPB = kBlock / G;  // rows per block pass
  const int gid = threadIdx.x / G, g = threadIdx.x % G;
  for (int64_t base = (int64_t)blockIdx.x * RPB; base < n; base += (int64_t)gridDim.x * RPB) {
    const int64_t row = base + gid;
    const bool valid = row < n;
    cplx<T> s = csr_row27<G, T>(rowptr, col, val, x, row, valid, g);
    if (valid && g == 0) y[row] = s;
  }
}

// y = A x in the slot-major 27-point layout, one thread per row (block-uniform grid-stride):
// real parts for every row, then, if any row of the block is flagged complex, its imaginary
// parts in a second pass.
template <typename T>
__global__ void __launch_bounds__(kBlock) spmv_dia_kernel(const cplx<T>* __restrict__ val,
                                                          const uint8_t* __restrict__ cflag,
                                                          const cplx<T>* __restrict__ x,
                                                          cplx<T>* __restrict__ y, int64_t n, int64_t Nx,
                                                          int64_t NxNy) {
  for (int64_t base = blockIdx.x * (int64_t)kBlock; base < n; base += (int64_t)gridDim.x * kBlock) {
    const int64_t row = base + threadIdx.x;
    const bool valid = row < n;
    const T* vre = reinterpret_cast<const T*>(val);  // split layout: real parts, then imaginary
    const T* vim = vre + 27 * n;
    cplx<T> s(T(0), T(0));
    int c = 0;
    if (valid) {
      s = dia_row_re<T>(vre, x, n, Nx, NxNy, row);
      c = cflag[row];
    }
    if (__syncthreads_or(c)) {
      if (c) {
        const cplx<T> si = dia_row_im<T>(vim, x, n, Nx, NxNy, row);
        s = cplx<T>(s.re + si.re, s.im + si.im);
      }
    }
    if (valid) y[row] = s;
  }
}

// Stage 1: block b sums the contiguous chunk [b*chunk, (b+1)*chunk) (threads strided inside).
__global__ void __launch_bounds__(kBlock) reduce_stage1(int op, const cd* __restrict__ x,
                                                         const cd* __restrict__ y, int64_t n,
                                                         int64_t chunk, double* __restrict__ part) {
  __shared__ double sh[2 * (kBlock / 32)];
  const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  double v[2] = {0.0, 0.0};
  for (int64_t i = lo + threadIdx.x; i < hi; i += kBlock) {
    cd a = x[i];
    if (op == 2) {
      v[0] += a.re * a.re + a.im * a.im;
    } else {
      cd b = y[i];
      if (op == 0) a.im = -a.im;  // conjugate x
      v[0] += a.re * b.re - a.im * b.im;
      v[1] += a.re * b.im + a.im * b.re;
    }
  }
  block_sum<2>(v, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = v[0];
    part[2 * blockIdx.x + 1] = v[1];
  }
}

__global__ void __launch_bounds__(kBlock) reduce_stage2(const double* __restrict__ part, int nparts,
                                                         double* __restrict__ out) {
  __shared__ double sh[2 * (kBlock / 32)];
  double v[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < nparts; i += kBlock) {
    v[0] += part[2 * i];
    v[1] += part[2 * i + 1];
  }
  block_sum<2>(v, sh);
  if (threadIdx.x == 0) {
    out[0] = v[0];
    out[1] = v[1];
  }
}

}  // namespace

// Lanes per row of the CSR product (tuning knobs HELM_SPMV_LANES_C128 / _C64: 2, 4, 8 or 16;
// defaults 4 and 8, the autotuner's choice on the 2.2 M-node lattice).
static int spmv_lanes(const char* env, int def) {
  const char* e = getenv(env);
  const int g = e ? atoi(e) : def;
  return (g == 2 || g == 4 || g == 8 || g == 16) ? g : def;
}

template <typename T>
static helm_status spmv_csr(int G, const int32_t* rowptr, const int32_t* col, const cplx<T>* val, const cplx<T>* x,
                            cplx<T>* y, int64_t n, cudaStream_t s) {
  if (n == 0) return HELM_OK;
  const int64_t blocks = std::min<int64_t>((n + kBlock / G - 1) / (kBlock / G), (int64_t)num_sms() * 8);
  switch (G) {
    case 2: spmv_kernel<2, T><<<(unsigned)blocks, kBlock, 0, s>>>(rowptr, col, val, x, y, n); break;
    case 4: spmv_kernel<4, T><<<(unsigned)blocks, kBlock, 0, s>>>(rowptr, col, val, x, y, n); break;
    case 8: spmv_kernel<8, T><<<(unsigned)blocks, kBlock, 0, s>>>(rowptr, col, val, x, y, n); break;
    default: spmv_kernel<16, T><<<(unsigned)blocks, kBlock, 0, s>>>(rowptr, col, val, x, y, n); break;
  }
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

helm_status spmv_c128(const int32_t* rowptr, const int32_t* col, const cd* val, const cd* x, cd* y,
                      int64_t n, cudaStream_t s) {
  return spmv_csr<double>(spmv_lanes("HELM_SPMV_LANES_C128", 4), rowptr, col, val, x, y, n, s);
}

helm_status spmv_c64(const int32_t* rowptr, const int32_t* col, const cf* val, const cf* x, cf* y,
                     int64_t n, cudaStream_t s) {
  return spmv_csr<float>(spmv_lanes("HELM_SPMV_LANES_C64", 8), rowptr, col, val, x, y, n, s);
}

helm_status spmv_dia_c128(const cd* val, const uint8_t* cflag, const cd* x, cd* y, int64_t n, int64_t Nx,
                          int64_t NxNy, cudaStream_t s) {
  if (n == 0) return HELM_OK;
  int64_t blocks = std::min<int64_t>((n + kBlock - 1) / kBlock, (int64_t)num_sms() * 8);
  spmv_dia_kernel<double><<<(unsigned)blocks, kBlock, 0, s>>>(val, cflag, x, y, n, Nx, NxNy);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

helm_status spmv_dia_c64(const cf* val, const uint8_t* cflag, const cf* x, cf* y, int64_t n, int64_t Nx,
                         int64_t NxNy, cudaStream_t s) {
  if (n == 0) return HELM_OK;
  int64_t blocks = std::min<int64_t>((n + kBlock - 1) / kBlock, (int64_t)num_sms() * 8);
  spmv_dia_kernel<float><<<(unsigned)blocks, kBlock, 0, s>>>(val, cflag, x, y, n, Nx, NxNy);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

helm_status reduce_c128(int op, int64_t n, const cd* x, const cd* y, double* out_host, cudaStream_t s) {
  // partial sums per SM (tuning knob HELM_REDUCE_PARTS_PER_SM, 1..64; default 1, the autotuner's
  // choice on the 2.2 M-node lattice)
  const char* penv = getenv("HELM_REDUCE_PARTS_PER_SM");
  const int per_sm = penv ? std::max(1, std::min(atoi(penv), 64)) : 1;
  const int nparts = std::max(1, std::min<int>(num_sms() * per_sm, (int)((n + kBlock - 1) / kBlock)));
  const int64_t chunk = (n + nparts - 1) / nparts;
  double* buf = nullptr;
  helm_status st = dev_alloc(&buf, 2 * (size_t)nparts + 2);
  if (st != HELM_OK) return st;
  reduce_stage1<<<nparts, kBlock, 0, s>>>(op, x, y, n, chunk, buf);
  reduce_stage2<<<1, kBlock, 0, s>>>(buf, nparts, buf + 2 * nparts);
  cudaError_t e = cudaMemcpyAsync(out_host, buf + 2 * nparts, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_error(e, "reduce");
  if (op == 2) {
    out_host[0] = sqrt(out_host[0]);
    out_host[1] = 0.0;
  }
  return HELM_OK;
}

// ---------------------------------------------------------------------------------------------
// Reduction without allocation. The partial sums live in a file-scope device array instead of
// a cudaMalloc'd buffer, for callers that must not allocate device memory while they run.
// Block b sums the fixed chunk [b*kNoAllocChunk, (b+1)*kNoAllocChunk), so n is limited to
// kNoAllocMaxParts * kNoAllocChunk elements.
// ---------------------------------------------------------------------------------------------
constexpr int kNoAllocMaxParts = 4096;
constexpr int64_t kNoAllocChunk = 4096;
constexpr int64_t kNoAllocMaxN = (int64_t)kNoAllocMaxParts * kNoAllocChunk;  // 16,777,216

// 2 doubles per partial + 2 for the result: 64 KiB + 16 B, held by every device that loads the
// library until the process exits. Shared by all calls: every call overwrites the entries it
// uses before reading them, so nothing needs clearing; calls that overlap on the GPU race.
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocMaxParts + 2];

namespace {
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[256] = {nullptr};  // device address of g_noalloc_scratch, per device
}  // namespace

// Device address of the scratch array on the current device; looked up once per device (the
// host-side symbol is only a stand-in and must never be passed to a kernel).
static helm_status noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "helm_reduce_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= 256) return set_error(HELM_ERR_ARG, "helm_reduce_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "helm_reduce_noalloc: cudaGetSymbolAddress");
    g_noalloc_ptr[dev] = static_cast<double*>(ptr);
  }
  *out = g_noalloc_ptr[dev];
  return HELM_OK;
}

helm_status reduce_c128_noalloc(int op, int64_t n, const cd* x, const cd* y, double* out_host, cudaStream_t s) {
  if (n > kNoAllocMaxN)
    return set_error(HELM_ERR_ARG, "helm_reduce_noalloc: n = " + std::to_string(n) + " exceeds the maximum " +
                                       std::to_string(kNoAllocMaxN) + " of its static scratch");
  double* buf = nullptr;
  helm_status st = noalloc_scratch(&buf);
  if (st != HELM_OK) return st;
  const int nparts = (int)((n + kNoAllocChunk - 1) / kNoAllocChunk);
  // an error left by earlier, unrelated work is reported as such, not as a launch failure here
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "helm_reduce_noalloc: error pending before the call");
  reduce_stage1<<<nparts, kBlock, 0, s>>>(op, x, y, n, kNoAllocChunk, buf);
  reduce_stage2<<<1, kBlock, 0, s>>>(buf, nparts, buf + 2 * kNoAllocMaxParts);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out_host, buf + 2 * kNoAllocMaxParts, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_error(e, "helm_reduce_noalloc");
  if (op == 2) {
    out_host[0] = sqrt(out_host[0]);
    out_host[1] = 0.0;
  }
  return HELM_OK;
}

}  // namespace helm
