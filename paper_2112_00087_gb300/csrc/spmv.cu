// Standalone SpMV (paper Sec. 4: CSR storage; SpMV "the most time consuming operation") and
// deterministic FP64 reductions (dot products / norms of the Krylov methods).
#include <algorithm>

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

helm_status spmv_c128(const int32_t* rowptr, const int32_t* col, const cd* val, const cd* x, cd* y,
                      int64_t n, cudaStream_t s) {
  if (n == 0) return HELM_OK;
  constexpr int G = 4;
  int64_t blocks = std::min<int64_t>((n + kBlock / G - 1) / (kBlock / G), (int64_t)num_sms() * 8);
  spmv_kernel<G, double><<<(unsigned)blocks, kBlock, 0, s>>>(rowptr, col, val, x, y, n);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

helm_status spmv_c64(const int32_t* rowptr, const int32_t* col, const cf* val, const cf* x, cf* y,
                     int64_t n, cudaStream_t s) {
  if (n == 0) return HELM_OK;
  constexpr int G = 8;
  int64_t blocks = std::min<int64_t>((n + kBlock / G - 1) / (kBlock / G), (int64_t)num_sms() * 8);
  spmv_kernel<G, float><<<(unsigned)blocks, kBlock, 0, s>>>(rowptr, col, val, x, y, n);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

helm_status reduce_c128(int op, int64_t n, const cd* x, const cd* y, double* out_host, cudaStream_t s) {
  const int nparts = std::max(1, std::min<int>(num_sms() * 4, (int)((n + kBlock - 1) / kBlock)));
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

}  // namespace helm
