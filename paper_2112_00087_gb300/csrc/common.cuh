// Internal declarations shared by the libhelm translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "helm.h"

namespace helm {

// ---------------------------------------------------------------------------------------------
// Complex arithmetic. Paper Sec. 4: instead of the vendor complex type, a small complex<T>
// template with the usual operators, stored as (re, im) -- here aligned so that one element
// is a single 16-byte (double) or 8-byte (float) vector load.
// ---------------------------------------------------------------------------------------------
template <typename T> struct alignas(2 * sizeof(T)) cplx {
  T re, im;
  cplx() = default;
  __host__ __device__ __forceinline__ constexpr cplx(T r, T i = T(0)) : re(r), im(i) {}
};
using cd = cplx<double>;
using cf = cplx<float>;

template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator*(cplx<T> a, cplx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator*(T s, cplx<T> a) { return {s * a.re, s * a.im}; }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> conj(cplx<T> a) { return {a.re, -a.im}; }
template <typename T>
__host__ __device__ __forceinline__ T abs2(cplx<T> a) { return a.re * a.re + a.im * a.im; }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> cdiv(cplx<T> a, cplx<T> b) {
  // plain (a conj(b)) / |b|^2; operands here are O(1)-scaled Krylov scalars
  T d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
// acc += a * b (complex multiply-add as four fused multiply-adds)
template <typename T>
__host__ __device__ __forceinline__ void cfma(cplx<T>& acc, cplx<T> a, cplx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}

// ---------------------------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------------------------
helm_status set_error(helm_status st, const std::string& msg);
helm_profile& last_profile();  // thread-local record behind helm_last_profile
helm_status cuda_error(cudaError_t e, const char* what);

#define HELM_CUDA(call)                                              \
  do {                                                               \
    cudaError_t _e = (call);                                         \
    if (_e != cudaSuccess) return ::helm::cuda_error(_e, #call);     \
  } while (0)

// Device-side status bits written by kernels into a global status word.
enum : int {
  DEV_TIMEOUT = 1,      // a bounded grid barrier gave up
  DEV_BAD_INDEX = 2,    // an index failed a bounds check
};

}  // namespace helm

// ---------------------------------------------------------------------------------------------
// Library objects
// ---------------------------------------------------------------------------------------------
struct helm_ctx {
  helm_mesh_desc mesh;
  helm_phys phys;
  cudaStream_t stream;
  int device;
  int64_t n, nnz, nbf;
  int32_t n_dir;
  bool has_boundary;
  // device buffers owned by the context
  int32_t* rowptr;      // [n+1]   27-point pattern, shared by every matrix of this context
  int32_t* col;         // [nnz]
  helm::cd* beta;       // [nbf]   admittance per boundary quad
  int32_t* dir_nodes;   // [n_dir]
  helm::cd* p_dir;      // [n_dir]
  uint8_t* is_dir;      // [n]     1 on Dirichlet nodes
  helm::cd* p_dir_full; // [n]     prescribed pressure scattered to nodes, 0 elsewhere
};

struct helm_matrix {
  const helm_ctx* ctx;  // pattern owner (must outlive the matrix)
  int64_t n, nnz;       // nnz: stored entries (CSR nnz, or 27 n for the slot-major layout)
  int32_t precision;
  int32_t format;       // HELM_FMT_CSR or HELM_FMT_DIA27
  double freq;
  helm::cd* val;        // complex128 values (always present)
  helm::cf* val32;      // complex64 values (HELM_C64 only)
  uint8_t* cflag;       // DIA27: 1 for rows with a non-zero imaginary entry
};

struct helm_shared {
  const helm_ctx* ctx;  // lattice and boundary data owner (must outlive this object)
  int64_t n;
  int32_t precision;
  double* comp;         // [K | M | Re B | Im B], 4 x 27 n doubles
  float* comp32;        // the same in FP32 (HELM_C64 only)
  uint8_t* bflag;       // [n] rows with a wall term
};

namespace helm {

// assemble.cu
helm_status build_pattern(helm_ctx* ctx);
// eliminate = false: the matrix before Dirichlet elimination (b is not written).
// dia = true: slot-major 27-point layout val[k * n + row] (27 n entries) instead of CSR.
// cflag (u8 [n], may be null): 1 for rows with a non-zero imaginary entry.
helm_status assemble_values(const helm_ctx* ctx, double freq, cd* val, cd* b, cudaStream_t s,
                            bool eliminate = true, bool dia = false, uint8_t* cflag = nullptr);
helm_status cast_values(const cd* val, cf* val32, int64_t nnz, cudaStream_t s);
// frequency-independent parts [K | M | Re B | Im B] (each 27 n, slot-major) of the eliminated
// matrix, their FP32 copy (if comp32 != null) and the rows with a wall term
helm_status assemble_components(const helm_ctx* ctx, double* comp, float* comp32, uint8_t* bflag, cudaStream_t s);
// double-word (hi, lo) float pairs of nslots slot arrays of n doubles, written with slot stride ns >= n
// (padding entries zero)
helm_status split_values(const double* val, float2* out, int64_t n, int64_t ns, int nslots, cudaStream_t s);

// spmv.cu
helm_status spmv_c128(const int32_t* rowptr, const int32_t* col, const cd* val, const cd* x, cd* y,
                      int64_t n, cudaStream_t s);
helm_status spmv_c64(const int32_t* rowptr, const int32_t* col, const cf* val, const cf* x, cf* y,
                     int64_t n, cudaStream_t s);
helm_status spmv_dia_c128(const cd* val, const uint8_t* cflag, const cd* x, cd* y, int64_t n, int64_t Nx,
                          int64_t NxNy, cudaStream_t s);
helm_status spmv_dia_c64(const cf* val, const uint8_t* cflag, const cf* x, cf* y, int64_t n, int64_t Nx,
                         int64_t NxNy, cudaStream_t s);
helm_status reduce_c128(int op, int64_t n, const cd* x, const cd* y, double* out_host, cudaStream_t s);
helm_status reduce_c128_noalloc(int op, int64_t n, const cd* x, const cd* y, double* out_host, cudaStream_t s);

// krylov_cocg.cu
struct BatchSystem {
  const helm_ctx* ctx;
  double freq;
  cd* p_out;
  helm_solve_stats* stats;
  const cd* rhs;  // null: the lifted right-hand side of the Dirichlet data; else this vector
};
helm_status solve_cocg_batch(const BatchSystem* sys, int nsys, const helm_solve_opts& o,
                             cudaStream_t s);

// gmres.cu
helm_status solve_gmres(const helm_ctx* ctx, double freq, const helm_solve_opts& o, cd* p_out,
                        helm_solve_stats* st);
// solve with a prepared matrix / right-hand side (used by the adjoint)
helm_status solve_gmres_system(const helm_ctx* ctx, const int32_t* rowptr, const int32_t* col,
                               const cd* val, double freq, const cd* b, const helm_solve_opts& o,
                               cd* x, helm_solve_stats* st);

// adjoint.cu: gp = dL/dRe p + i dL/dIm p for every frequency ([nfreq][n]); if w is given,
// gp = 2 w p (listener objective) is formed internally and J = sum w |p|^2 returned.
helm_status adjoint_grad(helm_ctx* ctx, const double* freqs, int nfreq, const helm_solve_opts& o,
                         const cd* p, const double* w, const cd* gp, cd* grad_beta, cd* grad_pdir, double* J);

// Host-side fault injection for the failure-detection tests, read from the environment
// variable HELM_FAULT_INJECT: "barrier" (persistent solver barriers wait for a block that does
// not exist and time out after 200 ms) or "oom" (the next device allocation of the library
// reports out-of-memory). Unset in normal use; nothing here can fault the GPU.
enum FaultMode { FAULT_NONE = 0, FAULT_BARRIER = 1, FAULT_OOM = 2 };
FaultMode fault_mode();

// alloc helper: cudaMalloc with OOM mapping
template <typename T>
helm_status dev_alloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return HELM_OK;
  if (fault_mode() == FAULT_OOM)
    return set_error(HELM_ERR_OOM, "device allocation of " + std::to_string(count * sizeof(T)) +
                                       " bytes failed (injected)");
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return set_error(HELM_ERR_OOM, "device allocation of " + std::to_string(count * sizeof(T)) + " bytes failed");
  }
  if (e != cudaSuccess) return cuda_error(e, "cudaMalloc");
  return HELM_OK;
}

}  // namespace helm
