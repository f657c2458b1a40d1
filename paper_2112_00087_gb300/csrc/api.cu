// extern "C" entry points of libhelm (declared and documented in include/helm.h).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"

namespace helm {

static thread_local std::string g_err;
static thread_local helm_profile g_prof;

helm_profile& last_profile() { return g_prof; }

FaultMode fault_mode() {
  const char* e = getenv("HELM_FAULT_INJECT");
  if (!e) return FAULT_NONE;
  if (strcmp(e, "barrier") == 0) return FAULT_BARRIER;
  if (strcmp(e, "oom") == 0) return FAULT_OOM;
  return FAULT_NONE;
}

helm_status set_error(helm_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

helm_status cuda_error(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky-free error so later calls are not poisoned
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? HELM_ERR_OOM : HELM_ERR_CUDA;
}

namespace {

__global__ void scatter_dirichlet(const int32_t* __restrict__ nodes, const cd* __restrict__ p, int n_dir,
                                  uint8_t* __restrict__ is_dir, cd* __restrict__ p_full) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n_dir) {
    is_dir[nodes[t]] = 1;
    p_full[nodes[t]] = p[t];
  }
}

bool valid_opts(const helm_solve_opts* o) {
  if (!o) return false;
  if (o->solver != HELM_SOLVER_GMRES && o->solver != HELM_SOLVER_COCG && o->solver != HELM_SOLVER_BICGSTAB &&
      o->solver != HELM_SOLVER_TFQMR)
    return false;
  if (!(o->tol > 0.0) || o->maxit < 1) return false;
  if (o->solver == HELM_SOLVER_GMRES && (o->restart < 1 || o->restart > 128)) return false;
  if (o->precond != HELM_PRECOND_NONE && o->precond != HELM_PRECOND_RAS && o->precond != HELM_PRECOND_JACOBI &&
      o->precond != HELM_PRECOND_ORAS && o->precond != HELM_PRECOND_ORAS2)
    return false;
  if (o->precond == HELM_PRECOND_JACOBI && o->solver == HELM_SOLVER_GMRES) return false;
  if (o->precond == HELM_PRECOND_RAS || o->precond == HELM_PRECOND_ORAS || o->precond == HELM_PRECOND_ORAS2) {
    if (o->solver != HELM_SOLVER_GMRES) return false;
    if (o->ras_parts[0] < 1 || o->ras_parts[1] < 1 || o->ras_parts[2] < 1 || o->ras_overlap < 0) return false;
  }
  if (o->precond == HELM_PRECOND_ORAS2)
    for (int q = 0; q < 2; ++q)
      if (!std::isfinite(o->robin_lo[q]) || !std::isfinite(o->robin_hi[q])) return false;
  if (o->mixed < 0 || o->mixed > 2) return false;
  if (o->mixed) {
    if (o->solver != HELM_SOLVER_COCG) return false;
    if (!(o->inner_tol > 0.0) || o->inner_maxit < 1 || o->max_outer < 1) return false;
  }
  return true;
}

}  // namespace
}  // namespace helm

using namespace helm;

extern "C" {

const char* helm_last_error(void) { return g_err.c_str(); }

helm_status helm_last_profile(helm_profile* out) {
  if (!out) return set_error(HELM_ERR_ARG, "helm_last_profile: null argument");
  *out = g_prof;
  return HELM_OK;
}

helm_status helm_create(helm_ctx** out, const helm_mesh_desc* mesh, const helm_phys* phys, void* stream) {
  if (!out || !mesh || !phys) return set_error(HELM_ERR_ARG, "helm_create: null argument");
  *out = nullptr;
  if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1)
    return set_error(HELM_ERR_ARG, "helm_create: nx, ny, nz must be >= 1");
  if (!(mesh->Lx > 0 && mesh->Ly > 0 && mesh->Lz > 0 && std::isfinite(mesh->Lx) && std::isfinite(mesh->Ly) &&
        std::isfinite(mesh->Lz)))
    return set_error(HELM_ERR_ARG, "helm_create: box lengths must be finite and > 0");
  if (!(phys->c > 0 && phys->rho > 0)) return set_error(HELM_ERR_ARG, "helm_create: c and rho must be > 0");
  const int64_t Nx = mesh->nx + 1, Ny = mesh->ny + 1, Nz = mesh->nz + 1;
  const int64_t n = Nx * Ny * Nz;
  const int64_t nnz = (3 * Nx - 2) * (3 * Ny - 2) * (3 * Nz - 2);
  if (nnz >= (int64_t)INT32_MAX) return set_error(HELM_ERR_ARG, "helm_create: lattice too large for int32 CSR");
  helm_ctx* c = new (std::nothrow) helm_ctx;
  if (!c) return set_error(HELM_ERR_OOM, "helm_create: host allocation failed");
  memset(c, 0, sizeof(*c));
  c->mesh = *mesh;
  c->phys = *phys;
  c->stream = (cudaStream_t)stream;
  c->n = n;
  c->nnz = nnz;
  c->nbf = 2 * ((int64_t)mesh->ny * mesh->nz + (int64_t)mesh->nx * mesh->nz + (int64_t)mesh->nx * mesh->ny);
  helm_status st = HELM_OK;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) st = cuda_error(e, "cudaGetDevice");
  if (st == HELM_OK) st = dev_alloc(&c->rowptr, n + 1);
  if (st == HELM_OK) st = dev_alloc(&c->col, nnz);
  if (st == HELM_OK) st = dev_alloc(&c->beta, c->nbf);
  if (st == HELM_OK) st = dev_alloc(&c->is_dir, n);
  if (st == HELM_OK) st = dev_alloc(&c->p_dir_full, n);
  if (st == HELM_OK) {
    e = cudaMemsetAsync(c->beta, 0, c->nbf * sizeof(cd), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->is_dir, 0, n, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->p_dir_full, 0, n * sizeof(cd), c->stream);
    if (e != cudaSuccess) st = cuda_error(e, "helm_create memset");
  }
  if (st == HELM_OK) st = build_pattern(c);
  if (st != HELM_OK) {
    helm_destroy(c);
    return st;
  }
  *out = c;
  return HELM_OK;
}

void helm_destroy(helm_ctx* c) {
  if (!c) return;
  if (c->stream || true) cudaStreamSynchronize(c->stream);
  cudaFree(c->rowptr);
  cudaFree(c->col);
  cudaFree(c->beta);
  cudaFree(c->dir_nodes);
  cudaFree(c->p_dir);
  cudaFree(c->is_dir);
  cudaFree(c->p_dir_full);
  delete c;
}

helm_status helm_set_boundary(helm_ctx* c, const double* beta_face, const int32_t* dir_nodes, int32_t n_dir,
                              const double* p_dir) {
  if (!c) return set_error(HELM_ERR_ARG, "helm_set_boundary: null context");
  if (n_dir < 0 || n_dir > c->n) return set_error(HELM_ERR_ARG, "helm_set_boundary: n_dir out of range");
  if (n_dir > 0 && (!dir_nodes || !p_dir)) return set_error(HELM_ERR_ARG, "helm_set_boundary: null Dirichlet data");
  // validate node ids on the host before any device work (small array)
  std::vector<int32_t> h(n_dir);
  if (n_dir > 0) {
    cudaError_t e = cudaMemcpyAsync(h.data(), dir_nodes, n_dir * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_error(e, "helm_set_boundary: reading dir_nodes");
    std::vector<int32_t> s(h);
    std::sort(s.begin(), s.end());
    if (s.front() < 0 || s.back() >= c->n) return set_error(HELM_ERR_ARG, "helm_set_boundary: node id out of range");
    if (std::adjacent_find(s.begin(), s.end()) != s.end())
      return set_error(HELM_ERR_ARG, "helm_set_boundary: duplicate Dirichlet node");
  }
  cudaFree(c->dir_nodes);
  cudaFree(c->p_dir);
  c->dir_nodes = nullptr;
  c->p_dir = nullptr;
  c->n_dir = 0;
  helm_status st = dev_alloc(&c->dir_nodes, n_dir);
  if (st == HELM_OK) st = dev_alloc(&c->p_dir, n_dir);
  if (st != HELM_OK) return st;
  cudaError_t e = cudaSuccess;
  if (beta_face) e = cudaMemcpyAsync(c->beta, beta_face, c->nbf * sizeof(cd), cudaMemcpyDeviceToDevice, c->stream);
  else e = cudaMemsetAsync(c->beta, 0, c->nbf * sizeof(cd), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->is_dir, 0, c->n, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->p_dir_full, 0, c->n * sizeof(cd), c->stream);
  if (n_dir > 0) {
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->dir_nodes, dir_nodes, n_dir * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->p_dir, p_dir, n_dir * sizeof(cd), cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) {
      scatter_dirichlet<<<(n_dir + 255) / 256, 256, 0, c->stream>>>(c->dir_nodes, c->p_dir, n_dir, c->is_dir,
                                                                  c->p_dir_full);
      e = cudaGetLastError();
    }
  }
  if (e != cudaSuccess) return cuda_error(e, "helm_set_boundary");
  c->n_dir = n_dir;
  c->has_boundary = true;
  return HELM_OK;
}

helm_status helm_sizes(const helm_ctx* c, int64_t* n_nodes, int64_t* nnz, int64_t* n_bface, int32_t* n_dir) {
  if (!c) return set_error(HELM_ERR_ARG, "helm_sizes: null context");
  if (n_nodes) *n_nodes = c->n;
  if (nnz) *nnz = c->nnz;
  if (n_bface) *n_bface = c->nbf;
  if (n_dir) *n_dir = c->n_dir;
  return HELM_OK;
}

helm_status helm_assemble(helm_ctx* c, double freq_hz, int32_t precision, int32_t format, helm_matrix** A_out,
                          double* b_out) {
  if (!c || !A_out) return set_error(HELM_ERR_ARG, "helm_assemble: null argument");
  *A_out = nullptr;
  if (!(freq_hz >= 0) || !std::isfinite(freq_hz)) return set_error(HELM_ERR_ARG, "helm_assemble: bad frequency");
  if (precision != HELM_C128 && precision != HELM_C64) return set_error(HELM_ERR_ARG, "helm_assemble: bad precision");
  if (format != HELM_FMT_CSR && format != HELM_FMT_DIA27) return set_error(HELM_ERR_ARG, "helm_assemble: bad format");
  helm_matrix* A = new (std::nothrow) helm_matrix;
  if (!A) return set_error(HELM_ERR_OOM, "helm_assemble: host allocation failed");
  memset(A, 0, sizeof(*A));
  A->ctx = c;
  A->n = c->n;
  A->nnz = format == HELM_FMT_DIA27 ? 27 * c->n : c->nnz;
  A->precision = precision;
  A->format = format;
  A->freq = freq_hz;
  helm_status st = dev_alloc(&A->val, A->nnz);
  if (st == HELM_OK && precision == HELM_C64) st = dev_alloc(&A->val32, A->nnz);
  if (st == HELM_OK && format == HELM_FMT_DIA27) st = dev_alloc(&A->cflag, c->n);
  if (st == HELM_OK)
    st = assemble_values(c, freq_hz, A->val, (cd*)b_out, c->stream, true, format == HELM_FMT_DIA27, A->cflag);
  if (st == HELM_OK && precision == HELM_C64) st = cast_values(A->val, A->val32, A->nnz, c->stream);
  if (st != HELM_OK) {
    helm_matrix_free(A);
    return st;
  }
  *A_out = A;
  return HELM_OK;
}

void helm_matrix_free(helm_matrix* A) {
  if (!A) return;
  cudaStreamSynchronize(A->ctx ? A->ctx->stream : 0);
  cudaFree(A->val);
  cudaFree(A->val32);
  cudaFree(A->cflag);
  delete A;
}

helm_status helm_matrix_csr(const helm_matrix* A, int64_t* n, int64_t* nnz, int32_t* precision,
                            const int32_t** rowptr, const int32_t** col, const void** val) {
  if (!A) return set_error(HELM_ERR_ARG, "helm_matrix_csr: null matrix");
  if (A->format != HELM_FMT_CSR) return set_error(HELM_ERR_ARG, "helm_matrix_csr: matrix is not CSR");
  if (n) *n = A->n;
  if (nnz) *nnz = A->nnz;
  if (precision) *precision = A->precision;
  if (rowptr) *rowptr = A->ctx->rowptr;
  if (col) *col = A->ctx->col;
  if (val) *val = A->precision == HELM_C64 ? (const void*)A->val32 : (const void*)A->val;
  return HELM_OK;
}

helm_status helm_matrix_dia27(const helm_matrix* A, int64_t* n, int32_t* precision, const void** val) {
  if (!A) return set_error(HELM_ERR_ARG, "helm_matrix_dia27: null matrix");
  if (A->format != HELM_FMT_DIA27) return set_error(HELM_ERR_ARG, "helm_matrix_dia27: matrix is not DIA27");
  if (n) *n = A->n;
  if (precision) *precision = A->precision;
  if (val) *val = A->precision == HELM_C64 ? (const void*)A->val32 : (const void*)A->val;
  return HELM_OK;
}

helm_status helm_spmv(const helm_matrix* A, const void* x, void* y, void* stream) {
  if (!A || !x || !y) return set_error(HELM_ERR_ARG, "helm_spmv: null argument");
  if (x == y) return set_error(HELM_ERR_ARG, "helm_spmv: x and y must not overlap");
  cudaStream_t s = stream ? (cudaStream_t)stream : A->ctx->stream;
  if (A->format == HELM_FMT_DIA27) {
    const int64_t Nx = A->ctx->mesh.nx + 1, NxNy = Nx * (A->ctx->mesh.ny + 1);
    if (A->precision == HELM_C64) return spmv_dia_c64(A->val32, A->cflag, (const cf*)x, (cf*)y, A->n, Nx, NxNy, s);
    return spmv_dia_c128(A->val, A->cflag, (const cd*)x, (cd*)y, A->n, Nx, NxNy, s);
  }
  if (A->precision == HELM_C64)
    return spmv_c64(A->ctx->rowptr, A->ctx->col, A->val32, (const cf*)x, (cf*)y, A->n, s);
  return spmv_c128(A->ctx->rowptr, A->ctx->col, A->val, (const cd*)x, (cd*)y, A->n, s);
}

helm_status helm_reduce(int32_t op, int64_t n, const double* x, const double* y, double* out, void* stream) {
  if (op < 0 || op > 2 || n < 0 || !out || (n > 0 && !x) || (n > 0 && op != 2 && !y))
    return set_error(HELM_ERR_ARG, "helm_reduce: bad argument");
  if (n == 0) {
    out[0] = out[1] = 0.0;
    return HELM_OK;
  }
  return reduce_c128(op, n, (const cd*)x, (const cd*)y, out, (cudaStream_t)stream);
}

helm_status helm_reduce_noalloc(int32_t op, int64_t n, const double* x, const double* y, double* out, void* stream) {
  if (op < 0 || op > 2 || n < 0 || !out || (n > 0 && !x) || (n > 0 && op != 2 && !y))
    return set_error(HELM_ERR_ARG, "helm_reduce_noalloc: bad argument");
  if (n == 0) {
    out[0] = out[1] = 0.0;
    return HELM_OK;
  }
  return reduce_c128_noalloc(op, n, (const cd*)x, (const cd*)y, out, (cudaStream_t)stream);
}

helm_status helm_solve(helm_ctx* c, const double* freqs_hz, int32_t nfreq, const helm_solve_opts* opts,
                       double* p_out, helm_solve_stats* stats) {
  if (!c || !freqs_hz || !p_out || !stats || nfreq < 0) return set_error(HELM_ERR_ARG, "helm_solve: bad argument");
  if (!valid_opts(opts)) return set_error(HELM_ERR_ARG, "helm_solve: invalid options");
  for (int f = 0; f < nfreq; ++f)
    if (!(freqs_hz[f] >= 0) || !std::isfinite(freqs_hz[f])) return set_error(HELM_ERR_ARG, "helm_solve: bad frequency");
  if (nfreq == 0) return HELM_OK;
  memset(&last_profile(), 0, sizeof(helm_profile));
  if (opts->solver == HELM_SOLVER_COCG || opts->solver == HELM_SOLVER_BICGSTAB || opts->solver == HELM_SOLVER_TFQMR) {
    std::vector<BatchSystem> sys(nfreq);
    for (int f = 0; f < nfreq; ++f) sys[f] = BatchSystem{c, freqs_hz[f], (cd*)p_out + (size_t)f * c->n, &stats[f], nullptr};
    return solve_cocg_batch(sys.data(), nfreq, *opts, c->stream);
  }
  helm_status overall = HELM_OK;
  for (int f = 0; f < nfreq; ++f) {
    helm_status st = solve_gmres(c, freqs_hz[f], *opts, (cd*)p_out + (size_t)f * c->n, &stats[f]);
    if (st == HELM_ERR_CUDA || st == HELM_ERR_OOM || st == HELM_TIMEOUT || st == HELM_ERR_ARG) return st;
    if (st != HELM_OK && overall == HELM_OK) overall = st;
  }
  if (overall != HELM_OK) set_error(overall, "helm_solve: at least one frequency did not converge");
  return overall;
}

helm_status helm_solve_batch(helm_ctx* const* ctxs, const double* freqs_hz, int32_t nsys, const helm_solve_opts* opts,
                             double* const* p_out, helm_solve_stats* stats) {
  if (!ctxs || !freqs_hz || !p_out || !stats || nsys < 0) return set_error(HELM_ERR_ARG, "helm_solve_batch: bad argument");
  if (!valid_opts(opts) || opts->solver == HELM_SOLVER_GMRES)
    return set_error(HELM_ERR_ARG, "helm_solve_batch: invalid options (COCG, BiCGSTAB or TFQMR)");
  if (nsys == 0) return HELM_OK;
  memset(&last_profile(), 0, sizeof(helm_profile));
  std::vector<BatchSystem> sys(nsys);
  for (int k = 0; k < nsys; ++k) {
    if (!ctxs[k] || !p_out[k] || !(freqs_hz[k] >= 0) || !std::isfinite(freqs_hz[k]))
      return set_error(HELM_ERR_ARG, "helm_solve_batch: bad system " + std::to_string(k));
    if (ctxs[k]->device != ctxs[0]->device) return set_error(HELM_ERR_ARG, "helm_solve_batch: mixed devices");
    sys[k] = BatchSystem{ctxs[k], freqs_hz[k], (cd*)p_out[k], &stats[k], nullptr};
  }
  return solve_cocg_batch(sys.data(), nsys, *opts, ctxs[0]->stream);
}

helm_status helm_adjoint_grad(helm_ctx* c, const double* freqs_hz, int32_t nfreq, const helm_solve_opts* opts,
                              const double* p, const double* w_node, double* grad_beta, double* grad_pdir,
                              double* J_out) {
  if (!c || !freqs_hz || nfreq < 0 || !p || !w_node || !grad_beta || (c->n_dir > 0 && !grad_pdir))
    return set_error(HELM_ERR_ARG, "helm_adjoint_grad: bad argument");
  if (!valid_opts(opts)) return set_error(HELM_ERR_ARG, "helm_adjoint_grad: invalid options");
  return adjoint_grad(c, freqs_hz, nfreq, *opts, (const cd*)p, w_node, nullptr, (cd*)grad_beta, (cd*)grad_pdir,
                      J_out);
}

helm_status helm_adjoint_seed(helm_ctx* c, const double* freqs_hz, int32_t nfreq, const helm_solve_opts* opts,
                              const double* p, const double* grad_p, double* grad_beta, double* grad_pdir) {
  if (!c || !freqs_hz || nfreq < 0 || !p || !grad_p || !grad_beta || (c->n_dir > 0 && !grad_pdir))
    return set_error(HELM_ERR_ARG, "helm_adjoint_seed: bad argument");
  if (!valid_opts(opts)) return set_error(HELM_ERR_ARG, "helm_adjoint_seed: invalid options");
  return adjoint_grad(c, freqs_hz, nfreq, *opts, (const cd*)p, nullptr, (const cd*)grad_p, (cd*)grad_beta,
                      (cd*)grad_pdir, nullptr);
}

}  // extern "C"
