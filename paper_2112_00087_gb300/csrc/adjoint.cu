// Adjoint gradients of a real loss of the frequency response.
//
// For A_red p = b (A_red complex symmetric after symmetric Dirichlet elimination), a real loss
// L(p) with PyTorch gradient g = dL/dRe p + i dL/dIm p, and lam = A_red^-1 conj(g) (one adjoint
// solve with the same matrix, since A_red^T = A_red), lam_F = lam with the Dirichlet entries
// zeroed:
//   dL/dbeta_e  = -conj(lam_F^T (i k rho c B_e) p)            per boundary quad e,
//   dL/dp_D     =  conj(lam_D - A_DF lam_F)                  per Dirichlet node (A before
//                                                            elimination),
// summed over frequencies. The listener objective J = sum_f sum_i w_i |p_i|^2 has g = 2 w p.
// The paper's Helmholtz problem (Sec. 3.2) supplies A; the gradients are the sensitivities of
// the cavity response to the wall admittance and to the sun-roof pressure.
#include <algorithm>
#include <vector>

#include "kernels.cuh"

namespace helm {
namespace {

__global__ void seed_kernel(const cd* __restrict__ p, const double* __restrict__ w, const cd* __restrict__ gp,
                            cd* __restrict__ rhs, int64_t n, int64_t total) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    if (w) {
      const cd pi = p[t];
      const double wi = 2.0 * w[t % n];
      rhs[t] = cd(wi * pi.re, -wi * pi.im);  // conj(2 w p)
    } else {
      const cd g = gp[t];
      rhs[t] = cd(g.re, -g.im);
    }
  }
}

// Node ids of boundary quad e (vertex (u,v) order (0,0),(1,0),(0,1),(1,1)) and its spacings.
__device__ void quad_nodes(int64_t e, int nx, int ny, int nz, double hx, double hy, double hz, int64_t nd[4],
                           double& hu, double& hv) {
  const int64_t Nx = nx + 1, Ny = ny + 1;
  const int64_t s0 = (int64_t)ny * nz, s1 = (int64_t)nx * nz, s2 = (int64_t)nx * ny;
  int side;
  int64_t q = e;
  if (q < 2 * s0) { side = q < s0 ? 0 : 1; q -= side * s0; }
  else if (q < 2 * s0 + 2 * s1) { q -= 2 * s0; side = q < s1 ? 2 : 3; q -= (side - 2) * s1; }
  else { q -= 2 * s0 + 2 * s1; side = q < s2 ? 4 : 5; q -= (side - 4) * s2; }
  int k = 0;
  for (int dv = 0; dv <= 1; ++dv)
    for (int du = 0; du <= 1; ++du) {
      int64_t i, j, l;
      if (side < 2) {
        const int64_t u = q % ny, v = q / ny;
        i = side == 0 ? 0 : nx; j = u + du; l = v + dv;
        hu = hy; hv = hz;
      } else if (side < 4) {
        const int64_t u = q % nx, v = q / nx;
        i = u + du; j = side == 2 ? 0 : ny; l = v + dv;
        hu = hx; hv = hz;
      } else {
        const int64_t u = q % nx, v = q / nx;
        i = u + du; j = v + dv; l = side == 4 ? 0 : nz;
        hu = hx; hv = hy;
      }
      nd[k++] = i + Nx * (j + Ny * l);
    }
}

__global__ void face_grad_kernel(helm_mesh_desc m, double krc, const cd* __restrict__ lam, const cd* __restrict__ p,
                                 const uint8_t* __restrict__ is_dir, cd* __restrict__ gb, int64_t nbf) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nbf) return;
  int64_t nd[4];
  double hu, hv;
  quad_nodes(e, m.nx, m.ny, m.nz, m.Lx / m.nx, m.Ly / m.ny, m.Lz / m.nz, nd, hu, hv);
  // quad mass entry for vertices a=(ua,va), b=(ub,vb): (hu/3 or hu/6)(hv/3 or hv/6)
  cd s(0.0, 0.0);
  for (int a = 0; a < 4; ++a) {
    if (is_dir[nd[a]]) continue;
    const cd la = lam[nd[a]];
    cd row(0.0, 0.0);
    for (int b = 0; b < 4; ++b) {
      const double wu = ((a & 1) == (b & 1)) ? hu / 3.0 : hu / 6.0;
      const double wv = ((a >> 1) == (b >> 1)) ? hv / 3.0 : hv / 6.0;
      const cd pb = p[nd[b]];
      row.re += wu * wv * pb.re;
      row.im += wu * wv * pb.im;
    }
    s.re += la.re * row.re - la.im * row.im;
    s.im += la.re * row.im + la.im * row.re;
  }
  // G = i krc s ; gb -= conj(G)
  const cd G(-krc * s.im, krc * s.re);
  const cd old = gb[e];
  gb[e] = cd(old.re - G.re, old.im + G.im);
}

__global__ void dir_grad_kernel(const int32_t* __restrict__ nodes, int n_dir, const int32_t* __restrict__ rowptr,
                                const int32_t* __restrict__ col, const cd* __restrict__ val, const cd* __restrict__ lam,
                                const uint8_t* __restrict__ is_dir, cd* __restrict__ gd) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_dir) return;
  const int64_t r = nodes[t];
  cd mu = lam[r];
  for (int q = rowptr[r]; q < rowptr[r + 1]; ++q) {
    const int64_t c = col[q];
    if (is_dir[c]) continue;
    const cd a = val[q], l = lam[c];
    mu.re -= a.re * l.re - a.im * l.im;
    mu.im -= a.re * l.im + a.im * l.re;
  }
  const cd old = gd[t];
  gd[t] = cd(old.re + mu.re, old.im - mu.im);
}

// deterministic sum of w |p|^2 over [n] (one block per chunk, then one block)
__global__ void __launch_bounds__(kBlock) wsum_stage1(const cd* __restrict__ p, const double* __restrict__ w, int64_t n,
                                                      int64_t chunk, double* __restrict__ part) {
  __shared__ double sh[kBlock / 32];
  const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  double v[1] = {0.0};
  for (int64_t i = lo + threadIdx.x; i < hi; i += kBlock) {
    const cd a = p[i];
    v[0] += w[i] * (a.re * a.re + a.im * a.im);
  }
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
}

__global__ void __launch_bounds__(kBlock) wsum_stage2(const double* __restrict__ part, int np, double* __restrict__ out,
                                                      int slot) {
  __shared__ double sh[kBlock / 32];
  double v[1] = {0.0};
  for (int i = threadIdx.x; i < np; i += kBlock) v[0] += part[i];
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) out[slot] = v[0];
}

}  // namespace

helm_status adjoint_grad(helm_ctx* ctx, const double* freqs, int nfreq, const helm_solve_opts& o, const cd* p,
                         const double* w, const cd* gp, cd* grad_beta, cd* grad_pdir, double* J) {
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->n;
  HELM_CUDA(cudaMemsetAsync(grad_beta, 0, ctx->nbf * sizeof(cd), s));
  if (ctx->n_dir > 0) HELM_CUDA(cudaMemsetAsync(grad_pdir, 0, ctx->n_dir * sizeof(cd), s));
  if (J) *J = 0.0;
  if (nfreq == 0) return HELM_OK;
  cd* rhs = nullptr;
  cd* lam = nullptr;
  cd* val = nullptr;
  double* part = nullptr;
  const int np = 256;
  helm_status st = dev_alloc(&rhs, (size_t)nfreq * n);
  if (st == HELM_OK) st = dev_alloc(&lam, (size_t)nfreq * n);
  if (st == HELM_OK) st = dev_alloc(&val, ctx->nnz);
  if (st == HELM_OK) st = dev_alloc(&part, np + nfreq);
  if (st == HELM_OK) {
    seed_kernel<<<1024, 256, 0, s>>>(p, w, gp, rhs, n, (int64_t)nfreq * n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_error(e, "seed");
  }
  std::vector<helm_solve_stats> stats(nfreq);
  if (st == HELM_OK) {
    if (o.solver != HELM_SOLVER_GMRES) {  // the persistent engine: COCG (any mode), BiCGSTAB, TFQMR
      std::vector<BatchSystem> sys(nfreq);
      for (int f = 0; f < nfreq; ++f) sys[f] = BatchSystem{ctx, freqs[f], lam + (size_t)f * n, &stats[f], rhs + (size_t)f * n};
      st = solve_cocg_batch(sys.data(), nfreq, o, s);
    } else {
      for (int f = 0; f < nfreq && st == HELM_OK; ++f) {
        st = assemble_values(ctx, freqs[f], val, nullptr, s);
        if (st == HELM_OK)
          st = solve_gmres_system(ctx, ctx->rowptr, ctx->col, val, freqs[f], rhs + (size_t)f * n, o, lam + (size_t)f * n,
                                  &stats[f]);
      }
    }
    if (st != HELM_OK) st = set_error(st, std::string("adjoint solve: ") + helm_last_error());
  }
  std::vector<double> hJ(nfreq, 0.0);
  for (int f = 0; f < nfreq && st == HELM_OK; ++f) {
    const double k = 2.0 * 3.14159265358979323846 * freqs[f] / ctx->phys.c;
    const cd* pf = p + (size_t)f * n;
    const cd* lf = lam + (size_t)f * n;
    st = assemble_values(ctx, freqs[f], val, nullptr, s, /*eliminate=*/false);
    if (st != HELM_OK) break;
    face_grad_kernel<<<(unsigned)((ctx->nbf + 255) / 256), 256, 0, s>>>(ctx->mesh, k * ctx->phys.rho * ctx->phys.c, lf,
                                                                       pf, ctx->is_dir, grad_beta, ctx->nbf);
    if (ctx->n_dir > 0)
      dir_grad_kernel<<<(ctx->n_dir + 255) / 256, 256, 0, s>>>(ctx->dir_nodes, ctx->n_dir, ctx->rowptr, ctx->col, val,
                                                              lf, ctx->is_dir, grad_pdir);
    if (w) {
      const int64_t chunk = (n + np - 1) / np;
      wsum_stage1<<<np, kBlock, 0, s>>>(pf, w, n, chunk, part);
      wsum_stage2<<<1, kBlock, 0, s>>>(part, np, part + np, f);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_error(e, "adjoint gradient kernels");
  }
  if (st == HELM_OK && w && J) {
    cudaError_t e = cudaMemcpyAsync(hJ.data(), part + np, nfreq * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) st = cuda_error(e, "J copy");
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess && st == HELM_OK) st = cuda_error(e, "adjoint sync");
  if (st == HELM_OK && w && J) {
    double acc = 0.0;
    for (int f = 0; f < nfreq; ++f) acc += hJ[f];
    *J = acc;
  }
  cudaFree(rhs);
  cudaFree(lam);
  cudaFree(val);
  cudaFree(part);
  return st;
}

}  // namespace helm
