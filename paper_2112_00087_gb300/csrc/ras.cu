// Restricted additive Schwarz (RAS) with exact subdomain solves.
//
// Paper Sec. 4: when one system outgrows a single device memory, overlapping Schwarz domain
// decomposition is used, each subdomain solved locally. Here the subdomains are the blocks of
// a parts[0] x parts[1] x parts[2] partition of the lattice, each extended by `overlap` layers
// (Chebyshev index distance, the 27-point graph distance), with homogeneous Dirichlet
// artificial boundaries (A_s is the principal submatrix). The preconditioner is
//     z = sum_s Rt_s^T A_s^{-1} R_s r,
// Rt_s keeping only the nodes subdomain s owns (restricted prolongation).
//
// GB300 design: one CTA per subdomain. A_s is ordered with its two smallest extents fastest,
// giving a band of half-width bw = e_a e_b + e_a + 1; its complex-symmetric LDL^T factor is
// computed in band storage without pivoting (right-looking, one column per step). Two copies
// of the factor are kept -- by columns for the forward sweep and by rows for the backward
// sweep -- so both triangular sweeps are axpy-form, reading one contiguous band row per step
// while the subdomain vector stays in shared memory.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "kernels.cuh"
#include "ras.cuh"

namespace helm {

struct RasSub {
  int i0, j0, l0;        // extended box origin
  int e[3];              // extended extents (x, y, z)
  int o0[3], o1[3];      // owned box [o0, o1) in lattice indices
  int perm[3];           // local axis order: perm[0] fastest
  int ns, bw;            // local size, band half-width
  int64_t off;           // offset of this subdomain's band (elements of cd)
};

struct RasPrecond {
  int nsub;
  int max_ns, max_bw;
  int Nx, Ny;
  RasSub* d_sub;
  cd* colband;   // [sum ns*(bw+1)]  colband[k][d] = L(k+d, k), d=0 holds D_k
  cd* rowband;   // [sum ns*(bw+1)]  rowband[i][d] = L(i, i-d)
  int* d_status;
  int threads;
  size_t smem;
};

namespace {

__device__ __forceinline__ void local_to_lattice(const RasSub& S, int k, int& i, int& j, int& l) {
  int u[3];
  const int ea = S.e[S.perm[0]], eb = S.e[S.perm[1]];
  u[S.perm[0]] = k % ea;
  u[S.perm[1]] = (k / ea) % eb;
  u[S.perm[2]] = k / (ea * eb);
  i = S.i0 + u[0];
  j = S.j0 + u[1];
  l = S.l0 + u[2];
}

__device__ __forceinline__ int lattice_to_local(const RasSub& S, int i, int j, int l) {
  int u[3] = {i - S.i0, j - S.j0, l - S.l0};
  if (u[0] < 0 || u[0] >= S.e[0] || u[1] < 0 || u[1] >= S.e[1] || u[2] < 0 || u[2] >= S.e[2]) return -1;
  const int ea = S.e[S.perm[0]], eb = S.e[S.perm[1]];
  return u[S.perm[0]] + ea * (u[S.perm[1]] + eb * u[S.perm[2]]);
}

// Extract the lower band (by columns) of A_s: W[k][d] = A(k+d, k) = A(k, k+d) (A symmetric).
__global__ void ras_extract(const RasSub* __restrict__ subs, const int32_t* __restrict__ rowptr,
                            const int32_t* __restrict__ col, const cd* __restrict__ val, cd* __restrict__ W,
                            int Nx, int Ny) {
  const RasSub S = subs[blockIdx.x];
  cd* Ws = W + S.off;
  const int64_t total = (int64_t)S.ns * (S.bw + 1);
  for (int64_t t = threadIdx.x; t < total; t += blockDim.x) Ws[t] = cd(0.0, 0.0);
  __syncthreads();
  for (int k = threadIdx.x; k < S.ns; k += blockDim.x) {
    int i, j, l;
    local_to_lattice(S, k, i, j, l);
    const int64_t g = i + (int64_t)Nx * (j + (int64_t)Ny * l);
    for (int q = rowptr[g]; q < rowptr[g + 1]; ++q) {
      const int64_t c = col[q];
      const int ci = (int)(c % Nx), cj = (int)((c / Nx) % Ny), cl = (int)(c / ((int64_t)Nx * Ny));
      const int kc = lattice_to_local(S, ci, cj, cl);
      if (kc < k) continue;  // outside the box (-1) or strictly upper part by columns
      const int d = kc - k;
      if (d <= S.bw) Ws[(int64_t)k * (S.bw + 1) + d] = val[q];
    }
  }
}

// Optimized-Schwarz interface terms: c * (face mass of each face of the extended box that lies
// inside the lattice), c = rb.lo on the box's low faces and rb.hi on its high faces (a plane that
// is both, in a box one layer thick, takes rb.lo), divided by the spacing normal to the face when
// rb.per_h; added to the lower band by columns, Dirichlet rows and columns excluded.
// On a face plane with in-plane axes u, v the Q1 face mass is M1_u (x) M1_v, M1 the 1D linear
// mass over the face's extent: diagonal h/3 per adjacent interval, neighbours h/6. Thread k owns
// column k of the band, so no two threads write the same entry.
__device__ __forceinline__ double mass1d(int c, int dc, int lo, int hi, double h) {
  if (dc == 0) return (h / 3.0) * ((c > lo ? 1 : 0) + (c < hi - 1 ? 1 : 0));
  const int c2 = c + dc;
  return (c2 >= lo && c2 < hi) ? h / 6.0 : 0.0;
}

__global__ void ras_robin(const RasSub* __restrict__ subs, const uint8_t* __restrict__ is_dir, cd* __restrict__ W,
                          int Nx, int Ny, int Nz, double hx, double hy, double hz, RasRobin rb) {
  const RasSub S = subs[blockIdx.x];
  cd* Ws = W + S.off;
  const int N[3] = {Nx, Ny, Nz};
  const int lo[3] = {S.i0, S.j0, S.l0};
  const double h[3] = {hx, hy, hz};
  for (int k = threadIdx.x; k < S.ns; k += blockDim.x) {
    int p[3];
    local_to_lattice(S, k, p[0], p[1], p[2]);
    if (is_dir[p[0] + (int64_t)Nx * (p[1] + (int64_t)Ny * p[2])]) continue;
    for (int a = 0; a < 3; ++a) {
      const int hi_a = lo[a] + S.e[a];
      const bool on_lo = p[a] == lo[a] && lo[a] > 0;
      const bool on_hi = p[a] == hi_a - 1 && hi_a < N[a];
      if (!on_lo && !on_hi) continue;  // (a one-layer box counts its single plane once)
      cd robin = on_lo ? rb.lo : rb.hi;
      if (rb.per_h) robin = cd(robin.re / h[a], robin.im / h[a]);
      const int u = a == 0 ? 1 : 0, v = a == 2 ? 1 : 2;
      for (int du = -1; du <= 1; ++du)
        for (int dv = -1; dv <= 1; ++dv) {
          const double m = mass1d(p[u], du, lo[u], lo[u] + S.e[u], h[u]) * mass1d(p[v], dv, lo[v], lo[v] + S.e[v], h[v]);
          if (m == 0.0) continue;
          int q[3] = {p[0], p[1], p[2]};
          q[u] += du;
          q[v] += dv;
          if (is_dir[q[0] + (int64_t)Nx * (q[1] + (int64_t)Ny * q[2])]) continue;
          const int kc = lattice_to_local(S, q[0], q[1], q[2]);
          if (kc < k) continue;  // the upper part of column k is the transpose, not stored
          const int d = kc - k;
          cd& w = Ws[(int64_t)k * (S.bw + 1) + d];
          w = cd(w.re + m * robin.re, w.im + m * robin.im);
        }
    }
  }
}

// Right-looking band LDL^T, one CTA per subdomain. After column k: W[k][0] = D_k,
// W[k][d] = L(k+d, k).
__global__ void ras_factor(const RasSub* __restrict__ subs, cd* __restrict__ W, int* __restrict__ status) {
  const RasSub S = subs[blockIdx.x];
  cd* Ws = W + S.off;
  const int bw = S.bw, ld = bw + 1, ns = S.ns;
  __shared__ double s_max;
  __shared__ cd s_a[1024];  // W[k][d] before scaling (= l_d D_k)
  __shared__ cd s_l[1024];  // l_d = W[k][d] / D_k
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int k = 0; k < ns; ++k) {
      const cd a = Ws[(int64_t)k * ld];
      mx = fmax(mx, sqrt(a.re * a.re + a.im * a.im));
    }
    s_max = mx;
  }
  __syncthreads();
  const double thresh = 1e-12 * s_max;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int k = 0; k < ns; ++k) {
    const cd dk = Ws[(int64_t)k * ld];
    const int nd = min(bw, ns - 1 - k);
    if (threadIdx.x == 0 && !(sqrt(dk.re * dk.re + dk.im * dk.im) > thresh)) atomicOr(status, 1);
    for (int d = 1 + threadIdx.x; d <= nd; d += blockDim.x) {
      const cd a = Ws[(int64_t)k * ld + d];
      const cd l = cdiv(a, dk);
      s_a[d] = a;
      s_l[d] = l;
      Ws[(int64_t)k * ld + d] = l;
    }
    __syncthreads();
    // A(k+di, k+dj) -= l_di D_k l_dj = l_di * W_k,dj for 1 <= dj <= di <= nd, stored at
    // column k+dj, offset di-dj: one warp per target column, lanes along the column
    for (int dj = 1 + warp; dj <= nd; dj += nwarps) {
      const cd aj = s_a[dj];
      cd* colp = Ws + (int64_t)(k + dj) * ld - dj;
      for (int di = dj + lane; di <= nd; di += 32) {
        const cd li = s_l[di];
        cd t = colp[di];
        t.re -= li.re * aj.re - li.im * aj.im;
        t.im -= li.re * aj.im + li.im * aj.re;
        colp[di] = t;
      }
    }
    __syncthreads();
  }
}

// rowband[i][d] = L(i, i-d) = colband[i-d][d]
__global__ void ras_transpose(const RasSub* __restrict__ subs, const cd* __restrict__ C, cd* __restrict__ R) {
  const RasSub S = subs[blockIdx.x];
  const int ld = S.bw + 1;
  const int64_t total = (int64_t)S.ns * ld;
  for (int64_t t = threadIdx.x; t < total; t += blockDim.x) {
    const int i = (int)(t / ld), d = (int)(t % ld);
    R[S.off + t] = (i - d >= 0) ? C[S.off + (int64_t)(i - d) * ld + d] : cd(0.0, 0.0);
  }
}

// z = sum_s Rt_s^T A_s^-1 R_s r: gather, forward (L), diagonal (D), backward (L^T), scatter owned.
__global__ void ras_apply_kernel(const RasSub* __restrict__ subs, const cd* __restrict__ C,
                                 const cd* __restrict__ R, const cd* in, cd* out, int Nx, int Ny,
                                 const int* skip_a, const int* skip_b) {
  if ((skip_a && *((volatile const int*)skip_a)) || (skip_b && *((volatile const int*)skip_b))) return;
  extern __shared__ cd y[];
  const RasSub S = subs[blockIdx.x];
  const int bw = S.bw, ld = bw + 1, ns = S.ns;
  const cd* Cs = C + S.off;
  const cd* Rs = R + S.off;
  for (int k = threadIdx.x; k < ns; k += blockDim.x) {
    int i, j, l;
    local_to_lattice(S, k, i, j, l);
    y[k] = in[i + (int64_t)Nx * (j + (int64_t)Ny * l)];
  }
  __syncthreads();
  const int d = threadIdx.x + 1;  // this thread's band offset
  // forward: y_{k+d} -= L(k+d,k) y_k
  cd lnext = (d <= bw && d < ns) ? Cs[d] : cd(0.0, 0.0);
  for (int k = 0; k < ns; ++k) {
    const cd lk = lnext;
    if (k + 1 < ns && d <= bw && k + 1 + d < ns) lnext = Cs[(int64_t)(k + 1) * ld + d];
    const cd yk = y[k];
    if (d <= bw && k + d < ns) {
      cd t = y[k + d];
      t.re -= lk.re * yk.re - lk.im * yk.im;
      t.im -= lk.re * yk.im + lk.im * yk.re;
      y[k + d] = t;
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < ns; k += blockDim.x) y[k] = cdiv(y[k], Cs[(int64_t)k * ld]);
  __syncthreads();
  // backward: x_{k-d} -= L(k, k-d) x_k
  lnext = (d <= bw && ns - 1 - d >= 0) ? Rs[(int64_t)(ns - 1) * ld + d] : cd(0.0, 0.0);
  for (int k = ns - 1; k >= 0; --k) {
    const cd lk = lnext;
    if (k - 1 >= 0 && d <= bw && k - 1 - d >= 0) lnext = Rs[(int64_t)(k - 1) * ld + d];
    const cd xk = y[k];
    if (d <= bw && k - d >= 0) {
      cd t = y[k - d];
      t.re -= lk.re * xk.re - lk.im * xk.im;
      t.im -= lk.re * xk.im + lk.im * xk.re;
      y[k - d] = t;
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < ns; k += blockDim.x) {
    int i, j, l;
    local_to_lattice(S, k, i, j, l);
    if (i >= S.o0[0] && i < S.o1[0] && j >= S.o0[1] && j < S.o1[1] && l >= S.o0[2] && l < S.o1[2])
      out[i + (int64_t)Nx * (j + (int64_t)Ny * l)] = y[k];
  }
}

// Owned ranges along one axis: point t belongs to part floor(t * parts / npts).
std::vector<std::pair<int, int>> block_ranges(int npts, int parts) {
  std::vector<std::pair<int, int>> r(parts, {npts, 0});
  for (int t = 0; t < npts; ++t) {
    const int p = (int)(((int64_t)t * parts) / npts);
    r[p].first = std::min(r[p].first, t);
    r[p].second = std::max(r[p].second, t + 1);
  }
  return r;
}

}  // namespace

helm_status ras_create(const helm_ctx* ctx, const int32_t* rowptr, const int32_t* col, const cd* val,
                       const int32_t parts[3], int overlap, const RasRobin& robin, RasPrecond** out,
                       cudaStream_t s) {
  *out = nullptr;
  const int N[3] = {ctx->mesh.nx + 1, ctx->mesh.ny + 1, ctx->mesh.nz + 1};
  for (int a = 0; a < 3; ++a)
    if (parts[a] > N[a]) return set_error(HELM_ERR_ARG, "RAS: more parts than lattice points along an axis");
  std::vector<std::pair<int, int>> R[3];
  for (int a = 0; a < 3; ++a) R[a] = block_ranges(N[a], parts[a]);
  std::vector<RasSub> subs;
  int64_t off = 0;
  int max_ns = 0, max_bw = 0;
  for (int bl = 0; bl < parts[2]; ++bl)
    for (int bj = 0; bj < parts[1]; ++bj)
      for (int bi = 0; bi < parts[0]; ++bi) {
        RasSub S;
        memset(&S, 0, sizeof(S));
        const std::pair<int, int> own[3] = {R[0][bi], R[1][bj], R[2][bl]};
        int lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
          S.o0[a] = own[a].first;
          S.o1[a] = own[a].second;
          lo[a] = std::max(0, own[a].first - overlap);
          hi[a] = std::min(N[a], own[a].second + overlap);
          S.e[a] = hi[a] - lo[a];
        }
        S.i0 = lo[0];
        S.j0 = lo[1];
        S.l0 = lo[2];
        int p[3] = {0, 1, 2};
        std::stable_sort(p, p + 3, [&](int x, int y) { return S.e[x] < S.e[y]; });
        for (int a = 0; a < 3; ++a) S.perm[a] = p[a];
        S.ns = S.e[0] * S.e[1] * S.e[2];
        S.bw = S.e[p[0]] * S.e[p[1]] + S.e[p[0]] + 1;
        S.bw = std::min(S.bw, S.ns - 1);
        S.off = off;
        off += (int64_t)S.ns * (S.bw + 1);
        max_ns = std::max(max_ns, S.ns);
        max_bw = std::max(max_bw, S.bw);
        subs.push_back(S);
      }
  const size_t smem = (size_t)max_ns * sizeof(cd);
  if (max_bw >= 1024) return set_error(HELM_ERR_ARG, "RAS: subdomain band too wide (use more parts)");
  if (smem > 220 * 1024) return set_error(HELM_ERR_ARG, "RAS: subdomain too large for shared memory (use more parts)");
  RasPrecond* P = new RasPrecond;
  memset(P, 0, sizeof(*P));
  P->nsub = (int)subs.size();
  P->max_ns = max_ns;
  P->max_bw = max_bw;
  P->Nx = N[0];
  P->Ny = N[1];
  P->threads = std::max(64, ((max_bw + 31) / 32) * 32);
  P->smem = smem;
  helm_status st = dev_alloc(&P->d_sub, subs.size());
  if (st == HELM_OK) st = dev_alloc(&P->colband, (size_t)off);
  if (st == HELM_OK) st = dev_alloc(&P->rowband, (size_t)off);
  if (st == HELM_OK) st = dev_alloc(&P->d_status, 1);
  if (st != HELM_OK) {
    ras_destroy(P);
    return st;
  }
  cudaError_t e = cudaMemcpyAsync(P->d_sub, subs.data(), subs.size() * sizeof(RasSub), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->d_status, 0, sizeof(int), s);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(ras_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) {
    ras_extract<<<P->nsub, 256, 0, s>>>(P->d_sub, rowptr, col, val, P->colband, P->Nx, P->Ny);
    if (robin.lo.re != 0.0 || robin.lo.im != 0.0 || robin.hi.re != 0.0 || robin.hi.im != 0.0)
      ras_robin<<<P->nsub, 256, 0, s>>>(P->d_sub, ctx->is_dir, P->colband, N[0], N[1], N[2],
                                        ctx->mesh.Lx / ctx->mesh.nx, ctx->mesh.Ly / ctx->mesh.ny,
                                        ctx->mesh.Lz / ctx->mesh.nz, robin);
    ras_factor<<<P->nsub, 512, 0, s>>>(P->d_sub, P->colband, P->d_status);
    ras_transpose<<<P->nsub, 256, 0, s>>>(P->d_sub, P->colband, P->rowband);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    ras_destroy(P);
    return cuda_error(e, "RAS setup");
  }
  *out = P;
  return HELM_OK;
}

helm_status ras_apply(RasPrecond* P, const cd* in, cd* out, const int* skip_a, const int* skip_b, cudaStream_t s) {
  ras_apply_kernel<<<P->nsub, P->threads, P->smem, s>>>(P->d_sub, P->colband, P->rowband, in, out, P->Nx, P->Ny,
                                                        skip_a, skip_b);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

helm_status ras_status(RasPrecond* P) {
  int h = 0;
  HELM_CUDA(cudaMemcpy(&h, P->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) return set_error(HELM_PIVOT, "RAS: a subdomain factorisation met a pivot below 1e-12 max|diag|");
  return HELM_OK;
}

void ras_destroy(RasPrecond* P) {
  if (!P) return;
  cudaDeviceSynchronize();
  cudaFree(P->d_sub);
  cudaFree(P->colband);
  cudaFree(P->rowband);
  cudaFree(P->d_status);
  delete P;
}

}  // namespace helm
