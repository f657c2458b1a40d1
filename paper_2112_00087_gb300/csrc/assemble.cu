// Assembly of the eliminated Q1 Helmholtz system on the box lattice (paper Sec. 3.2,
// Helmholtz eq.; Sec. 4 CSR storage).
//
// On a lattice of equal bricks the assembled Q1 stiffness and mass are Kronecker products of
// the assembled 1D linear-element matrices:
//   M = Mx (x) My (x) Mz,   K = Kx (x) My (x) Mz + Mx (x) Ky (x) Mz + Mx (x) My (x) Kz,
// with the 1D entries  K(i,i) = cnt/h, K(i,i+-1) = -1/h, M(i,i) = cnt h/3, M(i,i+-1) = h/6,
// cnt = number of cells touching node i (1 or 2). Every row is therefore computed in closed
// form by one thread, race-free and without atomics. The wall term adds, for each boundary
// quad e touching both nodes of an entry, beta_e times the quad-mass entry (h_u/3 or h_u/6)
// (h_v/3 or h_v/6). An entry and its transpose are produced by the same operations on the same
// operands, so the assembled matrix is bitwise symmetric.
#include "common.cuh"

namespace helm {
namespace {

struct Lattice {
  int nx, ny, nz;     // cells per axis
  int Nx, Ny, Nz;     // nodes per axis
  double hx, hy, hz;
};

__host__ __device__ inline Lattice make_lattice(const helm_mesh_desc& m) {
  Lattice L;
  L.nx = m.nx; L.ny = m.ny; L.nz = m.nz;
  L.Nx = m.nx + 1; L.Ny = m.ny + 1; L.Nz = m.nz + 1;
  L.hx = m.Lx / m.nx; L.hy = m.Ly / m.ny; L.hz = m.Lz / m.nz;
  return L;
}

// Row-length factor along one axis (neighbours inside the lattice, 2 or 3) and its prefix sum.
__device__ inline int64_t len1(int i, int N) { return 3 - (i == 0) - (i == N - 1); }
__device__ inline int64_t pre1(int i, int N) { return 3 * (int64_t)i - (i > 0) - (i == N); }

__global__ void pattern_kernel(Lattice L, int32_t* __restrict__ rowptr, int32_t* __restrict__ col,
                               int64_t n) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r > n) return;
  const int64_t SX = pre1(L.Nx, L.Nx), SY = pre1(L.Ny, L.Ny);
  if (r == n) {
    rowptr[n] = (int32_t)(SX * SY * pre1(L.Nz, L.Nz));
    return;
  }
  int i = (int)(r % L.Nx);
  int j = (int)((r / L.Nx) % L.Ny);
  int l = (int)(r / ((int64_t)L.Nx * L.Ny));
  int64_t start = pre1(l, L.Nz) * SY * SX + len1(l, L.Nz) * pre1(j, L.Ny) * SX +
                  len1(l, L.Nz) * len1(j, L.Ny) * pre1(i, L.Nx);
  rowptr[r] = (int32_t)start;
  int64_t k = start;
  for (int dl = -1; dl <= 1; ++dl) {
    if (l + dl < 0 || l + dl >= L.Nz) continue;
    for (int dj = -1; dj <= 1; ++dj) {
      if (j + dj < 0 || j + dj >= L.Ny) continue;
      for (int di = -1; di <= 1; ++di) {
        if (i + di < 0 || i + di >= L.Nx) continue;
        col[k++] = (int32_t)(r + di + (int64_t)L.Nx * (dj + (int64_t)L.Ny * dl));
      }
    }
  }
}

// 1D assembled stiffness / mass entries at node i, offset d in {-1,0,1}.
__device__ inline void entries1(int i, int d, int ncell, double h, double& k, double& m) {
  if (d == 0) {
    double cnt = (double)((i > 0) + (i < ncell));
    k = cnt / h;
    m = cnt * h / 3.0;
  } else {
    k = -1.0 / h;
    m = h / 6.0;
  }
}

// Sum over boundary quads of one side touching both in-plane nodes a and a+da (axis u) and
// b and b+db (axis v): beta_q * (quad-mass entry). Quads visited v-outer, u-inner ascending.
__device__ inline void side_term(const cd* __restrict__ beta, int64_t base, int a, int da, int nu,
                                 double hu, int b, int db, int nv, double hv, cd& acc) {
  const double w = ((da == 0) ? hu / 3.0 : hu / 6.0) * ((db == 0) ? hv / 3.0 : hv / 6.0);
  int u0 = max(max(a, a + da) - 1, 0), u1 = min(min(a, a + da), nu - 1);
  int v0 = max(max(b, b + db) - 1, 0), v1 = min(min(b, b + db), nv - 1);
  for (int v = v0; v <= v1; ++v)
    for (int u = u0; u <= u1; ++u) {
      cd be = beta[base + u + (int64_t)nu * v];
      acc.re += be.re * w;
      acc.im += be.im * w;
    }
}

// DIA = false: CSR values at rowptr[r]..; DIA = true: slot-major split layout, real parts at
// vre[k * n + r] and imaginary parts at vim[k * n + r] (vre = (double*)val, vim = vre + 27 n),
// k = (di+1) + 3 (dj+1) + 9 (dl+1), zeros for neighbours outside the lattice.
template <bool DIA>
__global__ void values_kernel(Lattice L, double k2, double krc, const int32_t* __restrict__ rowptr,
                              const cd* __restrict__ beta, const uint8_t* __restrict__ is_dir,
                              const cd* __restrict__ pdir, cd* __restrict__ val, cd* __restrict__ b,
                              uint8_t* __restrict__ cflag, int64_t n) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  int i = (int)(r % L.Nx);
  int j = (int)((r / L.Nx) % L.Ny);
  int l = (int)(r / ((int64_t)L.Nx * L.Ny));
  const int64_t o_xm = 0, o_xp = (int64_t)L.ny * L.nz, o_ym = 2 * o_xp,
                o_yp = o_ym + (int64_t)L.nx * L.nz, o_zm = o_yp + (int64_t)L.nx * L.nz,
                o_zp = o_zm + (int64_t)L.nx * L.ny;
  const bool rowD = is_dir != nullptr && is_dir[r] != 0;
  cd bsum(0.0, 0.0);
  bool row_complex = false;
  int64_t k = DIA ? 0 : rowptr[r];
  double* vre = reinterpret_cast<double*>(val);
  double* vim = vre + 27 * n;
  if (DIA)
    for (int s = 0; s < 27; ++s) {
      vre[(int64_t)s * n + r] = 0.0;
      vim[(int64_t)s * n + r] = 0.0;
    }
  for (int dl = -1; dl <= 1; ++dl) {
    if (l + dl < 0 || l + dl >= L.Nz) continue;
    double kz, mz;
    entries1(l, dl, L.nz, L.hz, kz, mz);
    for (int dj = -1; dj <= 1; ++dj) {
      if (j + dj < 0 || j + dj >= L.Ny) continue;
      double ky, my;
      entries1(j, dj, L.ny, L.hy, ky, my);
      for (int di = -1; di <= 1; ++di) {
        if (i + di < 0 || i + di >= L.Nx) continue;
        if (DIA) k = (int64_t)((di + 1) + 3 * (dj + 1) + 9 * (dl + 1)) * n + r;
        double kx, mx;
        entries1(i, di, L.nx, L.hx, kx, mx);
        const int64_t c = r + di + (int64_t)L.Nx * (dj + (int64_t)L.Ny * dl);
        const double K = kx * my * mz + mx * ky * mz + mx * my * kz;
        const double M = mx * my * mz;
        cd B(0.0, 0.0);
        if (beta != nullptr) {
          if (di == 0 && i == 0) side_term(beta, o_xm, j, dj, L.ny, L.hy, l, dl, L.nz, L.hz, B);
          if (di == 0 && i == L.nx) side_term(beta, o_xp, j, dj, L.ny, L.hy, l, dl, L.nz, L.hz, B);
          if (dj == 0 && j == 0) side_term(beta, o_ym, i, di, L.nx, L.hx, l, dl, L.nz, L.hz, B);
          if (dj == 0 && j == L.ny) side_term(beta, o_yp, i, di, L.nx, L.hx, l, dl, L.nz, L.hz, B);
          if (dl == 0 && l == 0) side_term(beta, o_zm, i, di, L.nx, L.hx, j, dj, L.ny, L.hy, B);
          if (dl == 0 && l == L.nz) side_term(beta, o_zp, i, di, L.nx, L.hx, j, dj, L.ny, L.hy, B);
        }
        // A = K - k^2 M + i (k rho c) B
        cd a(K - k2 * M - krc * B.im, krc * B.re);
        if (rowD) {
          a = cd(c == r ? 1.0 : 0.0, 0.0);
        } else if (is_dir != nullptr && is_dir[c]) {
          // lifting b_F -= A_FD p_D (ascending columns), then eliminate the column
          cd pc = pdir[c];
          bsum.re += a.re * pc.re - a.im * pc.im;
          bsum.im += a.re * pc.im + a.im * pc.re;
          a = cd(0.0, 0.0);
        }
        if (DIA) {
          vre[k] = a.re;
          vim[k] = a.im;
        } else {
          val[k] = a;
          ++k;
        }
        row_complex |= (a.im != 0.0);
      }
    }
  }
  if (b != nullptr) b[r] = rowD ? pdir[r] : cd(-bsum.re, -bsum.im);
  if (cflag != nullptr) cflag[r] = row_complex ? 1 : 0;
}

__global__ void cast_kernel(const cd* __restrict__ v, cf* __restrict__ v32, int64_t nnz) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; t < nnz; t += stride) {
    cd a = v[t];
    v32[t] = cf(__double2float_rn(a.re), __double2float_rn(a.im));
  }
}

}  // namespace

helm_status build_pattern(helm_ctx* ctx) {
  Lattice L = make_lattice(ctx->mesh);
  const int T = 256;
  int64_t blocks = (ctx->n + 1 + T - 1) / T;
  pattern_kernel<<<(unsigned)blocks, T, 0, ctx->stream>>>(L, ctx->rowptr, ctx->col, ctx->n);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

helm_status assemble_values(const helm_ctx* ctx, double freq, cd* val, cd* b, cudaStream_t s, bool eliminate,
                            bool dia, uint8_t* cflag) {
  Lattice L = make_lattice(ctx->mesh);
  const double k = 2.0 * 3.14159265358979323846 * freq / ctx->phys.c;
  const int T = 128;
  int64_t blocks = (ctx->n + T - 1) / T;
  (dia ? values_kernel<true> : values_kernel<false>)<<<(unsigned)blocks, T, 0, s>>>(L, k * k, k * ctx->phys.rho * ctx->phys.c, ctx->rowptr,
                                               ctx->beta, eliminate ? ctx->is_dir : nullptr,
                                               ctx->p_dir_full, val, eliminate ? b : nullptr, cflag, ctx->n);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

// Frequency-independent parts of the eliminated matrix, slot-major like the DIA-27 values:
// comp = [K | M | Re B | Im B], each 27 n doubles, with A(k) = K - k^2 M + i k rho c B on free
// rows and columns; a Dirichlet row holds K = 1 on the diagonal and zeros elsewhere, a Dirichlet
// column zeros (the lifting term, which depends on k, is not part of the operator). bflag[r] = 1
// for rows with a non-zero B entry.
__global__ void components_kernel(Lattice L, const cd* __restrict__ beta, const uint8_t* __restrict__ is_dir,
                                  double* __restrict__ comp, uint8_t* __restrict__ bflag, int64_t n) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  int i = (int)(r % L.Nx);
  int j = (int)((r / L.Nx) % L.Ny);
  int l = (int)(r / ((int64_t)L.Nx * L.Ny));
  const int64_t o_xm = 0, o_xp = (int64_t)L.ny * L.nz, o_ym = 2 * o_xp,
                o_yp = o_ym + (int64_t)L.nx * L.nz, o_zm = o_yp + (int64_t)L.nx * L.nz,
                o_zp = o_zm + (int64_t)L.nx * L.ny;
  const bool rowD = is_dir != nullptr && is_dir[r] != 0;
  double* Kc = comp;
  double* Mc = comp + 27 * n;
  double* Br = comp + 54 * n;
  double* Bi = comp + 81 * n;
  for (int s = 0; s < 27; ++s) {
    Kc[(int64_t)s * n + r] = 0.0;
    Mc[(int64_t)s * n + r] = 0.0;
    Br[(int64_t)s * n + r] = 0.0;
    Bi[(int64_t)s * n + r] = 0.0;
  }
  bool has_b = false;
  for (int dl = -1; dl <= 1; ++dl) {
    if (l + dl < 0 || l + dl >= L.Nz) continue;
    double kz, mz;
    entries1(l, dl, L.nz, L.hz, kz, mz);
    for (int dj = -1; dj <= 1; ++dj) {
      if (j + dj < 0 || j + dj >= L.Ny) continue;
      double ky, my;
      entries1(j, dj, L.ny, L.hy, ky, my);
      for (int di = -1; di <= 1; ++di) {
        if (i + di < 0 || i + di >= L.Nx) continue;
        const int64_t e = (int64_t)((di + 1) + 3 * (dj + 1) + 9 * (dl + 1)) * n + r;
        double kx, mx;
        entries1(i, di, L.nx, L.hx, kx, mx);
        const int64_t c = r + di + (int64_t)L.Nx * (dj + (int64_t)L.Ny * dl);
        if (rowD) {
          Kc[e] = c == r ? 1.0 : 0.0;
          continue;
        }
        if (is_dir != nullptr && is_dir[c]) continue;
        Kc[e] = kx * my * mz + mx * ky * mz + mx * my * kz;
        Mc[e] = mx * my * mz;
        cd B(0.0, 0.0);
        if (beta != nullptr) {
          if (di == 0 && i == 0) side_term(beta, o_xm, j, dj, L.ny, L.hy, l, dl, L.nz, L.hz, B);
          if (di == 0 && i == L.nx) side_term(beta, o_xp, j, dj, L.ny, L.hy, l, dl, L.nz, L.hz, B);
          if (dj == 0 && j == 0) side_term(beta, o_ym, i, di, L.nx, L.hx, l, dl, L.nz, L.hz, B);
          if (dj == 0 && j == L.ny) side_term(beta, o_yp, i, di, L.nx, L.hx, l, dl, L.nz, L.hz, B);
          if (dl == 0 && l == 0) side_term(beta, o_zm, i, di, L.nx, L.hx, j, dj, L.ny, L.hy, B);
          if (dl == 0 && l == L.nz) side_term(beta, o_zp, i, di, L.nx, L.hx, j, dj, L.ny, L.hy, B);
        }
        Br[e] = B.re;
        Bi[e] = B.im;
        has_b |= (B.re != 0.0 || B.im != 0.0);
      }
    }
  }
  bflag[r] = has_b ? 1 : 0;
}

__global__ void cast_real_kernel(const double* __restrict__ v, float* __restrict__ v32, int64_t m) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; t < m; t += stride) v32[t] = __double2float_rn(v[t]);
}

// Double-word copy of m doubles: out[t] = (hi, lo), hi = fl32(v), lo = fl32(v - hi).
// Double-word copy of `nslots` FP64 slot arrays of n values each (slot stride n) into (hi, lo)
// float pairs with slot stride ns >= n; the ns - n padding entries of every slot are zero.
__global__ void split_kernel(const double* __restrict__ v, float2* __restrict__ out, int64_t n, int64_t ns,
                             int64_t m) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; t < m; t += stride) {  // m = nslots * ns
    const int64_t k = t / ns, row = t - k * ns;
    float2 o = make_float2(0.f, 0.f);
    if (row < n) {
      const double a = v[k * n + row];
      const float hi = __double2float_rn(a);
      o = make_float2(hi, __double2float_rn(a - (double)hi));
    }
    out[t] = o;
  }
}

helm_status assemble_components(const helm_ctx* ctx, double* comp, float* comp32, uint8_t* bflag, cudaStream_t s) {
  Lattice L = make_lattice(ctx->mesh);
  const unsigned blocks = (unsigned)((ctx->n + 127) / 128);
  components_kernel<<<blocks, 128, 0, s>>>(L, ctx->beta, ctx->is_dir, comp, bflag, ctx->n);
  if (comp32) {
    const int64_t m = 108 * ctx->n;
    cast_real_kernel<<<(unsigned)std::min<int64_t>((m + 255) / 256, 152 * 16), 256, 0, s>>>(comp, comp32, m);
  }
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

helm_status split_values(const double* val, float2* out, int64_t n, int64_t ns, int nslots, cudaStream_t s) {
  const int64_t m = (int64_t)nslots * ns;
  if (m == 0) return HELM_OK;
  int blocks = (int)std::min<int64_t>((m + 255) / 256, 152 * 16);
  split_kernel<<<blocks, 256, 0, s>>>(val, out, n, ns, m);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

helm_status cast_values(const cd* val, cf* val32, int64_t nnz, cudaStream_t s) {
  if (nnz == 0) return HELM_OK;
  int blocks = (int)std::min<int64_t>((nnz + 255) / 256, 152 * 16);
  cast_kernel<<<blocks, 256, 0, s>>>(val, val32, nnz);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

}  // namespace helm
