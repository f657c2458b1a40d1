// Host side of the persistent batched Krylov engine: tiles the systems of a batch, allocates
// every per-system buffer from one arena, assembles (and scales / converts) each system's
// matrix, launches the solver's persistent kernel cooperatively with CUDA events around it, and
// returns per-system statistics. The kernels live in krylov_cocg.cu and krylov_bicg.cu.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "krylov_engine.cuh"

namespace helm {
namespace {
using namespace eng;

// Default minimum tile, applied while the batch still gives every block about 8 tiles of that
// size (a small batch keeps 512-row tiles so that all blocks have work). Measured on the
// 256-frequency sweep (double-word mode): 512 / 2,048 / 4,096 / 8,192 rows gave 25.8 / 28.3 /
// 31.8 / 31.5 freqs/s -- the per-tile reduction and arrival cost of a phase outweighs load
// balance below a few thousand rows.
constexpr int64_t kTileRowsMin = 4096;

// Simple bump allocator over one device allocation (256-byte aligned pieces).
struct Arena {
  char* base = nullptr;
  size_t off = 0, cap = 0;
  template <typename T> T* take(size_t count) {
    size_t bytes = ((count * sizeof(T)) + 255) & ~(size_t)255;
    T* p = reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};
inline size_t rnd(size_t bytes) { return (bytes + 255) & ~(size_t)255; }

}  // namespace

helm_status solve_cocg_batch(const BatchSystem* sys, int nsys, const helm_solve_opts& o, cudaStream_t s) {
  if (nsys <= 0) return HELM_OK;
  const int prec = o.mixed;  // 0 FP64, 1 complex64 inner, 2 double-word inner
  const bool mixed = prec != 0;
  int dev = 0, nsm = 1;
  HELM_CUDA(cudaGetDevice(&dev));
  HELM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  int coop = 0;
  HELM_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return set_error(HELM_ERR_CUDA, "device does not support cooperative launch");
  // Register budgets: 1 block per SM (255 registers, deep per-thread ILP) up to 4 (64
  // registers, more resident warps); HELM_PERSIST_BLOCKS_PER_SM selects one (tuning knob).
  const char* env = getenv("HELM_PERSIST_BLOCKS_PER_SM");
  const int want = env ? std::max(1, std::min(atoi(env), 4)) : HELM_DEFAULT_BLOCKS_PER_SM;
  const bool bicg = o.solver == HELM_SOLVER_BICGSTAB;
  const bool tfq = o.solver == HELM_SOLVER_TFQMR;
  const bool jac = o.precond == HELM_PRECOND_JACOBI && (bicg || tfq);   // right Jacobi A D^-1
  const bool sjac = o.precond == HELM_PRECOND_JACOBI && !(bicg || tfq);  // symmetric S A S (COCG)
  void (*kern)(KParams) = nullptr;
  if (bicg) kern = reinterpret_cast<void (*)(KParams)>(bicg_kernel(want));
  else if (tfq) kern = reinterpret_cast<void (*)(KParams)>(tfqmr_kernel(want));
  else kern = reinterpret_cast<void (*)(KParams)>(cocg_kernel(prec, want));
  int per_sm = 0;
  HELM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, 0));
  if (per_sm < 1) return set_error(HELM_ERR_CUDA, "persistent kernel cannot be resident");
  per_sm = std::min(per_sm, want);
  const int nblocks = nsm * per_sm;

  // tiles: about nblocks tiles for a system that fills the GPU, at least kTileRowsMin rows,
  // multiples of 2 * kBlock rows
  std::vector<KTile> tiles;
  std::vector<int> tile0(nsys), ntl(nsys);
  const int64_t TQ = 2 * kBlock;
  // minimum tile (rows): each tile carries a block reduction and an arrival per phase, so small
  // systems are cut into few, larger tiles (tuning knob HELM_TILE_ROWS)
  const char* tenv_rows = getenv("HELM_TILE_ROWS");
  int64_t total_rows = 0;
  for (int k = 0; k < nsys; ++k) total_rows += sys[k].ctx->n;
  const int64_t tile_cap = TQ * std::max<int64_t>(1, total_rows / ((int64_t)nblocks * 8 * TQ));
  const int64_t tile_req = tenv_rows ? atoll(tenv_rows) : std::min<int64_t>(kTileRowsMin, tile_cap);
  const int64_t tile_min = TQ * std::max<int64_t>(1, (tile_req + TQ - 1) / TQ);
  // a system with more than kTileRowsMin rows per block is cut into about HELM_TILES_PER_BLOCK x
  // nblocks tiles (tuning knob, default 2), but not below kTileRowsMin rows: more, shorter tiles
  // let the dynamic scheduler even out tiles of unequal cost (rows next to admittance walls take
  // a second, imaginary pass); measured on one 2,203,161-node lattice: 18 % less time per step
  const char* tenv_tpb = getenv("HELM_TILES_PER_BLOCK");
  const int64_t tpb = tenv_tpb ? std::max<int64_t>(1, std::min<int64_t>(atoll(tenv_tpb), 64)) : 2;
  for (int k = 0; k < nsys; ++k) {
    const int64_t n = sys[k].ctx->n;
    const int64_t one = TQ * std::max<int64_t>(1, (n + TQ * nblocks - 1) / (TQ * nblocks));  // ~1 per block
    const int64_t split = std::max(std::min<int64_t>(one, kTileRowsMin),
                                   TQ * std::max<int64_t>(1, (n + TQ * nblocks * tpb - 1) / (TQ * nblocks * tpb)));
    const int64_t per = std::max(tile_min, split);
    tile0[k] = (int)tiles.size();
    for (int64_t r0 = 0; r0 < n; r0 += per) tiles.push_back(KTile{k, 0, r0, std::min(n, r0 + per)});
    ntl[k] = (int)tiles.size() - tile0[k];
  }
  const int ntiles = (int)tiles.size();

  // one arena for every per-system buffer plus the control data
  size_t bytes = 0;
  for (int k = 0; k < nsys; ++k) {
    const size_t n = sys[k].ctx->n, nnz = 27 * n;  // slot-major 27-point values
    bytes += rnd(nnz * sizeof(cd)) + rnd(n * sizeof(cd)) * 2 + rnd(n);  // val, b, r, row flags
    if (prec == 1) bytes += rnd(nnz * sizeof(cf)) + 4 * rnd(n * sizeof(cf));
    if (prec == 2) bytes += rnd(54 * (n + (n & 1)) * sizeof(float2)) + 4 * rnd(n * sizeof(cw));
    bytes += 2 * rnd(n * sizeof(cd));  // p, q (FP64 COCG, also the fallback of the mixed solver)
    if (!(bicg || tfq)) bytes += rnd(n * sizeof(cd));  // best iterate of FP64 COCG
    if (bicg || tfq) bytes += 3 * rnd(n * sizeof(cd));  // rs, s, t (TFQMR: r0*, w, A u)
    if (tfq) bytes += rnd(n * sizeof(cd));              // TFQMR direction d
    if (jac) bytes += rnd(n * sizeof(cd));              // diag(A)
    if (sjac) bytes += rnd(n * sizeof(cd)) + rnd(n * sizeof(double)) + (mixed ? rnd(n * sizeof(float)) : 0);
  }
  const char* tenv = getenv("HELM_TRACE_STEPS");
  const int trace_steps = tenv ? std::max(0, std::min(atoi(tenv), 100000)) : 0;
  bytes += rnd((size_t)trace_steps * kTraceStride * sizeof(unsigned long long));
  bytes += rnd(nsys * sizeof(KSys)) + rnd(nsys * sizeof(KState)) + rnd(ntiles * sizeof(KTile)) +
           2 * rnd(ntiles * sizeof(int)) + rnd(CTRL_N * sizeof(int)) + rnd(2 * (size_t)ntiles * sizeof(cd)) +
           rnd(sizeof(GridBar));
  Arena A;
  A.cap = bytes;
  helm_status st = dev_alloc(&A.base, bytes);
  if (st != HELM_OK) return st;

  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  for (int q = 0; q < 3; ++q) cudaEventCreate(&ev[q]);
  cudaEventRecord(ev[0], s);
  std::vector<KSys> hs(nsys);
  std::vector<KState> hst(nsys);
  for (int k = 0; k < nsys; ++k) {
    const helm_ctx* c = sys[k].ctx;
    KSys& Y = hs[k];
    memset(&Y, 0, sizeof(Y));
    Y.n = c->n;
    Y.Nx = c->mesh.nx + 1;
    Y.NxNy = Y.Nx * (c->mesh.ny + 1);
    cd* val = A.take<cd>(27 * (size_t)c->n);
    cd* b = A.take<cd>(c->n);
    uint8_t* cflag = A.take<uint8_t>(c->n);
    Y.cflag = cflag;
    Y.val = val;
    Y.b = b;
    Y.x = sys[k].p_out;
    Y.r = A.take<cd>(c->n);
    if (prec == 2) {
      Y.nsw = c->n + (c->n & 1);  // even slot stride: every slot starts 16-byte aligned
      Y.valw = A.take<float2>(54 * (size_t)Y.nsw);
      Y.xw = A.take<cw>(c->n);
      Y.rw = A.take<cw>(c->n);
      Y.pw = A.take<cw>(c->n);
      Y.qw = A.take<cw>(c->n);
    }
    if (prec == 1) {
      cf* v32 = A.take<cf>(27 * (size_t)c->n);
      Y.val32 = v32;
      Y.x32 = A.take<cf>(c->n);
      Y.r32 = A.take<cf>(c->n);
      Y.p32 = A.take<cf>(c->n);
      Y.q32 = A.take<cf>(c->n);
    }
    Y.p = A.take<cd>(c->n);
    Y.q = A.take<cd>(c->n);
    if (!(bicg || tfq)) Y.xb = A.take<cd>(c->n);
    if (bicg || tfq) {
      Y.rs = A.take<cd>(c->n);
      Y.sv = A.take<cd>(c->n);
      Y.tv = A.take<cd>(c->n);
    }
    if (tfq) Y.dv = A.take<cd>(c->n);
    if (jac) Y.djac = A.take<cd>(c->n);
    double* wn = nullptr;
    float* wn32 = nullptr;
    if (sjac) {
      Y.jsc = A.take<cd>(c->n);
      wn = A.take<double>(c->n);
      if (mixed) wn32 = A.take<float>(c->n);
      Y.wn = wn;
      Y.wn32 = wn32;
    }
    Y.tile0 = tile0[k];
    Y.ntiles = ntl[k];
    if (st == HELM_OK) st = assemble_values(c, sys[k].freq, val, b, s, true, /*dia=*/true, cflag);
    if (st == HELM_OK && sys[k].rhs) {
      cudaError_t ce = cudaMemcpyAsync(b, sys[k].rhs, c->n * sizeof(cd), cudaMemcpyDeviceToDevice, s);
      if (ce != cudaSuccess) st = cuda_error(ce, "rhs copy");
    }
    if (st == HELM_OK && sjac)
      st = sym_jacobi_prepare(reinterpret_cast<double*>(val), cflag, b, Y.jsc, wn, wn32, c->n, c->mesh.nx, c->mesh.ny, s);
    if (st == HELM_OK && jac)
      st = jacobi_prepare(reinterpret_cast<double*>(val), cflag, Y.djac, c->n, c->mesh.nx, c->mesh.ny, c->mesh.nz, s);
    if (st == HELM_OK && prec == 1) st = cast_values(val, const_cast<cf*>(Y.val32), 27 * c->n, s);
    if (st == HELM_OK && prec == 2)
      st = split_values(reinterpret_cast<const double*>(val), const_cast<float2*>(Y.valw), c->n, Y.nsw, 54, s);
    if (st != HELM_OK) {
      cudaFree(A.base);
      return st;
    }
    memset(&hst[k], 0, sizeof(KState));
    hst[k].act = 1;
  }
  KSys* d_sys = A.take<KSys>(nsys);
  KState* d_st = A.take<KState>(nsys);
  KTile* d_tiles = A.take<KTile>(ntiles);
  int* d_l0 = A.take<int>(ntiles);
  int* d_l1 = A.take<int>(ntiles);
  int* d_ctrl = A.take<int>(CTRL_N);
  cd* d_part = A.take<cd>(2 * (size_t)ntiles);
  GridBar* d_bar = A.take<GridBar>(1);
  unsigned long long* d_trace = trace_steps ? A.take<unsigned long long>((size_t)trace_steps * kTraceStride) : nullptr;
  std::vector<int> l0(ntiles);
  for (int t = 0; t < ntiles; ++t) l0[t] = t;
  int ctrl[CTRL_N] = {0};
  ctrl[CTRL_CUR] = 0;
  ctrl[CTRL_CNT0] = ntiles;
  ctrl[CTRL_NACT] = nsys;
  cudaError_t e = cudaSuccess;
  auto H2D = [&](void* d, const void* h, size_t nb) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(d, h, nb, cudaMemcpyHostToDevice, s);
  };
  H2D(d_sys, hs.data(), nsys * sizeof(KSys));
  H2D(d_st, hst.data(), nsys * sizeof(KState));
  H2D(d_tiles, tiles.data(), ntiles * sizeof(KTile));
  H2D(d_l0, l0.data(), ntiles * sizeof(int));
  H2D(d_ctrl, ctrl, sizeof(ctrl));
  if (e == cudaSuccess) e = cudaMemsetAsync(d_bar, 0, sizeof(GridBar), s);

  KParams P;
  P.sys = d_sys;
  P.st = d_st;
  P.tiles = d_tiles;
  P.ntiles = ntiles;
  P.list0 = d_l0;
  P.list1 = d_l1;
  P.ctrl = d_ctrl;
  P.part = d_part;
  P.bar = d_bar;
  P.tol = o.tol;
  P.maxit = o.maxit;
  P.inner_tol = o.inner_tol;
  P.inner_maxit = o.inner_maxit;
  P.max_outer = o.max_outer;
  P.stall = o.stall_window;
  P.trace = d_trace;
  P.trace_steps = trace_steps;
  // tuning knobs of the double-word solve: HELM_PREFETCH (per-thread L2 prefetch distance of the
  // SpMV's matrix parts, block rows, 0 = off), HELM_PF_CHUNKS (bulk L2 prefetch distance of the
  // vector phases, 256-row chunks, 0 = off)
  const char* pfenv = getenv("HELM_PREFETCH");
  const char* pcenv = getenv("HELM_PF_CHUNKS");
  P.prefetch = pfenv ? std::max(0, std::min(atoi(pfenv), 8)) : 1;
  P.pf_chunks = pcenv ? std::max(0, std::min(atoi(pcenv), 16)) : 2;

  // Host-side fault injection for tests (never set in normal use): the barriers wait for one
  // block that does not exist and give up after 200 ms, so the launch ends with HELM_TIMEOUT
  // without faulting or hanging the GPU.
  const FaultMode fm = fault_mode();
  P.bar_extra = fm == FAULT_BARRIER ? 1u : 0u;
  P.bar_timeout = fm == FAULT_BARRIER ? 200000000ull : kTimeoutNs;
  // each super-step advances every active system by one Krylov step (one BiCGSTAB iteration),
  // except refinement residual steps (at most max_outer + 1 of them) and residual checks
  P.max_steps = 2 * o.maxit + 2 * (o.max_outer + 2) + 16;
  if (tfq) P.max_steps = 6 * o.maxit + 16;  // one barrier per sub-step, at most 4 per restart cycle
  void* args[] = {&P};
  if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
  if (e == cudaSuccess)
    e = cudaLaunchCooperativeKernel((const void*)kern, dim3(nblocks), dim3(kBlock), args, 0, s);
  if (e == cudaSuccess) e = cudaEventRecord(ev[2], s);
  // back to the unknowns of A x = b (also for a system that did not converge: its best iterate)
  if (jac)  // x = D^-1 y
    for (int k = 0; k < nsys && e == cudaSuccess; ++k)
      if (jacobi_unscale(hs[k].x, hs[k].djac, hs[k].n, s) != HELM_OK) e = cudaGetLastError();
  if (sjac)  // x = S y
    for (int k = 0; k < nsys && e == cudaSuccess; ++k)
      if (jacobi_rescale(hs[k].x, hs[k].jsc, hs[k].n, s) != HELM_OK) e = cudaGetLastError();
  GridBar hb;
  memset(&hb, 0, sizeof(hb));
  if (e == cudaSuccess) e = cudaMemcpyAsync(hst.data(), d_st, nsys * sizeof(KState), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, d_bar, sizeof(GridBar), cudaMemcpyDeviceToHost, s);
  std::vector<unsigned long long> htrace((size_t)trace_steps * kTraceStride);
  if (e == cudaSuccess && trace_steps)
    e = cudaMemcpyAsync(htrace.data(), d_trace, htrace.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(A.base);
  if (e == cudaSuccess && trace_steps > 1) {
    // mean durations (us) over the traced steps: own work of A, wait at barrier A, B work, B
    // wait, C work, C wait (block 0's view)
    double acc[6] = {0, 0, 0, 0, 0, 0};
    int cnt = 0;
    for (int k = 1; k < trace_steps; ++k) {
      const unsigned long long* t = &htrace[(size_t)k * kTraceStride];
      const unsigned long long prev = htrace[(size_t)(k - 1) * kTraceStride + 5];
      if (t[5] == 0 || prev == 0) break;
      acc[0] += (double)(t[0] - prev); acc[1] += (double)(t[1] - t[0]);
      acc[2] += (double)(t[2] - t[1]); acc[3] += (double)(t[3] - t[2]);
      acc[4] += (double)(t[4] - t[3]); acc[5] += (double)(t[5] - t[4]);
      ++cnt;
    }
    if (cnt)
      fprintf(stderr, "helm trace (%d steps, us): A work %.2f wait %.2f | B work %.2f wait %.2f | C work %.2f wait %.2f\n",
              cnt, acc[0] / cnt / 1e3, acc[1] / cnt / 1e3, acc[2] / cnt / 1e3, acc[3] / cnt / 1e3, acc[4] / cnt / 1e3,
              acc[5] / cnt / 1e3);
    // raw per-step record (HELM_TRACE_FILE=path): step, the six phase times relative to the
    // launch's first mark (ns), and the number of active tiles of the step
    const char* tf = getenv("HELM_TRACE_FILE");
    FILE* fh = tf ? fopen(tf, "w") : nullptr;
    if (fh) {
      const unsigned long long t0 = htrace[0];
      for (int k = 0; k < trace_steps; ++k) {
        const unsigned long long* t = &htrace[(size_t)k * kTraceStride];
        if (t[5] == 0) break;
        fprintf(fh, "%d %llu %llu %llu %llu %llu %llu %llu\n", k, t[0] - t0, t[1] - t0, t[2] - t0, t[3] - t0,
                t[4] - t0, t[5] - t0, t[6]);
      }
      fclose(fh);
    }
  }
  if (e == cudaSuccess) {
    float t_asm = 0.f, t_solve = 0.f;
    cudaEventElapsedTime(&t_asm, ev[0], ev[1]);
    cudaEventElapsedTime(&t_solve, ev[1], ev[2]);
    helm_profile& pr = last_profile();
    pr.assemble_ms += t_asm;
    pr.solve_ms += t_solve;
    // per system: assembly, + the complex64 cast or the double-word split, + Jacobi diagonal,
    // scaling and the final rescale; plus the persistent launch
    const int per_sys = 1 + (mixed ? 1 : 0) + ((jac || sjac) ? 3 : 0);
    pr.launches += (int64_t)nsys * per_sys + 1;
    pr.grid_blocks = nblocks;
    pr.ntiles = ntiles;
  }
  for (int q = 0; q < 3; ++q) cudaEventDestroy(ev[q]);
  if (e != cudaSuccess) return cuda_error(e, "cocg persistent solve");

  helm_status overall = HELM_OK;
  const bool dbg = getenv("HELM_DEBUG_STATE") != nullptr;  // diagnosis aid: state of failed systems
  for (int k = 0; k < nsys; ++k) {
    helm_solve_stats& S = *sys[k].stats;
    const KState& K = hst[k];
    if (dbg && (K.act || K.status != HELM_OK))
      fprintf(stderr,
              "helm state sys %d: status %d it %d bd %d est %.3e relres %.3e rho (%.3e,%.3e) alpha (%.3e,%.3e) "
              "omega (%.3e,%.3e) beta (%.3e,%.3e) tau %.3e theta %.3e\n",
              k, K.status, K.it, K.bd, K.est, K.relres, K.rho.re, K.rho.im, K.alpha.re, K.alpha.im, K.omega.re,
              K.omega.im, K.beta.re, K.beta.im, K.tau, K.theta);
    S.status = K.act ? HELM_NOT_CONVERGED : K.status;
    if (hb.status & DEV_TIMEOUT) S.status = HELM_TIMEOUT;
    S.iterations = K.it;
    S.restarts = K.restarts;
    S.outer = K.fell_back ? -K.outer : K.outer;
    S.iterations_c64 = K.it32;
    S.pad = 0;
    S.relres = K.relres;
    S.bnorm = K.bnorm;
    if (S.status != HELM_OK && overall == HELM_OK) overall = (helm_status)S.status;
  }
  if (hb.status & DEV_TIMEOUT) return set_error(HELM_TIMEOUT, "persistent solver: grid barrier timed out");
  if (overall != HELM_OK) set_error(overall, "at least one system did not converge");
  return overall;
}

}  // namespace helm
