/*
 * helm.h -- C ABI of the GB300 cavity-Helmholtz frequency-response library (libhelm.so).
 *
 * Problem (paper Sec. 3.2, Helmholtz equation): the time-harmonic acoustic pressure p in a
 * closed cavity satisfies -w^2 p - c^2 lap(p) = 0; the pressure fluctuation computed over the
 * sun-roof opening is imposed as Dirichlet data there. Discretised with trilinear (Q1) bricks
 * on a box lattice, each frequency f (k = 2 pi f / c) gives the complex symmetric system
 *
 *     (K - k^2 M + i k rho c B(beta)) p = 0   with p = p_D on the Dirichlet nodes,
 *
 * K the stiffness, M the mass, B(beta) = sum_e beta_e B_e the admittance (wall) term over
 * boundary quads e (quad mass B_e, beta_e complex, 0 = rigid). Sign reading: e^{+i w t}, so
 * Re(beta) > 0 absorbs. The Dirichlet nodes are eliminated symmetrically: their rows and
 * columns become identity rows/columns and b_F = -A_FD p_D, b_D = p_D, so the matrix stays
 * complex symmetric (A == A^T). Paper Sec. 4: the system is stored in CSR and solved by Krylov
 * methods in complex double precision on the GPU.
 *
 * Numbering (shared with every caller):
 *   node id       = i + (nx+1) * (j + (ny+1) * l),  0<=i<=nx, 0<=j<=ny, 0<=l<=nz, z vertical;
 *   boundary quads: sides in the order x-, x+, y-, y+, z-, z+; inside a side the quad at
 *                   in-plane element indices (u, v) is u + nu * v, u the first remaining axis
 *                   (x before y before z). n_bface = 2 (ny nz + nx nz + nx ny).
 *   CSR pattern   : full 27-point pattern of the lattice, columns ascending in every row;
 *                   entries forced to zero by the elimination stay as explicit zeros.
 *
 * Complex data are interleaved (re, im) pairs: double[2] for complex128, float[2] for
 * complex64 -- the layout of torch.complex128 / torch.complex64.
 *
 * Conventions for every entry point:
 *   - Pointers marked (dev) are device pointers of the current CUDA device, (host) host ones.
 *   - The caller owns every buffer it passes; the library owns helm_ctx / helm_matrix /
 *     helm_shared and the scratch they allocate (freed by helm_destroy / helm_matrix_free /
 *     helm_shared_free).
 *   - Work is ordered on the stream given to helm_create (or to helm_spmv); calls return
 *     without synchronising unless stated otherwise.
 *   - A non-HELM_OK status comes with a message from helm_last_error(). No C++ exception
 *     crosses this boundary. Argument errors are detected before any device work is queued.
 */
#ifndef HELM_H
#define HELM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { int32_t nx, ny, nz; double Lx, Ly, Lz; } helm_mesh_desc; /* box lattice, metres */
typedef struct { double c, rho; } helm_phys;                               /* m/s, kg/m^3 */

typedef enum {
  HELM_OK = 0,
  HELM_ERR_ARG = 1,        /* invalid argument (null pointer, bad size, bad option) */
  HELM_ERR_CUDA = 2,       /* a CUDA runtime call failed */
  HELM_ERR_OOM = 3,        /* device allocation failed */
  HELM_NOT_CONVERGED = 4,  /* solve hit maxit; best iterate and stats are still written */
  HELM_BREAKDOWN = 5,      /* Krylov breakdown (COCG p^T A p == 0 or r^T r == 0; BiCGSTAB / TFQMR
                              (r0*, v) == 0, rho == 0 or omega == 0) */
  HELM_NAN = 6,            /* non-finite residual */
  HELM_PIVOT = 7,          /* Schwarz local factorisation met a pivot below threshold */
  HELM_TIMEOUT = 8,        /* a device-side wait gave up (bounded barrier) */
  HELM_ERR_STATE = 9       /* call out of order (e.g. solve before helm_set_boundary) */
} helm_status;

enum { HELM_C128 = 0, HELM_C64 = 1 };                 /* matrix value precision */
enum { HELM_FMT_CSR = 0, HELM_FMT_DIA27 = 1 };         /* matrix layout (see helm_assemble) */
enum { HELM_SOLVER_GMRES = 0, HELM_SOLVER_COCG = 1, HELM_SOLVER_BICGSTAB = 2, HELM_SOLVER_TFQMR = 3 }; /* Krylov method */
enum { HELM_PRECOND_NONE = 0, HELM_PRECOND_RAS = 1, HELM_PRECOND_JACOBI = 2, HELM_PRECOND_ORAS = 3,
       HELM_PRECOND_ORAS2 = 4 };
/* preconditioner (right, except the symmetric Jacobi form of COCG) */

typedef struct {
  int32_t solver;       /* HELM_SOLVER_GMRES: restarted GMRES(restart), CGS2 Arnoldi, complex
                           Givens; HELM_SOLVER_COCG: conjugate-orthogonal CG (A complex symmetric);
                           HELM_SOLVER_BICGSTAB: BiCGSTAB (paper Sec. 4, Table 3),
                           stats.iterations counts iterations of two SpMVs;
                           HELM_SOLVER_TFQMR: transpose-free QMR (paper Sec. 4, Table 3),
                           stats.iterations counts steps (one SpMV each on average) */
  int32_t restart;      /* GMRES cycle length m (1..128) */
  double tol;           /* stop when the true ||b - A p||_2 / ||b||_2 <= tol */
  int32_t maxit;        /* Krylov steps (SpMVs inside the iteration) before HELM_NOT_CONVERGED */
  int32_t precond;      /* HELM_PRECOND_NONE; HELM_PRECOND_RAS (GMRES only); HELM_PRECOND_ORAS (GMRES
                           only): RAS whose subdomain matrices carry the optimized-Schwarz interface
                           term i k M_G (face mass of the subdomain's faces inside the lattice,
                           Dirichlet nodes excluded; paper Sec. 4 names absorbing Robin interface
                           conditions, i k is the matched impedance of the wall term);
                           HELM_PRECOND_ORAS2 (GMRES only): the two-sided form of the paper's
                           optimized Schwarz method (Sec. 4: different interface conditions on
                           the two sides of an interface): each subdomain matrix carries
                           (robin_lo / h_a) M_face on the low faces of its extended box (planes
                           i0, j0, l0) and (robin_hi / h_a) M_face on its high faces, h_a the
                           lattice spacing normal to the face, Dirichlet nodes excluded;
                           HELM_PRECOND_JACOBI
                           (not GMRES), the reading of the paper's unnamed "P": BiCGSTAB / TFQMR
                           run on A D^-1 (D = diag(A), right Jacobi) and return x = D^-1 y; COCG
                           (FP64 or mixed) runs on S A S with S = D^-1/2 (principal root; stays
                           complex symmetric), b scaled by S, residual norms weighted by |a_ii|,
                           and returns x = S y. Either way tol and stats.relres refer to
                           A x = b */
  int32_t ras_parts[3]; /* Schwarz blocks along x, y, z */
  int32_t ras_overlap;  /* lattice layers of overlap */
  int32_t mixed;        /* 0: FP64 COCG. 1: FP64 iterative refinement around a complex64 inner
                           COCG. 2: the same around a double-word inner COCG (every inner value a
                           pair of floats hi + lo, about 48 significand bits, computed on the
                           FP32 pipe; no counterpart in the paper, a GB300 choice: its FP64 rate
                           is 1/64 of its FP32 rate). COCG only. A system whose refinement step
                           fails to halve the FP64 residual is restarted as FP64 COCG from zero
                           (stats.outer < 0 marks such a fallback: -outer refinement steps were
                           taken before it) */
  double inner_tol;     /* mixed: inner relative residual reduction per refinement step; an inner
                           solve also stops once its residual reaches tol * ||b|| / 2, and (with
                           stall_window) when its estimate stops halving */
  int32_t inner_maxit;  /* mixed: inner steps per refinement step */
  int32_t max_outer;    /* mixed: refinement steps before HELM_NOT_CONVERGED */
  int32_t stall_window; /* COCG: if the residual estimate has not halved its best value within
                           this many steps, check the true residual and restart (0 = never;
                           counted in stats.restarts) -- from the iterate saved at the last
                           halving if that happened since the last restart and the estimate is
                           above it now, else from the current iterate; the same rule picks the
                           iterate returned at the step cap. Mixed: ends the inner solve (the
                           next refinement step restarts from the current iterate) */
  int32_t pad_;
  double robin_lo[2];   /* HELM_PRECOND_ORAS2: dimensionless complex coefficient (re, im) of the
                           low faces; finite */
  double robin_hi[2];   /* HELM_PRECOND_ORAS2: the same for the high faces */
} helm_solve_opts;

typedef struct {
  int32_t status;       /* helm_status of this system */
  int32_t iterations;   /* Krylov steps (inner steps included when mixed) */
  int32_t restarts;     /* GMRES cycles - 1 / COCG, BiCGSTAB, TFQMR restarts after a missed
                           true-residual check */
  int32_t outer;        /* mixed: refinement steps taken */
  double relres;        /* true FP64 ||b - A p|| / ||b|| at exit */
  double bnorm;         /* ||b||_2 */
  int32_t iterations_c64; /* mixed: the inner (complex64 or double-word) steps among `iterations` */
  int32_t pad;
} helm_solve_stats;

typedef struct {
  double assemble_ms;   /* device time of the assembly / lifting / cast kernels of the last solve */
  double solve_ms;      /* device time of the Krylov kernels of the last solve (CUDA events on
                           the solve stream around the persistent launch / the GMRES cycles) */
  int64_t launches;     /* kernels this library launched in the last solve call */
  int32_t grid_blocks;  /* blocks of the persistent launch (0 for GMRES) */
  int32_t ntiles;       /* row tiles of the persistent launch */
} helm_profile;

typedef struct helm_ctx helm_ctx;       /* one lattice + physics + boundary data */
typedef struct helm_matrix helm_matrix; /* one assembled, eliminated system matrix (CSR or DIA27) */
typedef struct helm_shared helm_shared; /* frequency-independent parts K, M, B of a lattice */

/* Last error message of the calling thread ("" if none). Owned by the library. */
const char* helm_last_error(void);

/* Create a context for the lattice `mesh` (nx,ny,nz >= 1, lengths > 0) and physics `phys`,
 * ordering its work on `stream` (a cudaStream_t, NULL = legacy default stream). */
helm_status helm_create(helm_ctx** out, const helm_mesh_desc* mesh, const helm_phys* phys,
                        void* stream);
void helm_destroy(helm_ctx* ctx);

/* Boundary data (paper Sec. 3.2: sun-roof pressure as Dirichlet data; walls by admittance).
 *   beta_face (dev) complex128 [n_bface]: admittance per boundary quad, 0 = rigid; may be NULL
 *                   (all rigid).
 *   dir_nodes (dev) int32 [n_dir]: distinct node ids with prescribed pressure, any order.
 *   p_dir     (dev) complex128 [n_dir]: the prescribed pressure at dir_nodes.
 * The library copies the data; the caller may free its buffers after the call returns and
 * the stream has passed it. n_dir may be 0 (pure admittance problem). */
helm_status helm_set_boundary(helm_ctx* ctx, const double* beta_face, const int32_t* dir_nodes,
                              int32_t n_dir, const double* p_dir);

/* Sizes of the context's lattice. Any output pointer may be NULL. */
helm_status helm_sizes(const helm_ctx* ctx, int64_t* n_nodes, int64_t* nnz, int64_t* n_bface,
                       int32_t* n_dir);

/* Assemble the eliminated system matrix at frequency freq_hz (paper Sec. 3.2 Helmholtz eq.)
 * in `precision` (HELM_C128, or HELM_C64: complex64 values rounded from the complex128 ones)
 * and `format`:
 *   HELM_FMT_CSR   -- compressed sparse rows (paper Sec. 4), the context's 27-point pattern;
 *   HELM_FMT_DIA27 -- slot-major 27-point layout with real and imaginary parts split: 27 n real
 *                     parts re[k * n + row] followed by 27 n imaginary parts im[k * n + row]
 *                     (FP64, or FP32 for HELM_C64), k = (di+1) + 3 (dj+1) + 9 (dl+1) for the
 *                     neighbour row + di + (nx+1) (dj + (ny+1) dl); slots whose neighbour is
 *                     outside the lattice hold zero. Same values as the CSR form.
 * If b_out (dev, complex128 [n]) is not NULL the lifted right-hand side b_F = -A_FD p_D,
 * b_D = p_D is written there. *A_out is owned by the caller's handle until helm_matrix_free and
 * must be freed before its context. */
helm_status helm_assemble(helm_ctx* ctx, double freq_hz, int32_t precision, int32_t format,
                          helm_matrix** A_out, double* b_out);
void helm_matrix_free(helm_matrix* A);

/* Read-only views of a CSR matrix: rowptr (dev int32 [n+1]), col (dev int32 [nnz]), val (dev
 * complex [nnz], complex128 or complex64 per precision). Any pointer may be NULL.
 * HELM_ERR_ARG for a DIA27 matrix. */
helm_status helm_matrix_csr(const helm_matrix* A, int64_t* n, int64_t* nnz, int32_t* precision,
                            const int32_t** rowptr, const int32_t** col, const void** val);

/* Read-only view of a DIA27 matrix: val (dev, 54 n reals: 27 n real parts then 27 n imaginary
 * parts, layout above). HELM_ERR_ARG for CSR. */
helm_status helm_matrix_dia27(const helm_matrix* A, int64_t* n, int32_t* precision, const void** val);

/* y = A x (paper Sec. 4: the SpMV dominates the cost of a Krylov step) for either layout. x, y (dev)
 * complex [n] in the matrix precision (complex64 matrices accumulate in FP32), must not overlap. Ordered on
 * `stream` (cudaStream_t; NULL = the context stream of the matrix). */
helm_status helm_spmv(const helm_matrix* A, const void* x, void* y, void* stream);

/* Frequency-independent parts of the context's eliminated operator A(k) = K - k^2 M
 * + i k rho c B(beta) (paper Sec. 3.2): K, M and the wall term B, slot-major like DIA27, with the
 * Dirichlet rows of K set to the identity and Dirichlet rows / columns of M, B and the other K
 * entries zero, so that A(k) of every frequency is the eliminated system matrix of helm_assemble
 * (the k-dependent lifting of b is not part of the operator). precision: HELM_C128 (FP64 parts)
 * or HELM_C64 (FP32 copies as well). Needs helm_set_boundary first; reflects the boundary data at
 * the time of the call. *out is owned by the caller until helm_shared_free; the context must
 * outlive it. Ordered on the context stream. */
helm_status helm_assemble_shared(helm_ctx* ctx, int32_t precision, helm_shared** out);
void helm_shared_free(helm_shared* S);

/* Shared-mesh multi-frequency product ("SpMM"): Y[f] = A(2 pi freqs_hz[f] / c) X[f] for
 * f < nfreq, reading K and M once per row for up to 8 frequencies at a time (B only on rows with
 * a wall term). X, Y (dev) complex in the precision of S, frequency-major [nfreq][n], must not
 * overlap; freqs_hz (host) >= 0. No counterpart in the paper's code: its FRF evaluates the
 * operator one frequency at a time. Ordered on `stream` (NULL = the context stream). */
helm_status helm_spmv_multi(const helm_shared* S, const double* freqs_hz, int32_t nfreq, const void* X,
                            void* Y, void* stream);

/* The same products with X and Y node-major ("frequency-interleaved"): X[i * nfreq + f] is node
 * i's value for frequency f, so one 16-byte-aligned block per node carries all frequencies and the
 * product gathers each neighbour's block once (paper Sec. 3.1: the FRF evaluates the Sec. 3.2
 * operator at many frequencies on one mesh). nfreq: 2, 4 or 8 for HELM_C64, 1, 2, 4 or 8 for
 * HELM_C128 (HELM_ERR_ARG otherwise); X, Y (dev) 16-byte aligned, not overlapping; freqs_hz (host)
 * >= 0. Ordered on `stream` (NULL = the context stream); does not synchronise. */
helm_status helm_spmv_multi_interleaved(const helm_shared* S, const double* freqs_hz, int32_t nfreq,
                                        const void* X, void* Y, void* stream);

/* Reductions over complex128 vectors x, y (dev, [n]), FP64 accumulation in a fixed order:
 * op 0: x^H y (conjugated, GMRES), op 1: x^T y (unconjugated, COCG), op 2: ||x||_2 (y unused).
 * The result (host, double[2]) is written after the call synchronises `stream`. */
helm_status helm_reduce(int32_t op, int64_t n, const double* x, const double* y, double* out,
                        void* stream);

/* The reduction of helm_reduce without any device allocation. The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc while they run -- e.g. an
 * application that reserves all device memory for its own pool at start-up, or a latency-bound
 * loop that cannot afford the implicit device synchronisation of cudaMalloc / cudaFree. The
 * caller still passes x, y (dev) and out (host, double[2]); the partial sums go to a static
 * device array of the library (64 KiB per device, kept until the process exits).
 *   - n may be at most 16,777,216 (4096 partial sums of 4096 elements); larger n returns
 *     HELM_ERR_ARG with a message naming the limit.
 *   - The first call on a device looks up the array's device address (once per device, with
 *     that device current); make that first call before any stream capture. The address is
 *     cached for the life of the process: after cudaDeviceReset (or any teardown of the
 *     device's primary context) this entry point must not be called again in that process.
 *   - Every call shares the array and overwrites what it uses; calls that overlap on the GPU
 *     (concurrent streams, threads) race and must be serialised by the caller.
 * Results agree with helm_reduce to rounding (the partial sums are grouped differently);
 * repeated calls with the same input are bitwise identical. Synchronises `stream`. */
helm_status helm_reduce_noalloc(int32_t op, int64_t n, const double* x, const double* y,
                                double* out, void* stream);

/* Frequency response: solve the system of every frequency freqs_hz[0..nfreq) (host) on the
 * context's lattice. p_out (dev, complex128 [nfreq][n]) receives the pressure (the best
 * iterate if not converged); stats (host, [nfreq]) the per-frequency statistics. COCG,
 * BiCGSTAB and TFQMR systems (COCG: FP64 or mixed) advance together in one persistent cooperative launch; GMRES systems run
 * one after another, each restart cycle a captured CUDA graph. Synchronises the stream.
 * Returns HELM_OK if every system converged, else the first failing status. */
helm_status helm_solve(helm_ctx* ctx, const double* freqs_hz, int32_t nfreq,
                       const helm_solve_opts* opts, double* p_out, helm_solve_stats* stats);

/* Batched frequency-response sweep over systems that may live on different lattices:
 * system s is context ctxs[s] (host array) at frequency freqs_hz[s] (host); its pressure goes
 * to p_out[s] (host array of dev pointers, complex128 [n_s]). COCG (FP64 or mixed), BiCGSTAB or TFQMR; all
 * systems advance together in one persistent cooperative launch. Synchronises the first
 * context's stream. */
helm_status helm_solve_batch(helm_ctx* const* ctxs, const double* freqs_hz, int32_t nsys,
                             const helm_solve_opts* opts, double* const* p_out,
                             helm_solve_stats* stats);

/* Adjoint gradient of the listener objective J = sum_f sum_i w_i |p_i(f)|^2.
 *   p      (dev) complex128 [nfreq][n]: forward pressures from helm_solve at freqs_hz.
 *   w_node (dev) float64 [n]: listener weights (e.g. 1/|S| inside the listener region).
 * Because A is complex symmetric the adjoint system is A lam = W conj(p), solved with
 * `opts` (any options helm_solve accepts: solver, precision mode, preconditioner). Outputs (PyTorch convention for a real loss:
 * d/dRe + i d/dIm), summed over frequencies:
 *   grad_beta (dev) complex128 [n_bface]: -2 conj(lam_F^T (i k rho c B_e) p) per boundary quad;
 *   grad_pdir (dev) complex128 [n_dir]  :  2 conj(W_D conj(p_D) - A_DF lam_F) per Dirichlet node
 *                                          (in the order given to helm_set_boundary);
 *   J_out     (host, may be NULL)       : the objective.
 * Synchronises the stream. */
helm_status helm_adjoint_grad(helm_ctx* ctx, const double* freqs_hz, int32_t nfreq,
                              const helm_solve_opts* opts, const double* p, const double* w_node,
                              double* grad_beta, double* grad_pdir, double* J_out);

/* Timing record of the calling thread's last helm_solve / helm_solve_batch (host, written). */
helm_status helm_last_profile(helm_profile* out);

/* Measurement aid (no counterpart in the paper's method; it calibrates the rooflines of the
 * complex double-precision kernels of paper Sec. 4, whose FP64 multiply-adds bound them on GPUs
 * with a reduced FP64 rate): runs a kernel of independent FP64 FMA chains over the whole device
 * for `iters` steps per chain on `stream` (NULL = default stream), times it with CUDA events and
 * writes the measured rate in FMA/s to *fma_per_s (host). Allocates and frees a small device
 * buffer; synchronises the stream. HELM_ERR_ARG for iters <= 0 or a null output. */
helm_status helm_probe_fp64_fma(int32_t iters, double* fma_per_s, void* stream);

/* Adjoint gradient for any real loss L(p) of the pressures (the backward step of an autograd
 * wrapper). grad_p (dev, complex128 [nfreq][n]) is PyTorch's gradient of L with respect to
 * p = helm_solve's output (dL/dRe p + i dL/dIm p). With lam = A^-1 conj(grad_p) (one adjoint
 * solve per frequency, A complex symmetric) and lam_F = lam zeroed on the Dirichlet nodes:
 *   grad_beta (dev, complex128 [n_bface]) += -conj(lam_F^T (i k rho c B_e) p) per boundary quad;
 *   grad_pdir (dev, complex128 [n_dir])   +=  conj(lam_D - A_DF lam_F) per Dirichlet node;
 * both overwritten (not accumulated across calls), summed over frequencies. helm_adjoint_grad is
 * this call with grad_p = 2 w p. Synchronises the stream. */
helm_status helm_adjoint_seed(helm_ctx* ctx, const double* freqs_hz, int32_t nfreq,
                              const helm_solve_opts* opts, const double* p, const double* grad_p,
                              double* grad_beta, double* grad_pdir);

#ifdef __cplusplus
}
#endif
#endif /* HELM_H */
