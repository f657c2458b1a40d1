"""Benchmark: frequency-response sweep throughput on GB300 (one JSON line on stdout).

Workload (default "sweep256"): 256 log-spaced frequencies 20-500 Hz, each solved on its own
wavelength-scaled 2.5 x 1.4 x 1.2 m cabin lattice (24x14x12 .. 148x83x71 bricks, 25.17 M nodes
in total) with the sun-roof Dirichlet pressure and random seat admittances, to a true FP64
relative residual of 1e-10. One step = assembly + lifting + COCG solve of all 256 systems in
one call (helm_solve_batch: one persistent cooperative launch). Inputs (lattices, boundary
data) are resident on the device before timing; the 10.9 GB of matrix values the step
assembles exceed L2, so no flush is needed.

The main (timed) leg is FP64 iterative refinement around a double-word inner COCG (pairs of
floats, about 48 bits) with symmetric Jacobi scaling. The same line reports the other batched
COCG modes (FP64, complex64 inner with FP64 refinement, FP64 without preconditioner), FP64 COCG
run one frequency per call, the SpMV roofline on the 2,203,161-node lattice (CSR and slot-major
layouts, complex128 and complex64, L2 flushed), the end-to-end figure through host buffers, the
CPU oracle on a fixed sample of the sweep (cpu_baseline) and the headline results' error against
the oracle on that sample (oracle_error). `--precision` picks another mode for the timed leg;
`--impl reference` times the CPU oracle alone on the same sample.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import helm_inputs as hi  # noqa: E402

METRIC = "FRF freqs/s at rel-res 1e-10: batched+mixed vs plain FP64; SpMV % HBM roofline"
TOL = 1e-10


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one persistent launch of the
# default benchmark step, from a single-pass ncu capture of the full-size run, valid only for
# the kernel sources it was taken on: reported as null once they change.
TRAFFIC_CAPTURE = {"config": "sweep256/cocg/dw/jacobi", "sources_sha256_16": "62572e8e3aaceb6c",
                   "bytes": 25750236950016 + 4990120506624}
KERNEL_SOURCES = ("paper_2112_00087_gb300/csrc/krylov_cocg.cu", "paper_2112_00087_gb300/csrc/krylov_engine.cuh",
                  "paper_2112_00087_gb300/csrc/kernels.cuh", "paper_2112_00087_gb300/csrc/dw.cuh",
                  "paper_2112_00087_gb300/csrc/common.cuh", "paper_2112_00087_gb300/csrc/krylov_host.cu",
                  "paper_2112_00087_gb300/csrc/bulk.cuh")


def captured_traffic(args):
    if args.traffic is not None:
        return args.traffic
    key = "%s/%s/%s/%s" % (args.workload if args.nfreq == 256 else "other", args.solver,
                           "c64" if args.mixed else args.precision, args.precond)
    if key != TRAFFIC_CAPTURE["config"] or TRAFFIC_CAPTURE["bytes"] is None:
        return None
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return TRAFFIC_CAPTURE["bytes"] if h.hexdigest()[:16] == TRAFFIC_CAPTURE["sources_sha256_16"] else None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------------------------
# algorithmic bytes (what each solver step must move)
# ---------------------------------------------------------------------------------------------

def spmv_bytes(n, nnz, vb):
    """CSR SpMV: values + int32 columns + rowptr + x read once + y written once."""
    return nnz * (vb + 4) + (n + 1) * 4 + 2 * vb * n


def dia_spmv_bytes(n, vb):
    """Slot-major split-layout SpMV: 27 n real parts (vb/2 bytes each) + x read once + y written
    once (the imaginary parts, read only for rows next to admittance walls, are not counted)."""
    return 27 * n * (vb // 2) + 2 * vb * n


def cocg_fp64_bytes(n, nnz, st):
    it, chk = st["iterations"], st["restarts"] + 1
    per_it = dia_spmv_bytes(n, 16) + 96 * n + 48 * n      # SpMV, x/r update, p update
    check = dia_spmv_bytes(n, 16) + 32 * n                # b read, r written
    return it * per_it + chk * check + 48 * n             # + init (b read, x and r written)


# FP64 flops per row of one FP64 COCG step: 27 complex-by-real stencil products (4 flops each),
# the p^T q and r^T r / ||r||^2 dot products, the x, r and p updates -- 152 in total.
FP64_FLOPS_PER_ROW_STEP = 27 * 4 + 8 + 8 + 8 + 8 + 4 + 8


def cocg_fp64_flops(n, st):
    return (st["iterations"] - st.get("iterations_c64", 0)) * n * FP64_FLOPS_PER_ROW_STEP


def bicgstab_bytes(n, nnz, st):
    """FP64 BiCGSTAB: per iteration two SpMVs (v = A p, t = A s) and 240 n bytes of vector
    traffic -- rs read (16), s = r - alpha v (48), x/r updates and rs^H r (112), p update (64)."""
    it, chk = st["iterations"], st["restarts"] + 1
    return it * (2 * dia_spmv_bytes(n, 16) + 240 * n) + chk * (dia_spmv_bytes(n, 16) + 32 * n) + 48 * n


def cocg_dw_bytes(n, nnz, st):
    """Double-word mixed mode: an inner step moves the SpMV (matrix parts as 8-byte (hi, lo) float
    pairs, x read once and y written once as 16-byte complex double-words), the r update (q and r
    read, r written: 48n) and the x and p updates together (r, p, x read, p and x written: 80n), 376
    bytes per row; FP64 fallback steps move an FP64 step's bytes; plus the FP64 refinement
    residuals, inner starts (r read, r and d written) and corrections (d, p and x read, x
    written)."""
    it_in, outer = st["iterations_c64"], abs(st["outer"])
    it64 = st["iterations"] - it_in
    step = dia_spmv_bytes(n, 16) + 48 * n + 80 * n
    step64 = dia_spmv_bytes(n, 16) + 96 * n + 48 * n
    resid = dia_spmv_bytes(n, 16) + 32 * n
    return it_in * step + it64 * step64 + (outer + 1) * resid + outer * (48 * n + 64 * n) + 48 * n


def tfqmr_bytes(n, nnz, st):
    """FP64 TFQMR, per step (half of a pair of two SpMVs): one SpMV and 208 n bytes of vector
    traffic (a pair moves 416 n: even step 112, odd step 144, u update 96, v update 64)."""
    it, chk = st["iterations"], st["restarts"] + 1
    # per (re)start cycle: true residual (SpMV, b read, r written), setup (r read, w u r0* d
    # written), first v = A u (SpMV, r0* read)
    return it * (dia_spmv_bytes(n, 16) + 208 * n) + chk * (2 * dia_spmv_bytes(n, 16) + 32 * n + 80 * n + 16 * n) + 48 * n


TFQMR_FLOPS_PER_ROW_STEP = (2 * 27 * 4 + 28 + 36 + 16 + 24) // 2


def tfqmr_flops(n, st):
    return st["iterations"] * n * TFQMR_FLOPS_PER_ROW_STEP


# FP64 flops per row of one BiCGSTAB iteration: two stencil products (2 x 108) and 80 for the
# rs^H v, t^H s, t^H t, rs^H r, ||r||^2 dots and the s, x, r, p updates.
BICG_FLOPS_PER_ROW_IT = 2 * 27 * 4 + 8 + 8 + 8 + 4 + 16 + 8 + 8 + 4 + 16


def bicgstab_flops(n, st):
    return st["iterations"] * n * BICG_FLOPS_PER_ROW_IT


def cocg_mixed_bytes(n, nnz, st):
    it32, outer = st["iterations_c64"], abs(st["outer"])
    it64 = st["iterations"] - it32                        # FP64 COCG steps after a fallback
    inner = dia_spmv_bytes(n, 8) + 48 * n + 24 * n        # c64 SpMV, x/r update, p update
    resid = dia_spmv_bytes(n, 16) + 32 * n                # FP64 true residual
    fp64 = dia_spmv_bytes(n, 16) + 96 * n + 48 * n
    return it32 * inner + it64 * fp64 + (outer + 1) * resid + outer * (32 * n + 40 * n) + 48 * n


# ---------------------------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ---------------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------------

def build_sweep(nfreq, helm, torch, workload="sweep256"):
    if workload == "sweep256":
        freqs = hi.sweep_freqs(256)
        if nfreq < 256:
            freqs = freqs[np.linspace(0, 255, nfreq).round().astype(int)]
        probs = [hi.cabin_problem(*hi.sweep_mesh_dims(f)) for f in freqs]
    else:  # one lattice, several frequencies (profiling cases)
        dims = {"cabin2m": (200, 112, 96), "cabin282k": (100, 56, 48)}[workload]
        lo, hi_ = (100.0, 400.0) if workload == "cabin2m" else (20.0, 200.0)
        freqs = np.geomspace(lo, hi_, max(1, nfreq))
        pr = hi.cabin_problem(*dims)
        probs = [pr] * len(freqs)
    ctxs = []
    for pr in probs:
        m = pr.mesh
        c = helm.Context(m.nx, m.ny, m.nz, m.Lx, m.Ly, m.Lz)
        c.set_boundary(torch.from_numpy(pr.beta).cuda(), torch.from_numpy(pr.dir_nodes).cuda(),
                       torch.from_numpy(pr.p_dir).cuda())
        ctxs.append(c)
    outs = [torch.empty(c.n, dtype=torch.complex128, device="cuda") for c in ctxs]
    return freqs, probs, ctxs, outs


# COCG stagnation window: longer than any plateau of a system that converges without a restart
# (the longest sweep system, 500 Hz, converges in about 13,500 steps), so the rule only touches
# systems that are genuinely stuck (374 Hz sits near rel-res 1e-2 without it).
STALL = 15000


def mixed_opts(helm, maxit=45000, precond=None):
    return helm.make_opts("cocg", tol=TOL, maxit=maxit, mixed=True, inner_tol=1e-4, inner_maxit=600, max_outer=40,
                          stall_window=STALL, precond=precond)


def fp64_opts(helm, maxit=45000, precond=None):
    return helm.make_opts("cocg", tol=TOL, maxit=maxit, stall_window=STALL, precond=precond)


def dw_opts(helm, maxit=45000, precond=None):
    # double-word inner solve straight to the outer target (inner_tol below it), FP64 refinement
    return helm.make_opts("cocg", tol=TOL, maxit=maxit, mixed="dw", inner_tol=1e-12, inner_maxit=maxit, max_outer=20,
                          stall_window=STALL, precond=precond)


def bicgstab_opts(helm, maxit=45000, precond=None):
    return helm.make_opts("bicgstab", tol=TOL, maxit=maxit, precond=precond)


def tfqmr_opts(helm, maxit=45000, precond=None):
    return helm.make_opts("tfqmr", tol=TOL, maxit=maxit, precond=precond)


def max_over_ranks(secs, dist, device):
    """Slowest rank's time (the benchmark's value divides every rank's work by it)."""
    if dist is None:
        return secs
    import torch
    t = torch.tensor([float(secs)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def job_value(world, units_per_rank, steps, secs):
    """Whole-job throughput: the units all ranks processed divided by the slowest rank's time."""
    return world * units_per_rank * steps / secs


def timed(fn, torch, K, W, dist=None):
    for _ in range(W):
        fn()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(s)
    outs = [fn() for _ in range(K)]
    e1.record(s)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if dist is not None:
        dist.barrier()
    return e0.elapsed_time(e1) / 1000.0, wall, outs


def spmv_roofline(helm, torch, peak_gbs, fp64_tflops=None):
    """helm_spmv on the 2,203,161-node lattice, complex128 and complex64, L2 flushed between reps.
    The complex128 products are bound by the FP64 pipe: for them the line also gives the FP64 rate
    (4 flops per stored entry: the real part of each entry times x's two components) against the
    measured FP64 peak."""
    pr = hi.cabin_problem(200, 112, 96)
    m = pr.mesh
    ctx = helm.Context(m.nx, m.ny, m.nz, m.Lx, m.Ly, m.Lz)
    ctx.set_boundary(torch.from_numpy(pr.beta).cuda(), torch.from_numpy(pr.dir_nodes).cuda(),
                     torch.from_numpy(pr.p_dir).cuda())
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    out = {}
    cases = (("csr_c128", helm.HELM_C128, helm.HELM_FMT_CSR, torch.complex128, 16),
             ("csr_c64", helm.HELM_C64, helm.HELM_FMT_CSR, torch.complex64, 8),
             ("dia27_c128", helm.HELM_C128, helm.HELM_FMT_DIA27, torch.complex128, 16),
             ("dia27_c64", helm.HELM_C64, helm.HELM_FMT_DIA27, torch.complex64, 8))
    for name, prec, fmt, dt, vb in cases:
        A = helm.helm_assemble(ctx, 250.0, prec, with_rhs=False, fmt=fmt)
        x = torch.randn(ctx.n, dtype=dt, device="cuda")
        y = torch.empty_like(x)
        for _ in range(3):
            helm.helm_spmv(A, x, y)
        times = []
        s = torch.cuda.current_stream()
        for _ in range(10):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            helm.helm_spmv(A, x, y)
            e1.record(s)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1000.0)
        # CSR: values + columns + rowptr + x + y; DIA27: the 27 n stored real parts (padding
        # included, no columns) + x + y
        b = spmv_bytes(ctx.n, ctx.nnz, vb) if fmt == helm.HELM_FMT_CSR else dia_spmv_bytes(ctx.n, vb)
        best, med = min(times), statistics.median(times)
        out[name] = {"n": ctx.n, "nnz": ctx.nnz, "bytes": b, "best_ms": best * 1e3, "median_ms": med * 1e3,
                     "gbs_best": b / best / 1e9, "gbs_median": b / med / 1e9, "frac_median": b / med / 1e9 / peak_gbs}
        if vb == 16 and fp64_tflops:
            fl = 4.0 * (ctx.nnz if fmt == helm.HELM_FMT_CSR else 27 * ctx.n)
            out[name]["fp64_tflops_median"] = fl / med / 1e12
            out[name]["fp64_frac_median"] = fl / med / 1e12 / fp64_tflops
        A.free()
    ctx.close()
    return out


def spmm_multi_roofline(helm, torch, peak_gbs, nfreqs=(8, 32)):
    """Shared-mesh multi-frequency product on the 2,203,161-node lattice against one DIA-27 product
    per frequency (matrices pre-assembled), complex128 and complex64, L2 flushed between reps."""
    pr = hi.cabin_problem(200, 112, 96)
    m = pr.mesh
    ctx = helm.Context(m.nx, m.ny, m.nz, m.Lx, m.Ly, m.Lz)
    ctx.set_boundary(torch.from_numpy(pr.beta).cuda(), torch.from_numpy(pr.dir_nodes).cuda(),
                     torch.from_numpy(pr.p_dir).cuda())
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    n = ctx.n

    def timed_med(fn, reps=7):
        for _ in range(2):
            fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            fn()
            e1.record(s)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1000.0)
        return statistics.median(ts)

    out = {}
    for prec, dt, vb, name in ((helm.HELM_C128, torch.complex128, 16, "c128"), (helm.HELM_C64, torch.complex64, 8, "c64")):
        S = helm.helm_assemble_shared(ctx, prec)
        for F in nfreqs:
            freqs = list(np.geomspace(100.0, 400.0, F))
            X = torch.randn(F, n, dtype=dt, device="cuda")
            Y = torch.empty_like(X)
            t_multi = timed_med(lambda: helm.helm_spmv_multi(S, freqs, X, Y))
            # one pre-assembled DIA-27 matrix per frequency (at most 8 resident: reuse them cyclically)
            mats = [helm.helm_assemble(ctx, f, prec, with_rhs=False, fmt=helm.HELM_FMT_DIA27) for f in freqs[:8]]

            def single():
                for f in range(F):
                    helm.helm_spmv(mats[f % len(mats)], X[f], Y[f])
            t_single = timed_med(single, reps=3)
            for A in mats:
                A.free()
            passes = (F + 7) // 8
            b_multi = passes * (27 * n * vb + n) + F * 2 * vb * n
            b_single = F * dia_spmv_bytes(n, vb)
            rec = {"multi_ms_per_freq": t_multi / F * 1e3, "single_ms_per_freq": t_single / F * 1e3,
                   "speedup": t_single / t_multi, "multi_gbs": b_multi / t_multi / 1e9,
                   "multi_frac": b_multi / t_multi / 1e9 / peak_gbs, "single_gbs": b_single / t_single / 1e9,
                   "bytes_per_freq_multi": b_multi / F, "bytes_per_freq_single": b_single / F}
            if F == 8:
                # the frequency-interleaved layout ([n][8]): one 16-byte-vector block per neighbour
                Xi = X.t().contiguous()
                Yi = torch.empty_like(Xi)
                t_il = timed_med(lambda: helm.helm_spmv_multi_interleaved(S, freqs, Xi, Yi))
                rec.update({"interleaved_ms_per_freq": t_il / F * 1e3, "interleaved_speedup_vs_single": t_single / t_il,
                            "interleaved_gbs": b_multi / t_il / 1e9, "interleaved_frac": b_multi / t_il / 1e9 / peak_gbs})
                del Xi, Yi
            out["%s_F%d" % (name, F)] = rec
            del X, Y
        S.close()
    ctx.close()
    return out


# Sweep systems the CPU oracle solves in both of its arms (cpu_baseline and --impl reference):
# every 32nd frequency from 20 Hz up to 150.7 Hz (lattices of 4,875 to 27,508 nodes).
ORACLE_SAMPLE = (0, 32, 64, 96, 128, 160)


def oracle_sample_systems(nfreq=256):
    """(sweep index, frequency) pairs of the oracle sample (the full sweep's indices; for a reduced
    --nfreq sweep the nearest frequencies of that sweep)."""
    freqs = hi.sweep_freqs(256)
    if nfreq >= 256:
        return [(k, float(freqs[k])) for k in ORACLE_SAMPLE]
    sub = hi.sweep_freqs(256)[np.linspace(0, 255, nfreq).round().astype(int)]
    out = []
    for k in ORACLE_SAMPLE:
        j = int(np.argmin(np.abs(sub - freqs[k])))
        out.append((j, float(sub[j])))
    return out


def oracle_solve(f, tol):
    """The oracle's solve of one sweep system: assembly, symmetric Jacobi scaling, FP64
    refinement around FP64 COCG (the benchmark's method with its inner solve in FP64)."""
    from oracle import fem, krylov
    pr = hi.cabin_problem(*hi.sweep_mesh_dims(f))
    A, b = fem.system(pr, f)
    Ah, sc, w = krylov.sym_jacobi(A)
    y, st, _ = krylov.cocg_ir(lambda v: Ah @ v, sc * b, tol=tol, inner_maxit=400000, maxit=400000,
                              stall=STALL, weights=w)
    return sc * y, st


def cpu_oracle_pass(nfreq=256):
    """One pass of the CPU oracle over the fixed sample at the benchmark's target. Returns
    (solutions by sweep index, seconds, cores, description)."""
    import scipy.sparse  # noqa: F401
    sols, t_total = {}, 0.0
    systems = oracle_sample_systems(nfreq)
    for k, f in systems:
        t0 = time.perf_counter()
        x, st = oracle_solve(f, TOL)
        t_total += time.perf_counter() - t0
        sols[k] = x
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    desc = ("oracle (numpy/scipy FP64: assembly, symmetric Jacobi, iterative refinement around COCG, to true "
            "rel-res 1e-10) on %d fixed sweep frequencies, %s Hz (every 32nd up to 150.7 Hz; 4,875-27,508 "
            "nodes); small lattices, so this overstates the oracle's full-sweep rate"
            % (len(systems), ", ".join("%.1f" % f for _, f in systems)))
    return sols, t_total, cores, desc


def oracle_error(head, nfreq=256):
    """Relative L2 error of the benchmark's solutions `head` (sweep index -> complex128 array)
    against the oracle on the fixed sample: against its result at the same target (1e-10) and
    against its result at rel-res 1e-13 (the solution to about cond(A) * 1e-13)."""
    same, tight, per = [], [], []
    for k, f in oracle_sample_systems(nfreq):
        g = head[k]
        x10, _ = oracle_solve(f, TOL)
        x13, _ = oracle_solve(f, 1e-13)
        e10 = float(np.linalg.norm(g - x10) / np.linalg.norm(x10))
        e13 = float(np.linalg.norm(g - x13) / np.linalg.norm(x13))
        same.append(e10)
        tight.append(e13)
        per.append({"freq": round(f, 2), "vs_oracle_1e-10": e10, "vs_oracle_1e-13": e13})
    return {"max_rel_l2_vs_oracle_1e-13": max(tight), "max_rel_l2_vs_oracle_same_target": max(same),
            "systems": per,
            "note": "benchmark results at true rel-res 1e-10; any such iterate lies within cond(A) * 1e-10 of the "
                    "solution, so the two columns also differ by that much"}


def run_gpu(args):
    import torch
    from paper_2112_00087_gb300 import helm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    peaks, peak_kind = measured_peaks()
    peak_gbs = float(peaks["hbm_gbs"])
    # FP64 FMA rate of this GPU, measured by the library's probe kernel (CUDA events): the
    # roofline of the FP64-bound kernels
    fp64_fma = helm.helm_probe_fp64_fma(20000)
    fp64_tflops = 2.0 * fp64_fma / 1e12

    freqs, probs, ctxs, outs = build_sweep(args.nfreq, helm, torch, args.workload)
    nsys = len(ctxs)
    # legs: name -> (options, algorithmic bytes, FP64 flops or None (HBM-bound), kernel, dtype, precision)
    pc = None if args.precond == "none" else args.precond
    pcs = "" if pc is None else ", Jacobi-preconditioned"
    legs = {
        "fp64": (fp64_opts(helm, args.maxit, pc), cocg_fp64_bytes, cocg_fp64_flops, "cocg_persistent<fp64>", "c128",
                 "fp64 COCG" + pcs),
        "c64": (mixed_opts(helm, args.maxit, pc), cocg_mixed_bytes, None, "cocg_persistent<c64 inner>",
                "c64-inner/c128-outer", "mixed: complex64 inner COCG, FP64 refinement" + pcs),
        "dw": (dw_opts(helm, args.maxit, pc), cocg_dw_bytes, None, "cocg_persistent<double-word inner>",
               "dw-inner/c128-outer", "mixed: double-word (2 x FP32, ~48-bit) inner COCG, FP64 refinement" + pcs),
        "bicgstab": (bicgstab_opts(helm, args.maxit, pc), bicgstab_bytes, bicgstab_flops, "bicg_persistent<fp64>", "c128",
                     "fp64 BiCGSTAB" + pcs),
        "tfqmr": (tfqmr_opts(helm, args.maxit, pc), tfqmr_bytes, tfqmr_flops, "tfqmr_persistent<fp64>", "c128",
                  "fp64 TFQMR" + pcs),
    }
    leg = args.solver if args.solver != "cocg" else ("c64" if args.mixed else args.precision)
    bicg = leg in ("bicgstab", "tfqmr")
    main_opts, bytes_fn, flops_fn, kname, dtype, prec_desc = legs[leg]

    def step():
        _, st = helm.helm_solve_batch(ctxs, freqs, main_opts, outs, raise_on_fail=False)
        return st, helm.helm_last_profile()

    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks.start()
    secs, wall, results = timed(step, torch, args.steps, 0, dist)
    clk = clocks.stop()
    secs = max_over_ranks(secs, dist, "cuda")
    stats, prof = results[-1]
    n_ok = sum(1 for s in stats if s["status"] == 0)
    # the timed leg's solutions of the oracle sample, kept before the other legs reuse `outs`
    head = ({k: outs[k].cpu().numpy() for k, _ in oracle_sample_systems(args.nfreq)}
            if args.workload == "sweep256" and rank == 0 and not args.no_cpu else None)
    value = job_value(world, nsys, args.steps, secs)

    # roofline of the dominant kernel (the persistent solve), from the last timed step
    alg = sum(bytes_fn(c.n, c.nnz, s) for c, s in zip(ctxs, stats))
    kern_s = prof["solve_ms"] / 1e3
    achieved = alg / kern_s / 1e9
    launches = sum(p["launches"] for _, p in results)
    traffic = captured_traffic(args)
    hbm = {"bound": "hbm", "achieved": achieved, "peak": peak_gbs, "unit": "GB/s", "frac": achieved / peak_gbs,
           "traffic": traffic, "kernel": kname,
           "algorithmic_bytes": alg, "kernel_ms": prof["solve_ms"], "peak_kind": peak_kind}
    if flops_fn is None:
        roof = hbm
    else:
        # the FP64 step is bound by the FP64 pipe on GB300: report that roofline, HBM beside it
        fl = sum(flops_fn(c.n, s) for c, s in zip(ctxs, stats))
        tf = fl / kern_s / 1e12
        roof = {"bound": "alu", "achieved": tf, "peak": fp64_tflops, "unit": "TFLOP/s",
                "frac": tf / fp64_tflops, "traffic": traffic,
                "kernel": kname, "algorithmic_flops": fl, "kernel_ms": prof["solve_ms"],
                "peak_kind": "measured: FP64 FMA probe kernel (helm_probe_fp64_fma), 2 flops per FMA",
                "hbm": {k: hbm[k] for k in ("achieved", "peak", "unit", "frac", "algorithmic_bytes", "peak_kind")}}
    desc = ("sweep256: %d log-spaced frequencies 20-500 Hz, each on its own wavelength-scaled 2.5x1.4x1.2 m "
            "cabin lattice (24x14x12..148x83x71, %d nodes total), sun-roof Dirichlet pressure + random seat "
            "admittance; assembly + lifting + %s to true rel-res 1e-10 for all systems in one persistent "
            "launch" % (nsys, sum(c.n for c in ctxs), prec_desc)) if args.workload == "sweep256" else args.workload
    out = {"metric": METRIC, "value": value, "unit": "freqs/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": dtype,
           "data": "synthetic",
           "config": {"workload": desc, "precision": prec_desc + " (the other modes, batched, under 'legs')",
                      "solver": args.solver, "precond": args.precond,
                      "l2": "inputs larger than L2 (%.1f GB of matrix values assembled per step)" %
                            (sum(c.n * 27 * 16 for c in ctxs) / 1e9),
                      "parallelism": "replicas" if world > 1 else "1 GPU"},
           "converged": "%d/%d" % (n_ok, nsys),
           "iterations": {"total": int(sum(s["iterations"] for s in stats)),
                          "c64_total": int(sum(s["iterations_c64"] for s in stats)),
                          "max": int(max(s["iterations"] for s in stats)),
                          "relres_max": max(s["relres"] for s in stats)},
           "phases_ms": {"assemble": prof["assemble_ms"], "solve": prof["solve_ms"]},
           "roofline": roof,
           "launch": {"grid_blocks": prof["grid_blocks"], "tiles": prof["ntiles"],
                      "knobs": {k: int(os.environ.get(k, v)) for k, v in autotune_defaults().items()},
                      "chosen_by": "bench.py --autotune on this workload (coordinate descent; the defaults won)"},
           "fp64_peak": {"fma_per_s": fp64_fma, "tflops": fp64_tflops,
                         "how": "helm_probe_fp64_fma: 8 independent FMA chains per thread, 16 blocks of 256 per SM, "
                                "CUDA events"},
           "gpu_launches": int(launches), "clocks": clk}

    if rank == 0 and not args.quick:
        # the other COCG modes, batched, timed once each
        out["legs"] = {}
        cmp_legs = [(name, legs[name][0], legs[name][5]) for name in ("fp64", "c64", "dw") if name != leg]
        if pc is not None:
            cmp_legs.append(("fp64_unpreconditioned", fp64_opts(helm, args.maxit), "fp64 COCG, no preconditioner"))
        for name, o2, desc2 in cmp_legs:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, st2 = helm.helm_solve_batch(ctxs, freqs, o2, outs, raise_on_fail=False)
            torch.cuda.synchronize()
            t2 = time.perf_counter() - t0
            out["legs"][name] = {"freqs_per_s": nsys / t2, "precision": desc2,
                                 "converged": sum(1 for s in st2 if s["status"] == 0),
                                 "iterations_total": int(sum(s["iterations"] for s in st2)),
                                 "inner_iterations": int(sum(s["iterations_c64"] for s in st2)),
                                 "fell_back_to_fp64": int(sum(1 for s in st2 if s["outer"] < 0))}
        if not args.no_sequential:
            # FP64 COCG (same preconditioning as the main leg), one frequency per call (no batching)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for c, f, o in zip(ctxs, freqs, outs):
                helm.helm_solve_batch([c], [f], legs["fp64"][0], [o], raise_on_fail=False)
            torch.cuda.synchronize()
            out["fp64_sequential"] = {"freqs_per_s": nsys / (time.perf_counter() - t0), "precision": legs["fp64"][5]}
        # the metric's comparison: batched main leg against plain FP64 COCG on the same GPU at
        # the same accuracy (true rel-res 1e-10), with and without the main leg's preconditioner
        out["speedups"] = {name: value / leg_["freqs_per_s"] for name, leg_ in
                           (("vs_fp64_same_preconditioner_batched", out["legs"].get("fp64")),
                            ("vs_fp64_unpreconditioned_batched", out["legs"].get("fp64_unpreconditioned")))
                           if leg_ is not None}
        if "fp64_sequential" in out:
            out["speedups"]["vs_fp64_same_preconditioner_sequential"] = value / out["fp64_sequential"]["freqs_per_s"]
        out["spmv"] = spmv_roofline(helm, torch, peak_gbs, fp64_tflops)

        # end to end through host buffers: boundary data in from pinned memory, pressures out
        hb = [(torch.from_numpy(p.beta).pin_memory(), torch.from_numpy(p.dir_nodes).pin_memory(),
               torch.from_numpy(p.p_dir).pin_memory()) for p in probs]
        hout = [torch.empty(c.n, dtype=torch.complex128).pin_memory() for c in ctxs]
        h2d = sum(b.numel() * 16 + d.numel() * 4 + q.numel() * 16 for b, d, q in hb)
        d2h = sum(c.n * 16 for c in ctxs)

        def e2e_step():
            for c, (b, d, q) in zip(ctxs, hb):
                c.set_boundary(b.cuda(non_blocking=True), d.cuda(non_blocking=True), q.cuda(non_blocking=True))
            helm.helm_solve_batch(ctxs, freqs, main_opts, outs, raise_on_fail=False)
            for o, h in zip(outs, hout):
                h.copy_(o, non_blocking=True)
            torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        e2e_s = time.perf_counter() - t0
        out["e2e"] = {"value": nsys / e2e_s, "unit": "freqs/s", "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h)}
    if args.verbose and rank == 0:
        for c, f, st_ in zip(ctxs, freqs, stats):
            print("sys f=%7.2f n=%8d its=%6d c64=%6d outer=%3d restarts=%3d status=%d relres=%.2e" %
                  (f, c.n, st_["iterations"], st_["iterations_c64"], st_["outer"], st_["restarts"], st_["status"],
                   st_["relres"]), file=sys.stderr, flush=True)
    if rank == 0 and not args.no_cpu:
        nf, t_cpu = 0, 0.0
        for _ in range(2):
            sols, t, cores, desc_cpu = cpu_oracle_pass(args.nfreq)
            nf += len(sols)
            t_cpu += t
        out["cpu_baseline"] = {"value": nf / t_cpu, "unit": "freqs/s", "cores": cores, "kind": "oracle",
                               "sample": desc_cpu + "; two passes timed"}
        if head is not None:
            out["oracle_error"] = oracle_error(head, args.nfreq)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_configs(args):
    """Secondary workloads (not the benchmark line): one JSON object with their measurements."""
    import torch
    from paper_2112_00087_gb300 import helm

    def ctx_of(pr):
        m = pr.mesh
        c = helm.Context(m.nx, m.ny, m.nz, m.Lx, m.Ly, m.Lz)
        c.set_boundary(torch.from_numpy(pr.beta).cuda(), torch.from_numpy(pr.dir_nodes).cuda(),
                       torch.from_numpy(pr.p_dir).cuda())
        return c

    def run(c, freqs, o):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p, st = helm.helm_solve(c, freqs, o, raise_on_fail=False)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        pr_ = helm.helm_last_profile()
        return p, st, dt, pr_

    res = {}
    names = args.configs or ["box100", "cabin282k", "cabin2m", "adjoint64", "resonance64", "spmm"]
    want = lambda name: name in names  # noqa: E731
    if want("box100"):
        # box100: GMRES(30) and COCG, FP64, 100 Hz
        c = ctx_of(hi.small_box_problem())
        out = {}
        for name, o in (("gmres30", helm.make_opts("gmres", restart=30, tol=TOL, maxit=20000)),
                        ("cocg", helm.make_opts("cocg", tol=TOL, maxit=20000)),
                        ("bicgstab", helm.make_opts("bicgstab", tol=TOL, maxit=20000))):
            run(c, [100.0], o)
            _, st, dt, pr_ = run(c, [100.0], o)
            out[name] = {"ms": dt * 1e3, "solve_ms": pr_["solve_ms"], "iterations": st[0]["iterations"],
                         "restarts": st[0]["restarts"], "relres": st[0]["relres"], "status": st[0]["status"]}
        res["box100"] = out
    if want("cabin282k"):
        # cabin282k: GMRES(50) + RAS 8x4x4 overlap 2 at 20/100/200 Hz, and COCG for comparison
        c = ctx_of(hi.cabin_problem(100, 56, 48))
        out = {}
        for f in (20.0, 100.0, 200.0):
            o = helm.make_opts("gmres", restart=50, tol=TOL, maxit=5000, precond="ras", ras_parts=(8, 4, 4), ras_overlap=2)
            _, st, dt, pr_ = run(c, [f], o)
            o2 = helm.make_opts("cocg", tol=TOL, maxit=40000, stall_window=STALL)
            _, st2, dt2, pr2 = run(c, [f], o2)
            _, st3, dt3, _ = run(c, [f], helm.make_opts("bicgstab", tol=TOL, maxit=40000))
            o4 = helm.make_opts("gmres", restart=50, tol=TOL, maxit=5000, precond="oras", ras_parts=(8, 4, 4), ras_overlap=2)
            _, st4, dt4, pr4 = run(c, [f], o4)
            out["%g" % f] = {"ras_gmres50": {"ms_total": dt * 1e3, "solve_ms": pr_["solve_ms"],
                                             "iterations": st[0]["iterations"], "relres": st[0]["relres"],
                                             "status": st[0]["status"]},
                             "cocg": {"ms_total": dt2 * 1e3, "iterations": st2[0]["iterations"],
                                      "relres": st2[0]["relres"], "status": st2[0]["status"]},
                             "bicgstab": {"ms_total": dt3 * 1e3, "iterations": st3[0]["iterations"],
                                          "relres": st3[0]["relres"], "status": st3[0]["status"]},
                             "oras_gmres50": {"ms_total": dt4 * 1e3, "solve_ms": pr4["solve_ms"],
                                              "iterations": st4[0]["iterations"], "relres": st4[0]["relres"],
                                              "status": st4[0]["status"]}}
        res["cabin282k"] = out
    if want("cabin2m"):
        # cabin2m: every 8th of the 32 frequencies, FP64 vs mixed, batched per precision
        pr = hi.cabin_problem(200, 112, 96)
        c = ctx_of(pr)
        fr = list(np.geomspace(100.0, 400.0, 32)[::8])
        p64, st64, dt64, _ = run(c, fr, helm.make_opts("cocg", tol=TOL, maxit=60000, stall_window=STALL))
        pmx, stmx, dtmx, _ = run(c, fr, mixed_opts(helm, 60000))
        pdw, stdw, dtdw, _ = run(c, fr, dw_opts(helm, 60000, "jacobi"))
        err_dw = [float((torch.linalg.norm(pdw[k] - p64[k]) / torch.linalg.norm(p64[k])).item()) for k in range(len(fr))]
        err = [float((torch.linalg.norm(pmx[k] - p64[k]) / torch.linalg.norm(p64[k])).item()) for k in range(len(fr))]
        res["cabin2m_sample"] = {"freqs": [float(f) for f in fr], "n": c.n,
                                 "fp64": {"freqs_per_s": len(fr) / dt64, "iterations": [s_["iterations"] for s_ in st64],
                                          "status": [s_["status"] for s_ in st64]},
                                 "mixed": {"freqs_per_s": len(fr) / dtmx, "iterations": [s_["iterations"] for s_ in stmx],
                                           "c64": [s_["iterations_c64"] for s_ in stmx], "outer": [s_["outer"] for s_ in stmx],
                                           "status": [s_["status"] for s_ in stmx]},
                                 "rel_l2_mixed_vs_fp64": err,
                                 "dw_jacobi": {"freqs_per_s": len(fr) / dtdw, "iterations": [s_["iterations"] for s_ in stdw],
                                               "status": [s_["status"] for s_ in stdw], "rel_l2_vs_fp64": err_dw}}
        del p64, pmx, pdw
    if want("schwarz282k"):
        # Schwarz variants on the 282k cabin, GMRES(50), 8x4x4 blocks, overlap 0 and 2, 100 and
        # 200 Hz: plain RAS, one-sided Robin interfaces (i k), two-sided (e^{+-3i pi/4} / h)
        c = ctx_of(hi.cabin_problem(100, 56, 48))
        two = (np.exp(0.75j * np.pi), np.exp(-0.75j * np.pi))
        out = {}
        for f in (100.0, 200.0):
            for ov in (0, 2):
                for name, pc, rb in (("ras", "ras", None), ("oras", "oras", None), ("oras2", "oras2", two)):
                    o = helm.make_opts("gmres", restart=50, tol=TOL, maxit=5000, precond=pc, ras_parts=(8, 4, 4),
                                       ras_overlap=ov, robin=rb)
                    _, st, dt, pr_ = run(c, [f], o)
                    out["%g Hz overlap %d %s" % (f, ov, name)] = {
                        "ms_total": dt * 1e3, "solve_ms": pr_["solve_ms"], "iterations": st[0]["iterations"],
                        "relres": st[0]["relres"], "status": st[0]["status"]}
        res["schwarz282k"] = out
    if want("ras282k"):
        # one GMRES(50) + RAS 8x4x4 (overlap 2) solve of the 282k cabin at 100 Hz (profiling case)
        c = ctx_of(hi.cabin_problem(100, 56, 48))
        o = helm.make_opts("gmres", restart=50, tol=TOL, maxit=5000, precond="ras", ras_parts=(8, 4, 4), ras_overlap=2)
        _, st, dt, pr_ = run(c, [100.0], o)
        res["ras282k"] = {"ms_total": dt * 1e3, "solve_ms": pr_["solve_ms"], "iterations": st[0]["iterations"],
                          "relres": st[0]["relres"], "status": st[0]["status"]}
    if want("cabin2m32"):
        # all 32 frequencies geomspace(100, 400, 32) on the 2,203,161-node cabin: FP64 COCG and the
        # benchmark's main mode, batched per mode; the main mode's error against the FP64 results
        pr = hi.cabin_problem(200, 112, 96)
        c = ctx_of(pr)
        fr = list(np.geomspace(100.0, 400.0, 32))
        out = {"n": c.n, "freqs": [fr[0], fr[-1], len(fr)]}
        p64, st64, dt64, _ = run(c, fr, helm.make_opts("cocg", tol=TOL, maxit=60000, stall_window=STALL))
        out["fp64"] = {"freqs_per_s": len(fr) / dt64, "iterations": [s_["iterations"] for s_ in st64],
                       "converged": sum(1 for s_ in st64 if s_["status"] == 0),
                       "relres_max": max(s_["relres"] for s_ in st64)}
        pdw, stdw, dtdw, _ = run(c, fr, dw_opts(helm, 60000, "jacobi"))
        err = [float((torch.linalg.norm(pdw[k] - p64[k]) / torch.linalg.norm(p64[k])).item()) for k in range(len(fr))]
        out["main_mode"] = {"freqs_per_s": len(fr) / dtdw, "iterations": [s_["iterations"] for s_ in stdw],
                            "converged": sum(1 for s_ in stdw if s_["status"] == 0),
                            "relres_max": max(s_["relres"] for s_ in stdw),
                            "rel_l2_vs_fp64": err, "rel_l2_vs_fp64_max": max(err)}
        out["speedup_main_vs_fp64"] = dt64 / dtdw
        res["cabin2m32"] = out
        del p64, pdw
    if want("adjoint64"):
        # adjoint64: 64 frequencies 20-300 Hz on the 282k cabin, forward + adjoint
        pr = hi.cabin_problem(100, 56, 48)
        c = ctx_of(pr)
        fr = list(np.geomspace(20.0, 300.0, 64))
        o = helm.make_opts("cocg", tol=TOL, maxit=40000, stall_window=STALL)
        p, st, dtf, _ = run(c, fr, o)
        w = torch.from_numpy(hi.listener_weights(pr.mesh)).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J, gb, gd = helm.helm_adjoint_grad(c, fr, o, p, w)
        torch.cuda.synchronize()
        dta = time.perf_counter() - t0
        # the same gradient through the benchmark's main mode (double-word inner COCG, FP64
        # refinement, symmetric Jacobi) for forward and adjoint solves, against the FP64 one
        od = dw_opts(helm, 40000, "jacobi")
        p2, st2, dtf2, _ = run(c, fr, od)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J2, gb2, gd2 = helm.helm_adjoint_grad(c, fr, od, p2, w)
        torch.cuda.synchronize()
        dta2 = time.perf_counter() - t0
        res["adjoint64"] = {"forward_s": dtf, "adjoint_s": dta, "ms_per_frequency_forward_plus_adjoint": (dtf + dta) / 64 * 1e3,
                            "J": J, "converged_forward": sum(1 for s_ in st if s_["status"] == 0),
                            "grad_beta_norm": float(torch.linalg.norm(gb).item()), "n_seat_faces": int((torch.from_numpy(pr.beta) != 0).sum()),
                            "main_mode": {"forward_s": dtf2, "adjoint_s": dta2,
                                          "ms_per_frequency_forward_plus_adjoint": (dtf2 + dta2) / 64 * 1e3,
                                          "J_rel_diff_vs_fp64": abs(J2 - J) / abs(J),
                                          "grad_beta_rel_l2_vs_fp64": float((torch.linalg.norm(gb2 - gb) / torch.linalg.norm(gb)).item()),
                                          "grad_pdir_rel_l2_vs_fp64": float((torch.linalg.norm(gd2 - gd) / torch.linalg.norm(gd)).item()),
                                          "converged_forward": sum(1 for s_ in st2 if s_["status"] == 0)}}
    if want("resonance64"):
        # resonance64: 64 FFT bins 2-33.5 Hz on the 282k cabin, sun-roof pressure shaped by the
        # synthetic PSD (the solve is linear in the Dirichlet data, so each solution is the unit-pattern
        # solution times the bin's complex amplitude); FP64 COCG and the double-word mode, batched
        pr = hi.cabin_problem(100, 56, 48)
        c = ctx_of(pr)
        fr = [float(f) for f in hi.resonance_freqs(64)]
        amp = torch.from_numpy(hi.resonance_spectrum(np.array(fr))).cuda()
        w = torch.from_numpy(hi.listener_weights(pr.mesh)).cuda()
        out = {"n": c.n, "freqs": [fr[0], fr[-1], len(fr)]}
        for name, o in (("fp64", fp64_opts(helm, 40000)), ("dw", dw_opts(helm, 40000)),
                        ("dw_jacobi", dw_opts(helm, 40000, "jacobi"))):
            run(c, fr, o)
            p, st, dt, _ = run(c, fr, o)
            level = [float((abs(amp[k]) ** 2 * (w * (p[k].abs() ** 2)).sum()).item()) for k in range(len(fr))]
            out[name] = {"freqs_per_s": len(fr) / dt, "iterations": int(sum(s_["iterations"] for s_ in st)),
                         "converged": sum(1 for s_ in st if s_["status"] == 0),
                         "listener_peak_hz": fr[int(np.argmax(level))]}
        res["resonance64"] = out
    if want("spmm"):
        peaks, _ = measured_peaks()
        res["spmm_cabin2m"] = spmm_multi_roofline(helm, torch, float(peaks["hbm_gbs"]))
    print(json.dumps({"configs": res}), flush=True)


def autotune_defaults():
    from paper_2112_00087_gb300 import autotune
    return dict(autotune.DEFAULTS)


def run_autotune_kernels(args):
    """Coordinate search of the standalone kernels' knobs (CSR lanes per row, reduction partials)
    on the 2,203,161-node lattice: the objective is the sum of the median times (L2 flushed) of a
    complex128 CSR product, a complex64 CSR product and an unconjugated dot product."""
    import torch
    from paper_2112_00087_gb300 import autotune, helm
    pr = hi.cabin_problem(200, 112, 96)
    m = pr.mesh
    ctx = helm.Context(m.nx, m.ny, m.nz, m.Lx, m.Ly, m.Lz)
    ctx.set_boundary(torch.from_numpy(pr.beta).cuda(), torch.from_numpy(pr.dir_nodes).cuda(),
                     torch.from_numpy(pr.p_dir).cuda())
    A128 = helm.helm_assemble(ctx, 250.0, helm.HELM_C128, with_rhs=False)
    A64 = helm.helm_assemble(ctx, 250.0, helm.HELM_C64, with_rhs=False)
    x128 = torch.randn(ctx.n, dtype=torch.complex128, device="cuda")
    x64 = x128.to(torch.complex64)
    y128, y64 = torch.empty_like(x128), torch.empty_like(x64)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()

    def med(fn, reps=7):
        times = []
        for _ in range(reps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            fn()
            e1.record(s)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        return statistics.median(times)

    def run():
        t = med(lambda: helm.helm_spmv(A128, x128, y128)) + med(lambda: helm.helm_spmv(A64, x64, y64))
        t0 = time.perf_counter()
        for _ in range(5):
            helm.helm_reduce(1, x128, x128)
        return t + (time.perf_counter() - t0) / 5

    run()
    best, log = autotune.autotune(run, space=autotune.KERNEL_SPACE, start=autotune.KERNEL_DEFAULTS)
    print(json.dumps({"autotune_kernels": {"best": best, "trials": [{"config": c, "time_s": t} for c, t in log]}}),
          flush=True)


def run_autotune(args):
    """Coordinate search of the launch-shape knobs for the main leg on the chosen workload."""
    import torch
    from paper_2112_00087_gb300 import autotune, helm
    freqs, probs, ctxs, outs = build_sweep(args.nfreq, helm, torch, args.workload)
    pc = None if args.precond == "none" else args.precond
    opts = {"fp64": fp64_opts, "c64": mixed_opts, "dw": dw_opts}["c64" if args.mixed else args.precision](helm, args.maxit, pc)

    def run():
        helm.helm_solve_batch(ctxs, freqs, opts, outs, raise_on_fail=False)
        return helm.helm_last_profile()["solve_ms"] / 1e3

    run()  # warm-up
    best, log = autotune.autotune(run)
    print(json.dumps({"autotune": {"best": best, "trials": [{"config": c, "solve_s": t} for c, t in log]}}), flush=True)


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_oracle_pass(args.nfreq)
    nf, tt, cores, desc = 0, 0.0, None, None
    for _ in range(args.steps):
        sols, t, cores, desc = cpu_oracle_pass(args.nfreq)
        nf += len(sols)
        tt += t
    value = nf / tt
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "freqs/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": tt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
           "config": {"workload": "sweep256 (the oracle's fixed sample of it each step, see cpu_baseline.sample)"},
           "cpu_baseline": {"value": value, "unit": "freqs/s", "cores": cores, "kind": "oracle", "sample": desc},
           "e2e": {"value": value, "unit": "freqs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nfreq", type=int, default=256, help="frequencies of the sweep (256 = full workload)")
    ap.add_argument("--quick", action="store_true", help="skip the FP64 / SpMV / e2e comparison legs")
    ap.add_argument("--no-sequential", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="sweep256", choices=["sweep256", "cabin2m", "cabin282k"],
                    help="sweep256 is the benchmark; the one-lattice cases serve profiling")
    ap.add_argument("--maxit", type=int, default=45000, help="Krylov step cap per system")
    ap.add_argument("--mixed", action="store_true", help="same as --precision c64")
    ap.add_argument("--precision", default="dw", choices=["fp64", "c64", "dw"],
                    help="COCG mode of the main leg: FP64, or FP64 refinement around a complex64 / double-word "
                         "inner solve")
    ap.add_argument("--solver", default="cocg", choices=["cocg", "bicgstab", "tfqmr"],
                    help="Krylov method of the main leg (BiCGSTAB / TFQMR: FP64)")
    ap.add_argument("--precond", default="jacobi", choices=["none", "jacobi"],
                    help="Jacobi preconditioning (symmetric for COCG, right for BiCGSTAB / TFQMR)")
    ap.add_argument("--verbose", action="store_true", help="per-system statistics on stderr")
    ap.add_argument("--configs", nargs="*", default=None,
                    help="measure the secondary workloads instead (all, or the named ones: box100 cabin282k "
                         "ras282k schwarz282k cabin2m cabin2m32 adjoint64 resonance64 spmm)")
    ap.add_argument("--autotune", action="store_true",
                    help="search the persistent engine's launch-shape knobs on this workload (one line of JSON)")
    ap.add_argument("--autotune-kernels", action="store_true",
                    help="search the standalone SpMV / reduction knobs on the 2.2 M-node lattice (one line of JSON)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes (read + write) of one persistent launch from an ncu capture, if known")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.autotune:
        run_autotune(args)
    elif args.autotune_kernels:
        run_autotune_kernels(args)
    elif args.configs is not None:
        run_configs(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
