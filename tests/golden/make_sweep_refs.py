"""Writes tests/golden/sweep_refs.json: the oracle's reference results for the large systems of
the 256-frequency sweep (every 16th from index 176, plus 248 and the last, 255), which the
oracle takes minutes to hours to solve, so the GPU tests read them instead of recomputing them.

Per system (symmetric Jacobi scaling, oracle.krylov.cocg_ir -- the refinement the
mixed-precision GPU solves run):
  * the inner step counts at the sweep's target (true relative residual 1e-10) for the system's
    right-hand side and for three right-hand sides perturbed at the rounding level (1e-14 of the
    largest entry, seeds 1-3), i.e. the rounding spread of the step count: with the inner solve
    in FP64 ("iterations") and in double-word arithmetic (oracle.dwfloat, "iterations_dw"), the
    arithmetic of the GPU's inner solve, which decides its step count; and in double-word
    arithmetic in the residual-product form of the inner COCG (dwfloat.make_inner(form="qrec"),
    "iterations_dw_qrec"), the iteration of a GPU form with one synchronisation point fewer;
  * the solution at relative residual 1e-13 (FP64 inner solve) sampled at 128 seeded node
    indices, its 2-norm and the relative residual reached.

Only oracle/ and the seeded input generators are used. Run from the repository root:
    python tests/golden/make_sweep_refs.py [--jobs 8] [--kinds value fp64 dw dwq] [--systems ...]
(results of the kinds run are merged into an existing file; the FP64 kinds take about an hour on
8 cores, the double-word counts about three; the 901,152-node system dominates both).
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SYSTEMS = (176, 192, 208, 224, 240, 248, 255)
TOL = 1e-10
VALUE_TOL = 1e-13
STALL = 15000
MAXIT = 45000
NSAMPLE = 128
PERTURB_SEEDS = (1, 2, 3)


def sample_nodes(k, n):
    """Seeded sample of node indices of sweep system k (shared with the tests)."""
    import numpy as np
    return np.sort(np.random.default_rng(1000 + k).choice(n, NSAMPLE, replace=False))


def perturbed_rhs(b, seed):
    import numpy as np
    rng = np.random.default_rng(seed)
    e = (rng.standard_normal(len(b)) + 1j * rng.standard_normal(len(b))) * 1e-14 * np.abs(b).max()
    return b + e


def job(args):
    k, what = args
    import numpy as np

    import helm_inputs as hi
    from oracle import dwfloat, fem, krylov

    f = float(hi.sweep_freqs(256)[k])
    prob = hi.cabin_problem(*hi.sweep_mesh_dims(f))
    A, b = fem.system(prob, f)
    Ah, s, w = krylov.sym_jacobi(A)
    mv = lambda v: Ah @ v  # noqa: E731
    t0 = time.time()
    if what == "value":
        y, st, outer = krylov.cocg_ir(mv, s * b, tol=VALUE_TOL, inner_maxit=MAXIT, maxit=MAXIT, stall=STALL,
                                      weights=w)
        x = s * y
        idx = sample_nodes(k, len(b))
        rel = float(np.linalg.norm(b - A @ x) / np.linalg.norm(b))
        return k, what, {"relres": rel, "converged": bool(st.converged), "outer": int(outer),
                         "iterations": int(st.iterations), "norm": float(np.linalg.norm(x)),
                         "idx": [int(i) for i in idx], "re": [float(v) for v in x[idx].real],
                         "im": [float(v) for v in x[idx].imag], "seconds": time.time() - t0}
    kind, seed = what
    inner = None
    if kind in ("dw", "dwq"):
        m = prob.mesh
        inner = dwfloat.make_inner(dwfloat.StencilMatrix(dwfloat.slots_from_csr(Ah, m.nx, m.ny), m.nx, m.ny),
                                   form="qrec" if kind == "dwq" else "plain")
    rhs = s * b if seed == 0 else perturbed_rhs(s * b, seed)
    _, st, outer = krylov.cocg_ir(mv, rhs, tol=TOL, inner_maxit=MAXIT, maxit=MAXIT, stall=STALL, weights=w,
                                  inner=inner)
    return k, what, {"iterations": int(st.iterations), "outer": int(outer), "converged": bool(st.converged),
                     "seconds": time.time() - t0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count())
    ap.add_argument("--systems", type=int, nargs="*", default=list(SYSTEMS))
    ap.add_argument("--kinds", nargs="*", default=["value", "fp64", "dw"], choices=["value", "fp64", "dw", "dwq"])
    args = ap.parse_args()
    import helm_inputs as hi
    path = os.path.join(HERE, "sweep_refs.json")
    out = {"tol": TOL, "value_tol": VALUE_TOL, "stall": STALL, "maxit": MAXIT, "nsample": NSAMPLE,
           "perturb_seeds": list(PERTURB_SEEDS),
           "solver": "oracle.krylov.cocg_ir on the symmetric-Jacobi scaled system; inner solve in FP64 "
                     "(iterations, value) or in double-word arithmetic, oracle.dwfloat (iterations_dw; "
                     "residual-product form: iterations_dw_qrec)",
           "systems": {}}
    if os.path.exists(path):
        old = json.load(open(path))
        out["systems"] = old.get("systems", {})
    work = []
    for k in sorted(args.systems, reverse=True):
        if "value" in args.kinds:
            work.append((k, "value"))
        for kind in ("fp64", "dw", "dwq"):
            if kind in args.kinds:
                work += [(k, (kind, sd)) for sd in (0,) + PERTURB_SEEDS]
    for k in args.systems:
        f = float(hi.sweep_freqs(256)[k])
        dims = hi.sweep_mesh_dims(f)
        rec = out["systems"].setdefault(str(k), {})
        rec.update({"freq": f, "dims": list(dims), "n": int((dims[0] + 1) * (dims[1] + 1) * (dims[2] + 1))})
    counts = {}
    with mp.get_context("spawn").Pool(args.jobs) as pool:
        for k, what, res in pool.imap_unordered(job, work):
            if what == "value":
                out["systems"][str(k)]["value"] = res
            else:
                counts.setdefault((k, what[0]), {})[what[1]] = res
            print(k, what, {a: b for a, b in res.items() if a not in ("idx", "re", "im")}, flush=True)
    for (k, kind), c in counts.items():
        rec = out["systems"][str(k)]
        sfx = {"fp64": "", "dw": "_dw", "dwq": "_dw_qrec"}[kind]
        rec["iterations" + sfx] = [c[sd]["iterations"] for sd in (0,) + PERTURB_SEEDS]
        rec["outer" + sfx] = [c[sd]["outer"] for sd in (0,) + PERTURB_SEEDS]
        rec["converged" + sfx] = all(c[sd]["converged"] for sd in (0,) + PERTURB_SEEDS)
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
