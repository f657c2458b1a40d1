"""CPU measurement: GMRES(40)-IR with a complex64 inner solve on sweep lattices (test
infrastructure; the numbers are recorded beside the design choice they decide).

For each system: FP64 refinement around complex64 GMRES(40) (oracle.krylov.gmres_ir) with an
inner reduction of 1e-4 per refinement step, on the symmetric-Jacobi scaled system, target true
rel-res 1e-10; the inner steps and the true residual after every refinement step, against the
steps of the refinement around double-word COCG in FP64 arithmetic (oracle.krylov.cocg_ir) on
the same system. Budget: 5,000 inner steps per refinement step, 3 refinement steps.

Run from the repository root:  python oracle/measure_gmres_ir.py [sweep indices ...]
"""
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def one(k):
    import numpy as np

    import helm_inputs as hi
    from oracle import fem, krylov
    f = float(hi.sweep_freqs(256)[k])
    prob = hi.cabin_problem(*hi.sweep_mesh_dims(f))
    A, b = fem.system(prob, f)
    Ah, s, w = krylov.sym_jacobi(A)
    A32 = Ah.astype(np.complex64)
    t0 = time.time()
    y, st, outer, log = krylov.gmres_ir(lambda v: Ah @ v, lambda v: A32 @ v, s * b, m=40, tol=1e-10,
                                        inner_reduction=1e-4, inner_maxit=5000, max_outer=3, maxit=15000)
    t1 = time.time()
    _, stc, oc = krylov.cocg_ir(lambda v: Ah @ v, s * b, tol=1e-10, inner_maxit=45000, maxit=45000, stall=15000,
                                weights=w)
    x = s * y
    true = float(np.linalg.norm(b - A @ x) / np.linalg.norm(b))
    return {"index": k, "freq": round(f, 1), "n": A.shape[0], "gmres_ir_steps": st.iterations,
            "converged": bool(st.converged), "outer": outer, "true_relres": true,
            "per_refinement": [(int(a), float(r)) for a, r in log], "cocg_ir_steps": stc.iterations,
            "seconds": round(t1 - t0, 1)}


if __name__ == "__main__":
    idx = [int(a) for a in sys.argv[1:]] or [96, 160, 192, 208]
    with mp.get_context("spawn").Pool(len(idx)) as pool:
        for res in pool.imap_unordered(one, idx):
            print(res, flush=True)
