"""CPU measurement: step counts of the refined COCG with its inner solve in the residual-product
form (oracle.krylov.cocg_inner_qrec: w = A s, A p carried by q = w + beta q) against the plain
form (oracle.krylov.cocg_inner), on sweep lattices (test infrastructure; the numbers are recorded
beside the design choice they decide).

For each system, on the symmetric-Jacobi scaled system, FP64 throughout, target true rel-res
1e-10: the inner steps of both forms for the system's right-hand side and for three right-hand
sides perturbed at the rounding level (1e-14 of the largest entry, seeds 1-3), i.e. each form's
rounding spread of the step count, and the number of refinement steps each took.

With --dw both inner solves run in double-word arithmetic (oracle.dwfloat.make_inner, forms
"plain" and "qrec"), the arithmetic of the GPU's inner solve.

Run from the repository root:  python oracle/measure_qrec.py [--dw] [sweep indices ...]
"""
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SEEDS = (0, 1, 2, 3)


def perturbed(b, seed):
    import numpy as np
    if seed == 0:
        return b
    rng = np.random.default_rng(seed)
    scale = 1e-14 * np.abs(b).max()
    return b + scale * (rng.standard_normal(b.shape[0]) + 1j * rng.standard_normal(b.shape[0]))


def one(args):
    k, form, seed, use_dw = args
    import helm_inputs as hi
    from oracle import dwfloat, fem, krylov
    f = float(hi.sweep_freqs(256)[k])
    prob = hi.cabin_problem(*hi.sweep_mesh_dims(f))
    A, b = fem.system(prob, f)
    Ah, s, w = krylov.sym_jacobi(A)
    mv = lambda v: Ah @ v  # noqa: E731
    inner = None
    if use_dw:
        m = prob.mesh
        inner = dwfloat.make_inner(dwfloat.StencilMatrix(dwfloat.slots_from_csr(Ah, m.nx, m.ny), m.nx, m.ny), form=form)
    elif form == "qrec":
        inner = lambda s_, t_, im_, ml_, st_, nm_: krylov.cocg_inner_qrec(mv, s_, t_, im_, ml_, st_, nm_)  # noqa: E731
    _, st, outer = krylov.cocg_ir(mv, perturbed(s * b, seed), tol=1e-10, inner_maxit=45000, maxit=45000,
                                  stall=15000, weights=w, inner=inner)
    return k, form, seed, st.iterations, outer, bool(st.converged), A.shape[0], f


def main():
    use_dw = "--dw" in sys.argv[1:]
    ks = [int(a) for a in sys.argv[1:] if a != "--dw"] or list(range(0, 161, 16)) + [176, 192, 208]
    work = [(k, form, sd, use_dw) for k in ks for form in ("plain", "qrec") for sd in SEEDS]
    res = {}
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        for k, form, sd, it, outer, cv, n, f in pool.imap_unordered(one, work):
            res[(k, form, sd)] = (it, outer, cv)
            res[k] = (n, f)
    print("| sweep system | nodes | f (Hz) | plain: steps (b, 3 perturbed) | residual-product form | "
          "form / plain spread |")
    print("|---:|---:|---:|---|---|---|")
    for k in ks:
        n, f = res[k]
        a = [res[(k, "plain", sd)] for sd in SEEDS]
        q = [res[(k, "qrec", sd)] for sd in SEEDS]
        pa, pq = [x[0] for x in a], [x[0] for x in q]
        note = "" if all(x[2] for x in a + q) else " (not all converged)"
        outs = sorted(set(x[1] for x in a + q))
        lo, hi_ = min(pa), max(pa)
        rel = "%+.1f %% .. %+.1f %%" % (100 * (min(pq) / hi_ - 1), 100 * (max(pq) / lo - 1))
        print("| %d | %d | %.1f | %s | %s | %s%s (refinement steps %s) |" % (k, n, f, pa, pq, rel, note, outs))


if __name__ == "__main__":
    main()
