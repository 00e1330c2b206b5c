"""Write the FP64 oracle's PCG iteration counts for the level-1 rows of the
paper's 100^3 Laplace experiment (Section 4, Tables runtime_SAIT and
runtime_Jacobi, level-1 ILU columns), for the GPU replica to match.

Recipe: 7-point Laplacian on 100^3 interior points, level-of-fill ILU(1)
factors (Saad, Algorithm 10.5), b ~ U[0, 1) (seed 2106128360), PCG to a
relative residual of 1e-10 with at most 2000 iterations, preconditioned by
SAIT_Thr(tau, 10), SAIT_Pat(p, 10), the exact substitution and k Jacobi
sweeps.  Only the oracle computes here.

    python tests/golden/make_level1_counts.py     # writes oracle_runtime_sait_level1.json
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

MAXIT = 2000


def main() -> None:
    g = json.load(open(os.path.join(HERE, "paper_runtime_sait_level1.json")))
    A = synth.laplace3d(100)
    L, U = oracle.iluk(A, 1)
    b = synth.uniform(synth.SEED_BASE, A.n, 0.0, 1.0)
    tol, m = g["pcg_tol"], g["loop_iterations_m"]

    def pcg(kind, lo, up):
        _, it, rr, st = oracle.pcg(A, b, kind, lo, up, tol=tol, maxit=MAXIT)
        print(kind, it, rr, st, flush=True)
        return {"iters": it, "rel_resid": rr, "status": st}

    out = {"_source": __doc__.strip().splitlines()[0], "maxit": MAXIT, "exact_ilu1": pcg("ilu", L, U),
           "sait_thr": [], "sait_pat": [], "jacobi": {}}
    for r in g["sait_thr"]:
        out["sait_thr"].append({"tau": r["tau"], **pcg("sait", oracle.sait(L, m + 1, "abs", r["tau"]),
                                                       oracle.sait(U, m + 1, "abs", r["tau"]))})
    for r in g["sait_pat"]:
        out["sait_pat"].append({"p": r["p"], **pcg("sait", oracle.sait(L, r["p"] + m + 1, "pattern", 0.0, r["p"]),
                                                   oracle.sait(U, r["p"] + m + 1, "pattern", 0.0, r["p"]))})
    for k in (1, 2, 4):
        out["jacobi"][str(k)] = pcg(f"jacobi{k}", L, U)
    with open(os.path.join(HERE, "oracle_runtime_sait_level1.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
