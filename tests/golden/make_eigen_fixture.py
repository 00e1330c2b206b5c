"""Write the FP64 oracle's eigenvalues for the variable-coefficient LOBPCG workload
at a size the oracle finishes on one host core (the benchmark runs the same
recipe at 96^3 on the GPU).

Recipe: 7-point diffusion with log-normal cell coefficients kappa = exp(g),
g ~ N(0, 1) (seed 2106128360 + 3), harmonic-mean faces, on G^3 interior
points; ILUT(1e-4, 10) factors (Saad, Algorithm 10.6); SAIT with 3 series
terms and a row-relative drop of 1e-3 for L and U (Algorithms 1-2); LOBPCG
(Knyazev 2001, the eigensolver of Section 4) for the 16 smallest eigenpairs
from X0 ~ U[0, 1) (seed 2106128360 + 10), residual tolerance 1e-8, and a
second run to 1e-11 as the tight reference.  Only the oracle computes here.

    python tests/golden/make_eigen_fixture.py [G]      # writes eigen_varcoef<G>.json
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402


def main(G: int) -> None:
    A = synth.varcoef3d(G, 1.0, synth.SEED_BASE + 3)
    X0 = synth.uniform(synth.SEED_BASE + 10, (A.n, 16))
    t0 = time.perf_counter()
    L, U = oracle.ilut(A, 1e-4, 10)
    ML, MU = oracle.sait(L, 3, "rowrel", 1e-3), oracle.sait(U, 3, "rowrel", 1e-3)
    out = {"_source": __doc__.strip().splitlines()[0], "grid": G, "n": A.n, "k": 16,
           "factors": "ilut(1e-4, 10)", "m_terms": 3, "drop": "rowrel", "tau": 1e-3}
    for name, tol, maxit in (("tol_1e-8", 1e-8, 2000), ("tol_1e-11", 1e-11, 4000)):
        lam, _, it, rr, st = oracle.lobpcg(A, X0, "sait", ML, MU, tol=tol, maxit=maxit)
        out[name] = {"lambda": [float(x) for x in lam], "iters": it, "max_resid": rr, "status": st}
        print(name, it, rr, st, f"{time.perf_counter() - t0:.1f} s", flush=True)
    with open(os.path.join(HERE, f"eigen_varcoef{G}.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 48)
