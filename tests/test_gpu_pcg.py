"""GPU PCG and the Jacobi-sweep preconditioner against the FP64 oracle, and
the paper's 100^3 Laplace experiment (Section 4, Tables runtime_SAIT and
runtime_Jacobi) replayed on the GPU.

Bars:
  * PCG: the GPU iterate's true residual, recomputed on the host, is <= tol;
    iteration counts within max(3, 3%) of the oracle's (CG rounding differs
    only in the order of the reductions).
  * Jacobi sweeps: |z - z_ref| <= 1e-12 k max|z_ref| against the oracle, and
    the same bound against the GPU's own undropped SAIT M_k (Section 2: k
    sweeps apply M_k).
  * Paper replica: nnz ratios equal to the printed two decimals; PCG
    iterations within 10% of the printed counts (the paper does not state its
    right-hand side; b ~ U[0,1) here), 3 for the exact ILU row, 5% for the
    Jacobi rows.
"""
import json
import os

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def sg():
    from paper_2106_12836_gb300 import build
    build.build()
    import paper_2106_12836_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(sg):
    torch.cuda.set_device(0)
    c = sg.Context()
    yield c
    torch.cuda.synchronize()
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def mat(sg, ctx, A):
    return sg.sait_mat_create_csr(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))


@pytest.fixture(scope="module")
def c1(oracle_lib):
    A = synth.poisson2d(64)
    b = synth.uniform(synth.SEED_BASE + 1, A.n)
    Lo, Uo = oracle_lib.ilu0(A)
    return A, b, Lo, Uo


@pytest.mark.parametrize("prec", ["none", "ilu", "sait", "jacobi3"])
def test_pcg_parity(sg, ctx, oracle_lib, c1, prec):
    A, b, Lo, Uo = c1
    Ag = mat(sg, ctx, A)
    L, U = sg.sait_ilu0(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
    lo, up = Lo, Uo
    if prec == "sait":
        P = sg.sait_prec_create_sait(ctx, sg.sait_build(ctx, L, True, 11, "abs", 0.02),
                                     sg.sait_build(ctx, U, False, 11, "abs", 0.02))
        lo, up = oracle_lib.sait(Lo, 11, "abs", 0.02), oracle_lib.sait(Uo, 11, "abs", 0.02)
    elif prec == "ilu":
        P = sg.sait_prec_create_ilu(ctx, L, U)
    elif prec == "jacobi3":
        P = sg.sait_prec_create_jacobi(ctx, L, U, 3)
    else:
        P, lo, up = None, None, None
    x, info, st = sg.sait_pcg(ctx, Ag, P, dev(b), tol=1e-10, maxit=5000)
    xo, ito, rro, sto = oracle_lib.pcg(A, b, prec, lo, up, tol=1e-10, maxit=5000)
    rel = np.linalg.norm(b - oracle_lib.spmv(A, x.cpu().numpy())) / np.linalg.norm(b)
    assert st == 0 and sto == 0
    assert rel <= 1e-10 and abs(info.rel_resid - rel) <= 1e-3 * rel
    assert abs(info.iters - ito) <= max(3, 0.03 * ito), (info.iters, ito)


def test_pcg_dense_spd(sg, ctx, oracle_lib):
    """A random SPD matrix stored densely: x matches a LAPACK solve."""
    rng = np.random.default_rng(5)
    Q = rng.standard_normal((60, 60))
    Ad = Q @ Q.T + 60 * np.eye(60)
    A = synth.from_dense(Ad)
    b = rng.standard_normal(60)
    x, info, st = sg.sait_pcg(ctx, mat(sg, ctx, A), None, dev(b), tol=1e-13, maxit=500)
    ref = np.linalg.solve(Ad, b)
    assert st == 0 and np.abs(x.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()


def test_pcg_limits(sg, ctx, oracle_lib, c1):
    A, b, _, _ = c1
    Ag = mat(sg, ctx, A)
    x, info, st = sg.sait_pcg(ctx, Ag, None, dev(b), tol=1e-12, maxit=5, check=False)
    assert st == 6 and info.iters == 5
    rel = np.linalg.norm(b - oracle_lib.spmv(A, x.cpu().numpy())) / np.linalg.norm(b)
    assert abs(info.rel_resid - rel) <= 1e-6 * rel
    x, info, st = sg.sait_pcg(ctx, Ag, None, torch.zeros(A.n, dtype=torch.float64, device="cuda"))
    assert st == 0 and float(x.abs().max()) == 0.0
    x, info, st = sg.sait_pcg(ctx, Ag, None, dev(b), tol=-1.0, check=False)
    assert st == 1


@pytest.mark.parametrize("k", [1, 2, 3, 7])
def test_jacobi_apply_parity(sg, ctx, oracle_lib, k):
    A = synth.convdiff3d(12)
    Lo, Uo = oracle_lib.ilu0(A)
    L, U = sg.sait_ilu0(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
    r = synth.uniform(41 + k, A.n, -1.0, 1.0)
    P = sg.sait_prec_create_jacobi(ctx, L, U, k)
    z = sg.sait_prec_apply(ctx, P, dev(r)).cpu().numpy()
    ref = oracle_lib.jacobi(Uo, oracle_lib.jacobi(Lo, r, k), k)
    bound = 1e-12 * k * np.abs(ref).max()
    assert np.abs(z - ref).max() <= bound
    ML, MU = sg.sait_build(ctx, L, True, k, "none"), sg.sait_build(ctx, U, False, k, "none")
    zs = sg.sait_apply(ctx, ML, MU, dev(r)).cpu().numpy()
    assert np.abs(z - zs).max() <= bound


def test_jacobi_errors(sg, ctx):
    A = synth.poisson2d(8)
    L, U = sg.sait_ilu0(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
    with pytest.raises(sg.SaitError) as e:
        sg.sait_prec_create_jacobi(ctx, L, U, 0)
    assert e.value.status == 1
    va = A.va.copy()
    rows = np.repeat(np.arange(A.n), np.diff(A.rp))
    va[(A.ci == rows) & (rows == 5)] = 0.0
    Z = sg.sait_mat_create_csr(ctx, A.n, dev(A.rp), dev(A.ci), dev(va))
    with pytest.raises(sg.SaitError) as e:
        sg.sait_prec_create_jacobi(ctx, Z, U, 2)
    assert e.value.status == 3


# ---------------------------------------------------------------------------
# Section 4 on the GPU: the 100^3 Laplacian, ILU(0), PCG to 1e-10.
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def laplace100(sg, ctx):
    A = synth.laplace3d(100)
    Ag = mat(sg, ctx, A)
    L, U = sg.sait_ilu0(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
    b = dev(synth.uniform(synth.SEED_BASE, A.n, 0.0, 1.0))
    return A, Ag, L, U, b


def test_paper_table_runtime_sait_on_gpu(sg, ctx, laplace100):
    with open(os.path.join(GOLDEN, "paper_runtime_sait.json")) as f:
        g = json.load(f)
    A, Ag, L, U, b = laplace100
    assert L.nnz == 3_970_000 and U.nnz == 3_970_000
    tol, m = g["pcg_tol"], g["loop_iterations_m"]
    _, info, st = sg.sait_pcg(ctx, Ag, sg.sait_prec_create_ilu(ctx, L, U), b, tol=tol)
    assert st == 0 and abs(info.iters - g["exact_ilu0_pcg_iters"]) <= 3
    exact = info.iters
    rows = [("abs", r["tau"], 0, m + 1, r) for r in g["sait_thr"]] + \
           [("pattern", 0.0, r["p"], r["p"] + m + 1, r) for r in g["sait_pat"]]
    for drop, tau, p, terms, row in rows:
        ML = sg.sait_build(ctx, L, True, terms, drop, tau, p)
        MU = sg.sait_build(ctx, U, False, terms, drop, tau, p)
        assert round(MU.nnz / U.nnz, 2) == row["ratio"], (drop, tau, p, MU.nnz)
        if drop == "abs":
            assert round(ML.nnz / L.nnz, 2) == row["ratio"], (drop, tau, ML.nnz)
        _, info, st = sg.sait_pcg(ctx, Ag, sg.sait_prec_create_sait(ctx, ML, MU), b, tol=tol)
        assert st == 0 and info.rel_resid <= tol
        assert abs(info.iters - row["pcg_iters"]) <= 0.1 * row["pcg_iters"], (drop, tau, p, info.iters)
        assert info.iters > exact


def test_paper_table_runtime_jacobi_on_gpu(sg, ctx, laplace100):
    with open(os.path.join(GOLDEN, "paper_runtime_jacobi.json")) as f:
        g = json.load(f)
    A, Ag, L, U, b = laplace100
    for k in (1, 2, 3, 4, 10):
        _, info, st = sg.sait_pcg(ctx, Ag, sg.sait_prec_create_jacobi(ctx, L, U, k), b, tol=g["pcg_tol"])
        want = g["level0_pcg_iters"][str(k)]
        assert st == 0 and abs(info.iters - want) <= 0.05 * want, (k, info.iters)


# ---------------------------------------------------------------------------
# The same experiment with level-1 ILU factors (the right-hand columns of
# Tables runtime_SAIT and runtime_Jacobi).  The nnz ratios and the exact and
# Jacobi rows match the paper; the SAIT rows' PCG counts are checked against
# the FP64 oracle's counts (tests/golden/make_level1_counts.py), which lie
# 6-26% above the printed ones (SAIT_Thr(0.02,10) stalls at 1.5e-10 after
# 2000 iterations: PCG with the nonsymmetric M_U M_L has no guarantee).
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def laplace100_level1(sg, ctx, oracle_lib):
    A = synth.laplace3d(100)
    Ag = mat(sg, ctx, A)
    L, U = sg.sait_iluk(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va), 1)
    b = dev(synth.uniform(synth.SEED_BASE, A.n, 0.0, 1.0))
    return A, Ag, L, U, b


def test_paper_table_runtime_sait_level1_on_gpu(sg, ctx, oracle_lib, laplace100_level1):
    with open(os.path.join(GOLDEN, "paper_runtime_sait_level1.json")) as f:
        g = json.load(f)
    path = os.path.join(GOLDEN, "oracle_runtime_sait_level1.json")
    if not os.path.exists(path):
        pytest.skip("oracle level-1 counts not generated")
    with open(path) as f:
        o = json.load(f)
    A, Ag, L, U, b = laplace100_level1
    assert L.nnz == U.nnz == 6_910_300
    tol, m, maxit = g["pcg_tol"], g["loop_iterations_m"], o["maxit"]
    _, info, st = sg.sait_pcg(ctx, Ag, sg.sait_prec_create_ilu(ctx, L, U), b, tol=tol, maxit=maxit)
    assert st == 0 and abs(info.iters - g["exact_ilu1_pcg_iters"]) <= 3
    assert abs(info.iters - o["exact_ilu1"]["iters"]) <= 3
    rows = [("abs", r["tau"], 0, m + 1, r, orow) for r, orow in zip(g["sait_thr"], o["sait_thr"])] + \
           [("pattern", 0.0, r["p"], r["p"] + m + 1, r, orow) for r, orow in zip(g["sait_pat"], o["sait_pat"])]
    for drop, tau, p, terms, row, orow in rows:
        ML = sg.sait_build(ctx, L, True, terms, drop, tau, p)
        MU = sg.sait_build(ctx, U, False, terms, drop, tau, p)
        # SAIT_Thr ratios on L (rounding splits threshold ties between L and U = D L^T
        # differently: 5.174 on L, 5.180 on U for tau = 0.01), SAIT_Pat on U
        M, T = (ML, L) if drop == "abs" else (MU, U)
        assert round(M.nnz / T.nnz, 2) == row["ratio"], (drop, tau, p, M.nnz)
        _, info, st = sg.sait_pcg(ctx, Ag, sg.sait_prec_create_sait(ctx, ML, MU), b, tol=tol, maxit=maxit,
                                  check=False)
        if orow["status"] == 0:
            assert st == 0 and info.rel_resid <= tol
            assert abs(info.iters - orow["iters"]) <= max(3, 0.03 * orow["iters"]), (drop, tau, p, info.iters)
        else:  # the oracle stalls near the tolerance within maxit: so does the GPU
            assert st != 0 or info.iters >= 0.9 * maxit, (drop, tau, p, info.iters)


def test_paper_table_runtime_jacobi_level1_on_gpu(sg, ctx, laplace100_level1):
    with open(os.path.join(GOLDEN, "paper_runtime_sait_level1.json")) as f:
        g = json.load(f)
    A, Ag, L, U, b = laplace100_level1
    for k in (1, 2, 4):
        _, info, st = sg.sait_pcg(ctx, Ag, sg.sait_prec_create_jacobi(ctx, L, U, k), b, tol=g["pcg_tol"])
        want = g["jacobi_level1_pcg_iters"][str(k)]
        assert st == 0 and abs(info.iters - want) <= 0.05 * want, (k, info.iters)
