"""GPU LOBPCG with the SAIT block preconditioner against closed forms, dense
eigenvalues and the oracle's LOBPCG.

Eigenvalues converge quadratically in the residual, so with residual
tolerance 1e-8 the eigenvalues agree with the exact ones to ~1e-12 relative;
the tests use 1e-10.  Reduced-precision storage of M only changes the
preconditioner, not the eigenvalues.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    from paper_2106_12836_gb300 import build
    build.build()
    import paper_2106_12836_gb300 as m
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def laplace_eigs(N, k):
    j = np.arange(1, N + 1)
    l1 = 4 * np.sin(j * np.pi / (2 * (N + 1))) ** 2
    return np.sort((l1[:, None, None] + l1[None, :, None] + l1[None, None, :]).ravel())[:k]


def setup(sg, ctx, A, store):
    L, U = sg.sait_ilu0(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
    P = sg.sait_prec_create_sait(ctx, sg.sait_build(ctx, L, True, 3, "rowrel", 1e-3, store=store),
                                 sg.sait_build(ctx, U, False, 3, "rowrel", 1e-3, store=store))
    Am = sg.sait_mat_create_csr(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
    return Am, P


@pytest.mark.parametrize("store", ["f64", "f32", "bf16"])
def test_lobpcg_laplace_closed_form(sg, store):
    N, k = 12, 16
    A = synth.laplace3d(N)
    with sg.Context() as ctx:
        Am, P = setup(sg, ctx, A, store)
        lam, X, info, st = sg.sait_lobpcg(ctx, Am, P, dev(synth.uniform(5, (A.n, k))), tol=1e-8, maxit=500)
        torch.cuda.synchronize()
    lam, X = lam.cpu().numpy(), X.cpu().numpy()
    assert st == 0 and info.rel_resid <= 1e-8
    assert np.abs(lam - laplace_eigs(N, k)).max() <= 1e-10 * lam.max()
    R = A.to_scipy() @ X - X * lam
    assert np.all(np.linalg.norm(R, axis=0) <= 1e-8 * lam * 1.001)
    assert np.abs(X.T @ X - np.eye(k)).max() <= 1e-9


def test_lobpcg_variable_coefficients(sg, oracle_lib):
    A = synth.varcoef3d(11, 1.0, 8)
    k = 8
    X0 = synth.uniform(6, (A.n, k))
    with sg.Context() as ctx:
        Am, P = setup(sg, ctx, A, "f32")
        lam, X, info, st = sg.sait_lobpcg(ctx, Am, P, dev(X0), tol=1e-8, maxit=800)
        _, _, info0, _ = sg.sait_lobpcg(ctx, Am, None, dev(X0), tol=1e-8, maxit=2000)
        torch.cuda.synchronize()
    lam = lam.cpu().numpy()
    ref = np.linalg.eigvalsh(A.to_dense())[:k]
    assert st == 0
    assert np.abs(lam - ref).max() <= 1e-10 * ref.max()
    Lo, Uo = oracle_lib.ilu0(A)
    lo, _, it, rr, sto = oracle_lib.lobpcg(A, X0, "sait", oracle_lib.sait(Lo, 3, "rowrel", 1e-3),
                                           oracle_lib.sait(Uo, 3, "rowrel", 1e-3), tol=1e-8, maxit=800)
    assert sto == 0 and np.abs(lam - lo).max() <= 1e-10 * ref.max()
    assert info.iters < info0.iters          # the SAIT preconditioner pays off
    assert abs(info.iters - it) <= max(3, 0.25 * it), (info.iters, it)


@pytest.mark.parametrize("store", ["f64", "f32", "bf16"])
def test_lobpcg_matches_oracle_fixture(sg, store):
    """The variable-coefficient eigenproblem of the benchmark (log-normal kappa,
    ILUT(1e-4, 10) factors, SAIT with 3 terms and a row-relative drop of 1e-3,
    16 smallest eigenpairs from the same X0) at 32^3, against the FP64 oracle's
    eigenvalues stored by tests/golden/make_eigen_fixture.py: with the factors
    stored in FP64, FP32 or BF16 the eigenvalues agree with the oracle's
    tight (1e-11) run to 1e-10 relative."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "eigen_varcoef32.json")) as f:
        fx = json.load(f)
    A = synth.varcoef3d(fx["grid"], 1.0, synth.SEED_BASE + 3)
    X0 = synth.uniform(synth.SEED_BASE + 10, (A.n, fx["k"]))
    with sg.Context() as ctx:
        L, U = sg.sait_ilut(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va), 1e-4, 10)
        P = sg.sait_prec_create_sait(ctx, sg.sait_build(ctx, L, True, 3, "rowrel", 1e-3, store=store),
                                     sg.sait_build(ctx, U, False, 3, "rowrel", 1e-3, store=store))
        Am = sg.sait_mat_create_csr(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
        lam, X, info, st = sg.sait_lobpcg(ctx, Am, P, dev(X0), tol=1e-8, maxit=1000)
        torch.cuda.synchronize()
    lam = lam.cpu().numpy()
    ref = np.array(fx["tol_1e-11"]["lambda"])
    assert st == 0 and info.rel_resid <= 1e-8
    assert np.abs(lam - ref).max() <= 1e-10 * ref.max(), np.abs(lam - ref).max() / ref.max()
    # the oracle's own 1e-8 run agrees with its tight run at the same level
    assert np.abs(np.array(fx["tol_1e-8"]["lambda"]) - ref).max() <= 1e-10 * ref.max()


def test_lobpcg_rejects_bad_sizes(sg):
    A = synth.laplace3d(3)
    with sg.Context() as ctx:
        Am = sg.sait_mat_create_csr(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
        with pytest.raises(sg.SaitError) as e:
            sg.sait_lobpcg(ctx, Am, None, dev(synth.uniform(1, (A.n, 10))))
        assert e.value.status == 1
