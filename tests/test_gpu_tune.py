"""Autotuners: the product kernel chosen per matrix and the batched tile size.

Bars: every candidate is timed (positive times), the chosen one is the
fastest, and results after tuning still meet the product / solver bars of
the parity tests (FP64 products within 1e-12 (|M||x|)_i of the oracle;
batched solves reach the tolerance on every system).
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


@pytest.fixture(scope="module")
def ctx(sg):
    torch.cuda.set_device(0)
    c = sg.Context()
    yield c
    torch.cuda.synchronize()
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("store", ["f64", "f32"])
def test_mat_autotune_keeps_products_exact(sg, ctx, oracle_lib, store):
    A = synth.convdiff3d(24)
    Lo, _ = oracle_lib.ilu0(A)
    L, _ = sg.sait_ilu0(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
    M = sg.sait_build(ctx, L, True, 3, "rowrel", 1e-3, store=store)
    Mo = oracle_lib.sait(Lo, 3, "rowrel", 1e-3)
    x = synth.uniform(3, A.n, -1.0, 1.0)
    rep = sg.sait_mat_autotune(ctx, M)
    assert rep.ncand >= 5 and 0 <= rep.chosen < rep.ncand
    us = [rep.us[i] for i in range(rep.ncand)]
    assert min(us) > 0.0 and rep.us[rep.chosen] == min(us)
    y = sg.sait_spmv(ctx, M, dev(x)).cpu().numpy()
    ref = oracle_lib.spmv(Mo, x)
    bound = np.abs(Mo.to_scipy()) @ np.abs(x)
    tol = 1e-12 if store == "f64" else 1e-5
    assert np.all(np.abs(y - ref) <= tol * bound + 1e-300)


def test_mat_autotune_ragged_matrix(sg, ctx, oracle_lib):
    """A matrix too ragged for SELL-32: only CSR candidates, and the result is still exact."""
    T = synth.random_triangular(3000, True, 7, max_row=20, long_frac=0.02, long_row=400)
    M = sg.sait_mat_create_csr(ctx, T.n, dev(T.rp), dev(T.ci), dev(T.va))
    rep = sg.sait_mat_autotune(ctx, M)
    assert rep.ncand in (5, 6)
    x = synth.uniform(5, T.n, -1.0, 1.0)
    y = sg.sait_spmv(ctx, M, dev(x)).cpu().numpy()
    bound = np.abs(T.to_scipy()) @ np.abs(x)
    assert np.all(np.abs(y - oracle_lib.spmv(T, x)) <= 1e-12 * bound + 1e-300)


def test_batch_autotune_then_solve(sg, ctx, oracle_lib):
    sides, eps = synth.aniso2d_batch_params(24, 99, smin=8, smax=40)
    systems = [synth.aniso2d(int(s), float(e)) for s, e in zip(sides, eps)]
    n = sum(m.n for m in systems)
    rp = np.zeros(n + 1, np.int64)
    ci, va, r0, e0 = [], [], 0, 0
    for m in systems:
        rp[r0 + 1:r0 + m.n + 1] = m.rp[1:].astype(np.int64) + e0
        ci.append(m.ci.astype(np.int64) + r0)
        va.append(m.va)
        r0 += m.n
        e0 += m.nnz
    A = synth.CSR(n, rp.astype(np.int32), np.concatenate(ci).astype(np.int32), np.concatenate(va))
    ptr = np.concatenate([[0], np.cumsum([m.n for m in systems])]).astype(np.int64)
    b = oracle_lib.spmv(A, synth.uniform(11, n, -1.0, 1.0))
    rep = sg.sait_batch_autotune(ctx, n, dev(ptr))
    assert rep.ncand == 5 and rep.tile_rows[rep.chosen] in (512, 1024, 2048, 4096, 8192)
    assert rep.us[rep.chosen] == min(rep.us[i] for i in range(rep.ncand))
    L, U = sg.sait_ilu0(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
    P = sg.sait_prec_create_sait(ctx, sg.sait_build(ctx, L, True, 3, "rowrel", 1e-3),
                                 sg.sait_build(ctx, U, False, 3, "rowrel", 1e-3))
    Am = sg.sait_mat_create_csr(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
    for tile in (rep.tile_rows[rep.chosen], 32):  # the tuned tile and a tiny one give the same answers
        sg.sait_ctx_set_batch_tile(ctx, tile)
        x, info, st, rr, its = sg.sait_bicgstab_batched(ctx, Am, P, dev(ptr), dev(b), tol=1e-10, maxit=2000)
        assert st == 0 and info.converged == len(systems) and info.max_rel_resid <= 1e-10
        xr = x.cpu().numpy()
        for s in range(len(systems)):
            sl = slice(ptr[s], ptr[s + 1])
            r = b[sl] - oracle_lib.spmv(systems[s], xr[sl])
            assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b[sl]) * 1.0001
    sg.sait_ctx_set_batch_tile(ctx, 2048)
    with pytest.raises(sg.SaitError) as e:
        sg.sait_ctx_set_batch_tile(ctx, 8)
    assert e.value.status == 1


def _tune_problem(sg, ctx, oracle_lib, side=24):
    A = synth.convdiff3d(side)
    b = oracle_lib.spmv(A, synth.uniform(21, A.n, -1.0, 1.0))
    L, U = sg.sait_ilu0(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
    Am = sg.sait_mat_create_csr(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
    return A, b, L, U, Am


CANDS = [{"m_terms": 2, "drop": "rowrel", "tau": 1e-3}, {"m_terms": 3, "drop": "rowrel", "tau": 1e-3},
         {"m_terms": 4, "drop": "rowrel", "tau": 1e-3}, {"m_terms": 4, "drop": "hybrid", "tau": 1e-2, "p": 1},
         {"m_terms": 3, "drop": "pattern", "p": 1}, {"m_terms": 1, "drop": "none"}]


@pytest.mark.parametrize("solver,count_build", [("gmres", True), ("bicgstab", False)])
def test_tune_params_picks_the_fastest_and_solves(sg, ctx, oracle_lib, solver, count_build):
    """Optimal parameters (Section 3): every candidate converges to the
    tolerance, the report's structure counts are the oracle's SAIT sizes, the
    chosen candidate has the smallest runtime by the requested measure, and
    x is a solution (true residual recomputed by the oracle)."""
    A, b, L, U, Am = _tune_problem(sg, ctx, oracle_lib)
    Lo, Uo = oracle_lib.ilu0(A)
    x, rep = sg.sait_tune_params(ctx, Am, L, U, dev(b), CANDS, solver=solver, restart=30, tol=1e-8,
                                 count_build=count_build)
    d = rep.as_dict(CANDS)
    assert rep.ncand == len(CANDS) and all(r["status"] == 0 for r in d["candidates"])
    for c, r in zip(CANDS, d["candidates"]):
        assert r["solve_ms"] > 0.0 and r["build_ms"] > 0.0 and r["rel_resid"] <= 1e-8
        want = (oracle_lib.sait(Lo, c["m_terms"], c["drop"], c.get("tau", 0.0), c.get("p", 0)).nnz
                + oracle_lib.sait(Uo, c["m_terms"], c["drop"], c.get("tau", 0.0), c.get("p", 0)).nnz)
        assert abs(r["nnz"] - want) <= 2  # entries exactly at a drop threshold may fall either way
    cost = [r["solve_ms"] + (r["build_ms"] if count_build else 0.0) for r in d["candidates"]]
    assert rep.chosen == int(np.argmin(cost))
    # more series terms at the same threshold never need more iterations here
    its = [r["iters"] for r in d["candidates"]]
    assert its[2] <= its[1] <= its[0] <= its[5]
    xr = x.cpu().numpy()
    assert np.linalg.norm(b - oracle_lib.spmv(A, xr)) <= 1e-8 * np.linalg.norm(b) * 1.0001


def test_tune_params_nonconvergence(sg, ctx, oracle_lib):
    """Candidates that miss the tolerance within maxit are recorded and
    skipped; when none converges the call reports SAIT_ERR_NOT_CONVERGED."""
    A, b, L, U, Am = _tune_problem(sg, ctx, oracle_lib, side=16)
    cands = [{"m_terms": 1, "drop": "none"}, {"m_terms": 4, "drop": "rowrel", "tau": 1e-4}]
    with pytest.raises(sg.SaitError) as e:  # 5 Arnoldi steps are far from enough (oracle: 65 and 18)
        sg.sait_tune_params(ctx, Am, L, U, dev(b), cands, solver="gmres", restart=10, tol=1e-8, maxit=5)
    assert e.value.status == 6


def test_tune_params_partial_convergence(sg, ctx, oracle_lib):
    A, b, L, U, Am = _tune_problem(sg, ctx, oracle_lib, side=16)
    NOT_CONVERGED = 6
    # oracle GMRES(40) steps to 1e-8: 65 with one term (no preconditioning), 18 with the m=4 pair
    cands = [{"m_terms": 1, "drop": "none"}, {"m_terms": 4, "drop": "rowrel", "tau": 1e-4}]
    x, rep = sg.sait_tune_params(ctx, Am, L, U, dev(b), cands, solver="gmres", restart=40, tol=1e-8, maxit=40)
    assert rep.status[0] == NOT_CONVERGED and rep.status[1] == 0 and rep.chosen == 1
    xr = x.cpu().numpy()
    assert np.linalg.norm(b - oracle_lib.spmv(A, xr)) <= 1e-8 * np.linalg.norm(b) * 1.0001


def test_tune_params_errors(sg, ctx, oracle_lib):
    A, b, L, U, Am = _tune_problem(sg, ctx, oracle_lib, side=8)
    with pytest.raises(ValueError):
        sg.sait_tune_params(ctx, Am, L, U, dev(b), [])
    with pytest.raises(sg.SaitError) as e:  # m_terms = 0 is invalid: the call stops at once
        sg.sait_tune_params(ctx, Am, L, U, dev(b), [{"m_terms": 0, "drop": "none"}])
    assert e.value.status == 1
