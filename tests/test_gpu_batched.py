"""Batched solves: many independent systems (block diagonal) and many right-hand sides.

Each system / column is checked on its own: the true FP64 relative residual
of the GPU solution, recomputed on the host, is <= tol; with FP64 SAIT storage
the per-system iteration counts are within 10% (or 2) of the oracle's
BiCGSTAB run on that system alone with the oracle's SAIT factors.
"""
import numpy as np
import pytest
import scipy.sparse as sp
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


def block_diag(mats):
    B = sp.block_diag([m.to_scipy() for m in mats], format="csr")
    B.sort_indices()
    return synth.CSR(B.shape[0], B.indptr.astype(np.int32), B.indices.astype(np.int32), B.data.copy())


@pytest.mark.parametrize("store", ["f64", "f32", "f32x64"])
def test_batched_independent_systems(sg, oracle_lib, store):
    sides, eps = synth.aniso2d_batch_params(12, synth.SEED_BASE + 40, smin=5, smax=40)
    systems = [synth.aniso2d(int(s), float(e)) for s, e in zip(sides, eps)]
    A = block_diag(systems)
    ptr = np.concatenate([[0], np.cumsum([m.n for m in systems])]).astype(np.int64)
    xt = synth.uniform(7, A.n)
    b = A.to_scipy() @ xt
    b[ptr[3]:ptr[4]] = 0.0                                  # one system with b = 0
    with sg.Context() as ctx:
        L, U = sg.sait_ilu0(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
        P = sg.sait_prec_create_sait(ctx, sg.sait_build(ctx, L, True, 3, "rowrel", 1e-3, store=store),
                                     sg.sait_build(ctx, U, False, 3, "rowrel", 1e-3, store=store))
        Am = sg.sait_mat_create_csr(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
        x, info, st, rr, its = sg.sait_bicgstab_batched(ctx, Am, P, dev(ptr), dev(b), tol=1e-8, maxit=2000)
        torch.cuda.synchronize()
    x, rr, its = x.cpu().numpy(), rr.cpu().numpy(), its.cpu().numpy()
    assert st == 0 and info.converged == len(systems)
    # the iterations loop on the device: one graph launch per restart round
    assert info.device_loop == 1 and 1 <= info.graph_launches <= 4, info.as_dict()
    assert info.graph_replays % 8 == 0 and info.graph_replays >= int(its.max())
    for s, M in enumerate(systems):
        sl = slice(ptr[s], ptr[s + 1])
        bs = b[sl]
        if not bs.any():
            continue
        rel = np.linalg.norm(bs - M.to_scipy() @ x[sl]) / np.linalg.norm(bs)
        assert rel <= 1e-8 and abs(rel - rr[s]) <= 1e-6 * max(rel, 1e-300), (s, rel, rr[s])
        if store == "f64":
            Lo, Uo = oracle_lib.ilu0(M)
            _, ito, _, sto = oracle_lib.bicgstab(M, bs, "sait", oracle_lib.sait(Lo, 3, "rowrel", 1e-3),
                                                 oracle_lib.sait(Uo, 3, "rowrel", 1e-3), tol=1e-8)
            assert sto == 0 and abs(int(its[s]) - ito) <= max(2, 0.1 * ito), (s, its[s], ito)


@pytest.mark.parametrize("k", [8, 64])
def test_multi_rhs(sg, oracle_lib, k):
    A = synth.laplace3d(14)
    Xt = synth.uniform(9, (A.n, k))
    B = np.ascontiguousarray((A.to_scipy() @ Xt))
    with sg.Context() as ctx:
        L, U = sg.sait_ilu0(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
        P = sg.sait_prec_create_sait(ctx, sg.sait_build(ctx, L, True, 3, "rowrel", 1e-3),
                                     sg.sait_build(ctx, U, False, 3, "rowrel", 1e-3))
        Am = sg.sait_mat_create_csr(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
        X, info, st, rr, its = sg.sait_bicgstab_multi(ctx, Am, P, dev(B), tol=1e-8, maxit=2000)
        torch.cuda.synchronize()
    X, its = X.cpu().numpy(), its.cpu().numpy()
    assert st == 0 and info.converged == k
    assert info.device_loop == 1 and 1 <= info.graph_launches <= 4, info.as_dict()
    Lo, Uo = oracle_lib.ilu0(A)
    MLo, MUo = oracle_lib.sait(Lo, 3, "rowrel", 1e-3), oracle_lib.sait(Uo, 3, "rowrel", 1e-3)
    for c in range(0, k, max(1, k // 8)):
        rel = np.linalg.norm(B[:, c] - A.to_scipy() @ X[:, c]) / np.linalg.norm(B[:, c])
        assert rel <= 1e-8, (c, rel)
        _, ito, _, sto = oracle_lib.bicgstab(A, B[:, c], "sait", MLo, MUo, tol=1e-8)
        assert abs(int(its[c]) - ito) <= max(2, 0.1 * ito), (c, its[c], ito)


@pytest.mark.parametrize("maxit", [5, 16])
def test_batched_device_loop_stops_at_maxit(sg, maxit):
    """Too few iterations to converge: the device loop ends after ceil(maxit / 8)
    passes of its 8-iteration body, every system stops at maxit, none restarts,
    and the solve reports not converged."""
    sides, eps = synth.aniso2d_batch_params(6, synth.SEED_BASE + 41, smin=30, smax=40)
    systems = [synth.aniso2d(int(s), float(e)) for s, e in zip(sides, eps)]
    A = block_diag(systems)
    ptr = np.concatenate([[0], np.cumsum([m.n for m in systems])]).astype(np.int64)
    b = A.to_scipy() @ synth.uniform(8, A.n)
    with sg.Context() as ctx:
        Am = sg.sait_mat_create_csr(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
        x, info, st, rr, its = sg.sait_bicgstab_batched(ctx, Am, None, dev(ptr), dev(b), tol=1e-14, maxit=maxit,
                                                        check=False)
        torch.cuda.synchronize()
    its = its.cpu().numpy()
    assert st == 6 and info.converged == 0  # SAIT_ERR_NOT_CONVERGED
    assert info.device_loop == 1 and info.graph_launches == 1
    assert info.graph_replays == 8 * ((maxit + 7) // 8)
    assert (its == maxit).all(), its


def test_device_loop_and_host_replays_agree(sg):
    """The WHILE-node loop and the host-replayed graph run the same kernels in
    the same order: the iterates and iteration counts are identical, and only
    the number of graph launches differs."""
    sides, eps = synth.aniso2d_batch_params(10, synth.SEED_BASE + 42, smin=5, smax=40)
    systems = [synth.aniso2d(int(s), float(e)) for s, e in zip(sides, eps)]
    A = block_diag(systems)
    ptr = np.concatenate([[0], np.cumsum([m.n for m in systems])]).astype(np.int64)
    b = A.to_scipy() @ synth.uniform(11, A.n)
    out = {}
    with sg.Context() as ctx:
        L, U = sg.sait_ilu0(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
        P = sg.sait_prec_create_sait(ctx, sg.sait_build(ctx, L, True, 3, "rowrel", 1e-3),
                                     sg.sait_build(ctx, U, False, 3, "rowrel", 1e-3))
        Am = sg.sait_mat_create_csr(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
        B = dev(np.ascontiguousarray(np.stack([b, 2.0 * b + 1.0], axis=1)))
        for on in (True, False):
            sg.sait_ctx_set_device_loop(ctx, on)
            x, info, st, rr, its = sg.sait_bicgstab_batched(ctx, Am, P, dev(ptr), dev(b), tol=1e-8, maxit=2000)
            X, minfo, mst, mrr, mits = sg.sait_bicgstab_multi(ctx, Am, P, B, tol=1e-8, maxit=2000)
            torch.cuda.synchronize()
            out[on] = (x.cpu().numpy(), its.cpu().numpy(), info, X.cpu().numpy(), mits.cpu().numpy(), minfo)
    (x1, i1, f1, X1, mi1, g1), (x0, i0, f0, X0, mi0, g0) = out[True], out[False]
    assert np.array_equal(x1, x0) and np.array_equal(i1, i0)
    assert np.array_equal(X1, X0) and np.array_equal(mi1, mi0)
    assert f1.device_loop == 1 and f0.device_loop == 0 and g1.device_loop == 1 and g0.device_loop == 0
    assert f1.graph_replays == f0.graph_replays and g1.graph_replays == g0.graph_replays
    assert f0.graph_launches == f0.graph_replays // 8 and f1.graph_launches < f0.graph_launches
