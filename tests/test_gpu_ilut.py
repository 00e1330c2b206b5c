"""GPU ILUT(tau, lfil) against the oracle's row-by-row Algorithm 10.6 (Saad).

Bar: bit-exact.  Both sides run the same fma chain per entry in the same order
(columns k ascending), the same IEEE division and square root, and the same
tie rule for the lfil largest entries, so L and U must be equal array for
array (row pointers, columns and values).
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


def host(M):
    rp, ci, va = (t.cpu().numpy() for t in M.export())
    return synth.CSR(M.n, rp, ci, va)


def gpu_ilut(sg, ctx, A, tau, lfil):
    L, U = sg.sait_ilut(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va), tau, lfil)
    return host(L), host(U)


def assert_same(G, O):
    assert np.array_equal(G.rp, O.rp)
    assert np.array_equal(G.ci, O.ci)
    assert np.array_equal(G.va, O.va)


CASES = [
    ("convdiff3d_12", lambda: synth.convdiff3d(12), 1e-4, 10),
    ("varcoef3d_16", lambda: synth.varcoef3d(16, 1.0, 5), 1e-4, 10),
    ("varcoef3d_16_tight", lambda: synth.varcoef3d(16, 1.0, 6), 1e-2, 3),
    ("varcoef3d_10_nodrop", lambda: synth.varcoef3d(10, 1.0, 7), 0.0, 32),
    ("aniso2d_40", lambda: synth.aniso2d(40, 0.001), 1e-3, 5),
    ("poisson2d_33_lfil0", lambda: synth.poisson2d(33), 0.0, 0),
]


@pytest.mark.parametrize("name,make,tau,lfil", CASES, ids=[c[0] for c in CASES])
def test_ilut_bit_exact(sg, ctx, oracle_lib, name, make, tau, lfil):
    A = make()
    Lo, Uo = oracle_lib.ilut(A, tau, lfil)
    L, U = gpu_ilut(sg, ctx, A, tau, lfil)
    assert_same(L, Lo)
    assert_same(U, Uo)


def test_ilut_random_nonsymmetric(sg, ctx, oracle_lib):
    """Irregular rows and a ragged number of entries per row."""
    rng = np.random.default_rng(11)
    n = 700
    Ad = np.zeros((n, n))
    for i in range(n):
        cols = rng.choice(n, size=rng.integers(1, 12), replace=False)
        Ad[i, cols] = rng.uniform(-1.0, 1.0, size=cols.size)
        Ad[i, i] = 12.0 + rng.uniform(0.0, 1.0)
    A = synth.from_dense(Ad)
    for tau, lfil in ((1e-3, 6), (1e-2, 12)):
        Lo, Uo = oracle_lib.ilut(A, tau, lfil)
        L, U = gpu_ilut(sg, ctx, A, tau, lfil)
        assert_same(L, Lo)
        assert_same(U, Uo)


def test_ilut_full_size_96(sg, ctx, oracle_lib):
    """The 96^3 log-normal diffusion matrix with ILUT(1e-4, 10), the eigenproblem's factors."""
    A = synth.varcoef3d(96, 1.0, synth.SEED_BASE + 3)
    Lo, Uo = oracle_lib.ilut(A, 1e-4, 10)
    L, U = gpu_ilut(sg, ctx, A, 1e-4, 10)
    assert_same(L, Lo)
    assert_same(U, Uo)


def test_ilut_errors(sg, ctx):
    A = synth.poisson2d(6)
    with pytest.raises(sg.SaitError) as e:
        gpu_ilut(sg, ctx, A, -1.0, 4)
    assert e.value.status == 1
    with pytest.raises(sg.SaitError) as e:
        gpu_ilut(sg, ctx, A, 0.0, 33)
    assert e.value.status == 10
    # a zero pivot: the first row's diagonal is zero
    rows = np.repeat(np.arange(A.n), np.diff(A.rp))
    va = A.va.copy()
    va[(A.ci == rows) & (rows == 0)] = 0.0
    with pytest.raises(sg.SaitError) as e:
        gpu_ilut(sg, ctx, synth.CSR(A.n, A.rp, A.ci, va), 0.0, 4)
    assert e.value.status == 3
    # a row with 300 entries does not fit the working row
    Ad = np.eye(300) * 4.0
    Ad[0, :] = 1.0
    Ad[0, 0] = 400.0
    with pytest.raises(sg.SaitError) as e:
        gpu_ilut(sg, ctx, synth.from_dense(Ad), 0.0, 4)
    assert e.value.status == 10
    # the context still works after the failures
    L, U = gpu_ilut(sg, ctx, A, 0.0, 4)
    assert L.n == A.n


def test_ilut_feeds_sait(sg, ctx, oracle_lib):
    """SAIT of ILUT factors equals the oracle's SAIT of the oracle's factors (same structure and values)."""
    A = synth.varcoef3d(14, 1.0, 9)
    L, U = sg.sait_ilut(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va), 1e-4, 10)
    Lo, Uo = oracle_lib.ilut(A, 1e-4, 10)
    for T, To, lower in ((L, Lo, True), (U, Uo, False)):
        M = host(sg.sait_build(ctx, T, lower, 3, "rowrel", 1e-3))
        Mo = oracle_lib.sait(To, 3, "rowrel", 1e-3)
        assert np.array_equal(M.rp, Mo.rp) and np.array_equal(M.ci, Mo.ci)
        assert np.all(np.abs(M.va - Mo.va) <= 1e-12 * np.abs(Mo.va))


def test_dependency_wait_limit_times_out_and_context_recovers(sg, ctx, oracle_lib):
    """A one-poll limit on the rows' dependency waits: rows whose predecessors
    are still being factored give up, the call returns SAIT_ERR_TIMEOUT (the
    kernel ends, nothing traps or hangs), and the same context then factors the
    matrix bit for bit like the oracle with the default limit."""
    A = synth.varcoef3d(24, 1.0, 5)
    sg.sait_ctx_set_wait_limit(ctx, 1)
    try:
        with pytest.raises(sg.SaitError) as ei:
            gpu_ilut(sg, ctx, A, 1e-4, 10)
        assert ei.value.status == 8  # SAIT_ERR_TIMEOUT
    finally:
        sg.sait_ctx_set_wait_limit(ctx, 0)
    L, U = gpu_ilut(sg, ctx, A, 1e-4, 10)
    Lo, Uo = oracle_lib.ilut(A, 1e-4, 10)
    assert_same(L, Lo)
    assert_same(U, Uo)
