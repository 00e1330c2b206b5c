"""Block products: sait_spmm and sait_apply_multi against the oracle, column by column.

Tolerance as for single products: |Y - Y_ref| <= tol * (|M| |X|) entrywise
(1e-12 FP64, 1e-5 FP32, 1e-2 BF16 storage).
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 1e-2, "f32x64": 1e-6, "bf16x64": 1e-2}


@pytest.fixture(scope="module")
def sg():
    from paper_2106_12836_gb300 import build
    build.build()
    import paper_2106_12836_gb300 as m
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("k", [1, 3, 16, 40, 64, 70])
def test_spmm_matches_columns(sg, oracle_lib, k):
    T = synth.random_triangular(1500, True, k, max_row=40, empty_frac=0.1, long_frac=0.02, long_row=600)
    X = synth.uniform(k, (T.n, k))
    with sg.Context() as ctx:
        M = sg.sait_mat_create_csr(ctx, T.n, dev(T.rp), dev(T.ci), dev(T.va))
        Xp = torch.zeros((T.n, k + 5), dtype=torch.float64, device="cuda")   # ld > k
        Xp[:, :k] = dev(X)
        Y = sg.sait_spmm(ctx, M, Xp[:, :k]).cpu().numpy()
        torch.cuda.synchronize()
    absT = synth.CSR(T.n, T.rp, T.ci, np.abs(T.va))
    for t in range(k):
        ref = oracle_lib.spmv(T, X[:, t])
        bound = oracle_lib.spmv(absT, np.abs(X[:, t]))
        assert np.all(np.abs(Y[:, t] - ref) <= 1e-12 * bound), t


@pytest.mark.parametrize("store", ["f64", "f32", "bf16", "f32x64"])
@pytest.mark.parametrize("k", [8, 16, 40, 64, 128])
def test_apply_multi_matches_columns(sg, oracle_lib, store, k):
    A = synth.varcoef3d(14, 1.0, 4)
    Lo, Uo = oracle_lib.ilu0(A)
    MLo, MUo = oracle_lib.sait(Lo, 3, "rowrel", 1e-3), oracle_lib.sait(Uo, 3, "rowrel", 1e-3)
    R = synth.uniform(k + 1, (A.n, k))
    with sg.Context() as ctx:
        L = sg.sait_mat_create_csr(ctx, Lo.n, dev(Lo.rp), dev(Lo.ci), dev(Lo.va))
        U = sg.sait_mat_create_csr(ctx, Uo.n, dev(Uo.rp), dev(Uo.ci), dev(Uo.va))
        ML = sg.sait_build(ctx, L, True, 3, "rowrel", 1e-3, store=store)
        MU = sg.sait_build(ctx, U, False, 3, "rowrel", 1e-3, store=store)
        Z = sg.sait_apply_multi(ctx, ML, MU, dev(R)).cpu().numpy()
        torch.cuda.synchronize()
    aL = synth.CSR(A.n, MLo.rp, MLo.ci, np.abs(MLo.va))
    aU = synth.CSR(A.n, MUo.rp, MUo.ci, np.abs(MUo.va))
    for t in range(k):
        ref = oracle_lib.apply(MLo, MUo, R[:, t])
        bound = oracle_lib.apply(aL, aU, np.abs(R[:, t]))
        assert np.all(np.abs(Z[:, t] - ref) <= TOL[store] * bound), t


@pytest.mark.parametrize("store", ["f32", "bf16"])
@pytest.mark.parametrize("k", [8, 64, 128])
def test_apply_multi_four_column_gather_same_bits(sg, store, k):
    """FP32 block products gather four columns per lane when the blocks are
    16-byte aligned with leading dimensions divisible by 4, and one column per
    lane otherwise (here: Z with leading dimension k + 1).  Both sum each
    column's entries in entry order, so Z is the same bit for bit."""
    A = synth.varcoef3d(12, 1.0, 5)
    R = synth.uniform(k + 2, (A.n, k))
    with sg.Context() as ctx:
        L, U = sg.sait_ilu0(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
        ML = sg.sait_build(ctx, L, True, 3, "rowrel", 1e-3, store=store)
        MU = sg.sait_build(ctx, U, False, 3, "rowrel", 1e-3, store=store)
        Za = sg.sait_apply_multi(ctx, ML, MU, dev(R))
        Zw = torch.full((A.n, k + 1), 7.0, dtype=torch.float64, device="cuda")
        sg.sait_apply_multi(ctx, ML, MU, dev(R), Zw[:, :k])
        torch.cuda.synchronize()
    Za, Zw = Za.cpu().numpy(), Zw.cpu().numpy()
    assert np.array_equal(Za, Zw[:, :k])
    assert (Zw[:, k] == 7.0).all()
