"""Parity at the benchmark's full size: 7-point convection-diffusion on 128^3
(n = 2,097,152), ILU(0), SAIT with m = 3 terms and row-relative drop 1e-3,
GMRES(50) to 1e-8 -- the configuration bench.py times.

The oracle computes the ILU(0) factors and both SAIT matrices in full (a few
seconds); the GMRES solution is checked through a property that holds at any
size: its true FP64 residual, recomputed on the host, is below the tolerance.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def problem(oracle_lib):
    A = synth.convdiff3d(128)
    Lo, Uo = oracle_lib.ilu0(A)
    MLo = oracle_lib.sait(Lo, 3, "rowrel", 1e-3)
    MUo = oracle_lib.sait(Uo, 3, "rowrel", 1e-3)
    return A, Lo, Uo, MLo, MUo


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_full_size_chain(oracle_lib, problem):
    from paper_2106_12836_gb300 import build
    build.build()
    import paper_2106_12836_gb300 as sg
    A, Lo, Uo, MLo, MUo = problem
    with sg.Context() as ctx:
        L, U = sg.sait_ilu0(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
        for G, O in ((L, Lo), (U, Uo)):
            rp, ci, va = (t.cpu().numpy() for t in G.export())
            assert np.array_equal(rp, O.rp) and np.array_equal(ci, O.ci)
            assert np.array_equal(va, O.va)            # same fma chains: bit-exact
        ML = sg.sait_build(ctx, L, True, 3, "rowrel", 1e-3)
        MU = sg.sait_build(ctx, U, False, 3, "rowrel", 1e-3)
        for G, O in ((ML, MLo), (MU, MUo)):
            rp, ci, va = (t.cpu().numpy() for t in G.export())
            assert np.array_equal(rp, O.rp) and np.array_equal(ci, O.ci)
            assert np.all(np.abs(va - O.va) <= 1e-12 * np.abs(O.va))
        r = synth.uniform(17, A.n)
        z = sg.sait_apply(ctx, ML, MU, dev(r)).cpu().numpy()
        zo = oracle_lib.apply(MLo, MUo, r)
        bound = oracle_lib.apply(synth.CSR(A.n, MLo.rp, MLo.ci, np.abs(MLo.va)),
                                 synth.CSR(A.n, MUo.rp, MUo.ci, np.abs(MUo.va)), np.abs(r))
        assert np.all(np.abs(z - zo) <= 1e-12 * bound)
        xt = synth.uniform(synth.SEED_BASE + 2, A.n)
        b = A.to_scipy() @ xt
        Am = sg.sait_mat_create_csr(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
        for store in ("f64", "f32", "bf16"):
            sg.sait_mat_set_store(ctx, ML, store)
            sg.sait_mat_set_store(ctx, MU, store)
            P = sg.sait_prec_create_sait(ctx, ML, MU)
            x, info, st = sg.sait_gmres(ctx, Am, P, dev(b), restart=50, tol=1e-8)
            rel = np.linalg.norm(b - A.to_scipy() @ x.cpu().numpy()) / np.linalg.norm(b)
            assert st == 0 and rel <= 1e-8, (store, rel, info.iters)
            x, info, st = sg.sait_bicgstab(ctx, Am, P, dev(b), tol=1e-8)
            rel = np.linalg.norm(b - A.to_scipy() @ x.cpu().numpy()) / np.linalg.norm(b)
            assert st == 0 and rel <= 1e-8, (store, rel, info.iters)
        torch.cuda.synchronize()
