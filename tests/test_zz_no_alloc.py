"""The allocation-free SAIT apply, sait_apply_static, against sait_apply and the oracle.

Callers that cannot let the library allocate device memory when they apply
the preconditioner -- loops that forbid allocator calls, runtimes that own all
device memory -- use sait_apply_static, whose intermediate vector lives in a
fixed array inside the library.  This test checks, through the C ABI, that
two consecutive calls give the same result as sait_apply and as the FP64
oracle's apply of the same matrices (within the product tolerances of the
parity tests), that a context created after the first call (which drops the
cached address of the array) leaves the next call correct, and that sizes
above the array's capacity are refused.  It is collected last so that a
failure here does not stop the rest of the suite.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("store", ["f64", "f32"])
def test_apply_static_matches_apply(oracle_lib, store):
    from paper_2106_12836_gb300 import build
    build.build()
    import paper_2106_12836_gb300 as sg
    torch.cuda.set_device(0)
    A = synth.convdiff3d(26)
    Lo, Uo = oracle_lib.ilu0(A)
    with sg.Context() as ctx:
        L = sg.sait_mat_create_csr(ctx, Lo.n, dev(Lo.rp), dev(Lo.ci), dev(Lo.va))
        U = sg.sait_mat_create_csr(ctx, Uo.n, dev(Uo.rp), dev(Uo.ci), dev(Uo.va))
        ML = sg.sait_build(ctx, L, True, 4, "rowrel", 1e-3, store=store)
        MU = sg.sait_build(ctx, U, False, 4, "rowrel", 1e-3, store=store)
        eML = synth.CSR(Lo.n, *(t.cpu().numpy() for t in ML.export()))
        eMU = synth.CSR(Uo.n, *(t.cpu().numpy() for t in MU.export()))
        absML = synth.CSR(Lo.n, eML.rp, eML.ci, np.abs(eML.va))
        absMU = synth.CSR(Uo.n, eMU.rp, eMU.ci, np.abs(eMU.va))
        for call, seed in enumerate((31, 32, 33)):
            if call == 2:
                sg.Context().close()   # a new context drops the cached address of the array
            r = synth.uniform(seed, A.n)
            ref = sg.sait_apply(ctx, ML, MU, dev(r)).cpu().numpy()
            z = torch.full((A.n,), float("nan"), dtype=torch.float64, device="cuda")
            st = sg.sait_apply_static(ML, MU, dev(r), z, ctx.stream)
            assert st == 0, (call, st)
            torch.cuda.synchronize()
            zs = z.cpu().numpy()
            bound = oracle_lib.apply(absML, absMU, np.abs(r))
            assert np.all(np.abs(zs - ref) <= TOL[store] * bound), call
            zo = oracle_lib.apply(eML, eMU, r)   # FP64 oracle on the same (FP64 master) values
            assert np.all(np.abs(zs - zo) <= TOL[store] * bound), call


def test_apply_static_rejects_oversized():
    from paper_2106_12836_gb300 import build
    build.build()
    import paper_2106_12836_gb300 as sg
    n = sg.APPLY_STATIC_MAX_N + 1
    with sg.Context() as ctx:
        rp = torch.arange(n + 1, dtype=torch.int32, device="cuda")
        ci = torch.arange(n, dtype=torch.int32, device="cuda")
        va = torch.ones(n, dtype=torch.float64, device="cuda")
        D = sg.sait_mat_create_csr(ctx, n, rp, ci, va)
        r = torch.ones(n, dtype=torch.float64, device="cuda")
        z = torch.zeros(n, dtype=torch.float64, device="cuda")
        assert sg.sait_apply_static(D, D, r, z, ctx.stream) == 10   # SAIT_ERR_UNSUPPORTED
        torch.cuda.synchronize()
        assert float(z.abs().max()) == 0.0
