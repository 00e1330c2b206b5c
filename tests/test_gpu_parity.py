"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bars (written out in each test):
  * ILU(0) values and the SAIT structure: bit-exact (both sides run the same
    fma chains); SAIT entries whose |(M D)_ij| lies within 1e-12 of the drop
    threshold are excluded from the structure check.
  * SAIT values: within 1e-12 relative.
  * FP64 products: |y - y_ref| <= 1e-12 * (|M| |x|)_i (the usual bound for a
    reordered sum); FP32 storage 1e-5 and BF16 storage 1e-2 of the same bound.
  * Solvers: the GPU iterate's true residual, recomputed by the oracle, is
    <= tol; iteration counts within 2 of the oracle's (CGS2 vs MGS).
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


def mat(sg, ctx, A):
    return sg.sait_mat_create_csr(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))


def host_csr(M):
    rp, ci, va = (t.cpu().numpy() for t in M.export())
    return synth.CSR(M.n, rp, ci, va)


def assert_sait_parity(G: synth.CSR, O: synth.CSR, T: synth.CSR, drop: str, tau: float):
    """Structure bit-exact outside the threshold band, values within 1e-12."""
    assert G.n == O.n
    d = np.zeros(T.n)
    rows_t = np.repeat(np.arange(T.n), np.diff(T.rp))
    diag = T.ci == rows_t
    d[rows_t[diag]] = T.va[diag]
    if np.array_equal(G.rp, O.rp) and np.array_equal(G.ci, O.ci):
        assert np.all(np.abs(G.va - O.va) <= 1e-12 * np.abs(O.va))
        return
    # structures differ: every differing entry must sit at the threshold
    assert drop in ("abs", "rowrel", "hybrid"), "structure mismatch without a threshold rule"

    def entries(M):
        rows = np.repeat(np.arange(M.n), np.diff(M.rp))
        return {(int(r), int(c)): v for r, c, v in zip(rows, M.ci, M.va)}

    eg, eo = entries(G), entries(O)
    rowmax = np.zeros(T.n)
    for (r, c), v in eo.items():
        rowmax[r] = max(rowmax[r], abs(v * d[c]))
    for key in set(eg) ^ set(eo):
        v = (eg.get(key, eo.get(key))) * d[key[1]]
        thr = tau * (rowmax[key[0]] if drop == "rowrel" else 1.0)
        assert abs(abs(v) - thr) <= 1e-12 * thr, ("structure differs away from the threshold", key)
    for key in set(eg) & set(eo):
        assert abs(eg[key] - eo[key]) <= 1e-12 * abs(eo[key])


# ---- ILU(0) -------------------------------------------------------------------
@pytest.mark.parametrize("make", [lambda: synth.poisson2d(37), lambda: synth.convdiff3d(17),
                                  lambda: synth.varcoef3d(13, 1.0, 5), lambda: synth.aniso2d(50, 1e-3)])
def test_ilu0_bit_exact(sg, ctx, oracle_lib, make):
    A = make()
    L, U = sg.sait_ilu0(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
    Lo, Uo = oracle_lib.ilu0(A)
    for G, O in ((host_csr(L), Lo), (host_csr(U), Uo)):
        assert np.array_equal(G.rp, O.rp) and np.array_equal(G.ci, O.ci)
        assert np.array_equal(G.va, O.va), np.abs(G.va - O.va).max()


# ---- ILU(1) (level of fill) ---------------------------------------------------------
@pytest.mark.parametrize("make", [lambda: synth.poisson2d(37), lambda: synth.convdiff3d(17),
                                  lambda: synth.varcoef3d(13, 1.0, 5), lambda: synth.aniso2d(50, 1e-3),
                                  lambda: synth.from_dense(np.where(np.random.default_rng(3).uniform(size=(90, 90)) < 0.08,
                                                                    np.random.default_rng(4).uniform(-1, 1, (90, 90)),
                                                                    0.0) + 9 * np.eye(90))])
@pytest.mark.parametrize("level", [0, 1])
def test_iluk_bit_exact(sg, ctx, oracle_lib, make, level):
    """ILU(level) through sait_iluk: structure and values bit-identical to the
    oracle's row-by-row level-of-fill elimination (Saad, Algorithm 10.5)."""
    A = make()
    L, U = sg.sait_iluk(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va), level)
    Lo, Uo = oracle_lib.iluk(A, level)
    for G, O in ((host_csr(L), Lo), (host_csr(U), Uo)):
        assert np.array_equal(G.rp, O.rp) and np.array_equal(G.ci, O.ci)
        assert np.array_equal(G.va, O.va), np.abs(G.va - O.va).max()


def test_iluk_rejects_level_two(sg, ctx):
    A = synth.poisson2d(5)
    with pytest.raises(sg.SaitError) as e:
        sg.sait_iluk(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va), 2)
    assert e.value.status == 10    # SAIT_ERR_UNSUPPORTED


def test_ilu0_zero_pivot(sg, ctx):
    A = synth.from_dense(np.array([[1.0, 2.0], [2.0, 4.0]]))   # U_11 = 4 - 2*2 = 0
    with pytest.raises(sg.SaitError) as e:
        sg.sait_ilu0(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
    assert e.value.status == 3


# ---- SAIT build -------------------------------------------------------------------
CASES = [
    ("rowrel", 1e-3, 0, 3), ("rowrel", 1e-3, 0, 6), ("abs", 0.05, 0, 11), ("abs", 0.01, 0, 5),
    ("none", 0.0, 0, 4), ("pattern", 0.0, 2, 8), ("pattern", 0.0, 0, 4), ("pattern", 0.0, 3, 3),
    ("hybrid", 0.02, 2, 6), ("hybrid", 0.05, 0, 4),
]


@pytest.mark.parametrize("drop,tau,p,m", CASES)
def test_sait_build_pde_factors(sg, ctx, oracle_lib, drop, tau, p, m):
    A = synth.convdiff3d(19)
    Lo, Uo = oracle_lib.ilu0(A)
    for T, lower in ((Lo, True), (Uo, False)):
        Tg = mat(sg, ctx, T)
        M = sg.sait_build(ctx, Tg, lower, m, drop, tau, p)
        O = oracle_lib.sait(T, m, drop, tau, p)
        assert_sait_parity(host_csr(M), O, T, drop, tau)


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("lower", [True, False])
@pytest.mark.parametrize("drop,tau,m", [("rowrel", 0.02, 4), ("abs", 0.05, 5), ("none", 0.0, 3)])
def test_sait_build_random_ragged(sg, ctx, oracle_lib, seed, lower, drop, tau, m):
    """Empty rows, long rows (the dense overflow kernel) and several tiles of rows."""
    T = synth.random_triangular(900, lower, seed, max_row=24, empty_frac=0.15, long_frac=0.03,
                                long_row=300)
    M = sg.sait_build(ctx, mat(sg, ctx, T), lower, m, drop, tau)
    O = oracle_lib.sait(T, m, drop, tau)
    assert_sait_parity(host_csr(M), O, T, drop, tau)


@pytest.mark.parametrize("lower", [True, False])
def test_sait_exact_inverse_long_rows(sg, ctx, oracle_lib, lower):
    """m_terms = n without dropping: the exact inverse, rows up to n long."""
    n = 300
    T = synth.random_triangular(n, lower, 7, max_row=6, long_frac=0.0)
    M = sg.sait_build(ctx, mat(sg, ctx, T), lower, n, "none")
    O = oracle_lib.sait(T, n, "none")
    assert_sait_parity(host_csr(M), O, T, "none", 0.0)
    Md = host_csr(M).to_dense()
    assert np.abs(T.to_dense() @ Md - np.eye(n)).max() <= 1e-12


def test_sait_degenerate_sizes(sg, ctx, oracle_lib):
    for n in (1, 2):
        T = synth.random_triangular(n, True, 3)
        for m in (1, 2, 5):
            M = sg.sait_build(ctx, mat(sg, ctx, T), True, m, "rowrel", 1e-3)
            O = oracle_lib.sait(T, m, "rowrel", 1e-3)
            assert_sait_parity(host_csr(M), O, T, "rowrel", 1e-3)
    E = synth.CSR(0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    M = sg.sait_build(ctx, mat(sg, ctx, E), True, 3, "abs", 0.1)
    assert M.n == 0 and M.nnz == 0


def test_sait_errors(sg, ctx):
    T = synth.from_dense(np.array([[1.0, 2.0], [3.0, 4.0]]))
    with pytest.raises(sg.SaitError) as e:
        sg.sait_build(ctx, mat(sg, ctx, T), True, 3)
    assert e.value.status == 2
    Z = synth.from_dense(np.array([[1.0, 0.0], [3.0, 0.0]]))
    with pytest.raises(sg.SaitError) as e:
        sg.sait_build(ctx, mat(sg, ctx, Z), True, 3)
    assert e.value.status == 3
    T = synth.from_dense(np.tril(np.ones((3, 3))))
    with pytest.raises(sg.SaitError) as e:
        sg.sait_build(ctx, mat(sg, ctx, T), True, 0)
    assert e.value.status == 1
    with pytest.raises(sg.SaitError) as e:
        sg.sait_build(ctx, mat(sg, ctx, T), True, 3, "abs", 1.5)
    assert e.value.status == 1
    bad = synth.CSR(2, np.array([0, 2, 3], np.int32), np.array([1, 0, 1], np.int32),
                    np.ones(3))
    with pytest.raises(sg.SaitError) as e:
        mat(sg, ctx, bad)
    assert e.value.status == 1


# ---- products -------------------------------------------------------------------
@pytest.mark.parametrize("store,tol", [("f64", 1e-12), ("f32", 1e-5), ("bf16", 1e-2), ("f32x64", 1e-6),
                                       ("bf16x64", 1e-2)])
def test_apply_parity(sg, ctx, oracle_lib, store, tol):
    A = synth.convdiff3d(23)
    Lo, Uo = oracle_lib.ilu0(A)
    MLo, MUo = oracle_lib.sait(Lo, 4, "rowrel", 1e-3), oracle_lib.sait(Uo, 4, "rowrel", 1e-3)
    ML = sg.sait_build(ctx, mat(sg, ctx, Lo), True, 4, "rowrel", 1e-3, store=store)
    MU = sg.sait_build(ctx, mat(sg, ctx, Uo), False, 4, "rowrel", 1e-3, store=store)
    r = synth.uniform(11, A.n)
    z = sg.sait_apply(ctx, ML, MU, dev(r)).cpu().numpy()
    zo = oracle_lib.apply(MLo, MUo, r)
    absML = synth.CSR(MLo.n, MLo.rp, MLo.ci, np.abs(MLo.va))
    absMU = synth.CSR(MUo.n, MUo.rp, MUo.ci, np.abs(MUo.va))
    bound = oracle_lib.apply(absML, absMU, np.abs(r))
    assert np.all(np.abs(z - zo) <= tol * bound)


@pytest.mark.parametrize("store,rounding", [("f32x64", np.float32), ("bf16x64", "bf16")])
def test_apply_x64_is_the_rounded_matrix_in_fp64(sg, ctx, oracle_lib, store, rounding):
    """*_X64 storage applies exactly the rounded matrix: compare with the
    oracle applying round(M) (rounded on the host) in FP64, FP64 tolerance."""
    import torch as _t
    A = synth.convdiff3d(21)
    Lo, Uo = oracle_lib.ilu0(A)
    MLo, MUo = oracle_lib.sait(Lo, 3, "rowrel", 1e-3), oracle_lib.sait(Uo, 3, "rowrel", 1e-3)

    def rnd(v):
        if rounding == "bf16":
            return _t.from_numpy(v).to(_t.bfloat16).to(_t.float64).numpy()
        return v.astype(np.float32).astype(np.float64)

    MLr = synth.CSR(A.n, MLo.rp, MLo.ci, rnd(MLo.va))
    MUr = synth.CSR(A.n, MUo.rp, MUo.ci, rnd(MUo.va))
    ML = sg.sait_build(ctx, mat(sg, ctx, Lo), True, 3, "rowrel", 1e-3, store=store)
    MU = sg.sait_build(ctx, mat(sg, ctx, Uo), False, 3, "rowrel", 1e-3, store=store)
    r = synth.uniform(12, A.n)
    z = sg.sait_apply(ctx, ML, MU, dev(r)).cpu().numpy()
    zo = oracle_lib.apply(MLr, MUr, r)
    bound = oracle_lib.apply(synth.CSR(A.n, MLr.rp, MLr.ci, np.abs(MLr.va)),
                             synth.CSR(A.n, MUr.rp, MUr.ci, np.abs(MUr.va)), np.abs(r))
    assert np.all(np.abs(z - zo) <= 1e-12 * bound)


def test_fp32_storage_narrows_like_ieee(sg, ctx):
    """An FP32-stored identity applied to FP64 x gives float(x) widened back: the
    products narrow FP64 entries to FP32 with integer round-to-nearest-even and
    widen FP32 sums exactly, so the result must equal numpy's IEEE conversion bit
    for bit, ties and the top of the range included; below the smallest normal
    FP32 magnitude (2^-126) the narrowing gives zero."""
    rng = np.random.default_rng(11)
    f = rng.uniform(1, 2, 4000).astype(np.float32).astype(np.float64) * np.exp2(rng.integers(-120, 120, 4000))
    ulp = np.spacing(f.astype(np.float32)).astype(np.float64)
    x = np.concatenate([
        rng.standard_normal(20000) * np.exp2(rng.integers(-100, 100, 20000)),  # generic values
        f + ulp / 2, f - ulp / 4, f + 3 * ulp / 4,                                # exact ties and near ties
        -(f + ulp / 2),
        [np.float64(np.finfo(np.float32).max), 3.4028235e38 * (1 + 2 ** -30), 2.0 ** -126, -(2.0 ** -126),
         0.0, -0.0, 1.0, 1 + 2 ** -24, 1 + 3 * 2 ** -24, 2.0 ** -130, -(2.0 ** -140)],
    ])
    n = len(x)
    I = synth.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n))
    M = sg.sait_mat_create_csr(ctx, n, dev(I.rp), dev(I.ci), dev(I.va))
    sg.sait_mat_set_store(ctx, M, "f32")
    y = sg.sait_spmv(ctx, M, dev(x)).cpu().numpy()
    with np.errstate(over="ignore"):
        want = x.astype(np.float32).astype(np.float64)
    normal = np.abs(x) >= 2.0 ** -126
    assert np.array_equal(y[normal].view(np.int64), want[normal].view(np.int64))
    assert np.all(y[~normal] == 0.0)   # (the sum starts from +0, so the sign of a zero is not kept)


def test_spmv_parity_ragged(sg, ctx, oracle_lib):
    T = synth.random_triangular(2000, True, 5, max_row=60, empty_frac=0.2, long_frac=0.02,
                                long_row=1500)
    x = synth.uniform(3, T.n)
    y = sg.sait_spmv(ctx, mat(sg, ctx, T), dev(x)).cpu().numpy()
    yo = oracle_lib.spmv(T, x)
    bound = oracle_lib.spmv(synth.CSR(T.n, T.rp, T.ci, np.abs(T.va)), np.abs(x))
    assert np.all(np.abs(y - yo) <= 1e-12 * bound)


def _sigma_case(n=8192, seed=17):
    """Rows of 2 and 40 entries, 24 short then 8 long in every 32 rows: each
    natural 32-row slice pads to 40 slots, while sorting 256-row windows by
    length puts the long rows into slices of their own."""
    rng = np.random.default_rng(seed)
    lens = np.where(np.arange(n) % 32 < 24, 2, 40)
    ci = np.concatenate([np.sort(rng.choice(n, size=k, replace=False)) for k in lens]).astype(np.int32)
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum(lens)
    return synth.CSR(n, rp, ci, rng.uniform(-1.0, 1.0, size=int(rp[-1])))


def _sell_padding(lens, sigma):
    """Padded slots / entries of SELL-32 after sorting windows of sigma rows by
    length (longest first, stable); sigma = 1 keeps the natural order."""
    n = len(lens)
    order = np.arange(n)
    if sigma > 1:
        order = np.concatenate([w + np.argsort(-lens[w:w + sigma], kind="stable") for w in range(0, n, sigma)])
    ls = lens[order]
    return sum(32 * int(ls[s:s + 32].max()) for s in range(0, n, 32)) / int(lens.sum())


def test_spmv_sigma_sorted_sell(sg, ctx, oracle_lib):
    """A matrix too ragged for natural-order SELL-32 (3.5x padding) gets the
    sorted-window layout (no padding) instead of CSR products; the product
    writes each row back to its place."""
    A = _sigma_case()
    lens = np.diff(A.rp)
    assert _sell_padding(lens, 1) > 1.2 and _sell_padding(lens, 256) <= 1.2
    M = mat(sg, ctx, A)
    x = synth.uniform(5, A.n)
    y = sg.sait_spmv(ctx, M, dev(x)).cpu().numpy()
    yo = oracle_lib.spmv(A, x)
    bound = oracle_lib.spmv(synth.CSR(A.n, A.rp, A.ci, np.abs(A.va)), np.abs(x))
    assert np.all(np.abs(y - yo) <= 1e-12 * bound)
    # FP32 values with FP64-accurate sums through the same permuted slices: the
    # rounded matrix, to FP64 tolerance
    sg.sait_mat_set_store(ctx, M, "f32x64")
    y32 = sg.sait_spmv(ctx, M, dev(x)).cpu().numpy()
    Ar = synth.CSR(A.n, A.rp, A.ci, A.va.astype(np.float32).astype(np.float64))
    assert np.all(np.abs(y32 - oracle_lib.spmv(Ar, x)) <= 1e-12 * bound)
    rep = sg.sait_mat_autotune(ctx, M).as_dict()
    assert any(c["format"] == "sell32" for c in rep["candidates"])


def _banded(n, far, lower, seed):
    """Triangular rows with the diagonal, a neighbour and one entry at distance
    `far` (where it exists): the band is exactly `far` wide."""
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(n):
        c = [i]
        j = i - 1 if lower else i + 1
        if 0 <= j < n:
            c.append(j)
        j = i - far if lower else i + far
        if 0 <= j < n:
            c.append(j)
        c.sort()
        rows.append(len(c))
        cols.extend(c)
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum(rows)
    return synth.CSR(n, rp, np.array(cols, np.int32), rng.uniform(-1.0, 1.0, len(cols)))


@pytest.mark.parametrize("far,lower", [(65535, True), (70000, False), (300, True)])
def test_sell_wide_band(sg, ctx, oracle_lib, far, lower):
    """SELL-32 with columns far from the diagonal (beyond any 16-bit offset)
    and a ragged tail: the FP64 product bar, then the same after tuning."""
    T = _banded(70001, far, lower, far)
    M = mat(sg, ctx, T)
    x = synth.uniform(9, T.n, -1.0, 1.0)
    bound = oracle_lib.spmv(synth.CSR(T.n, T.rp, T.ci, np.abs(T.va)), np.abs(x))
    ref = oracle_lib.spmv(T, x)
    y = sg.sait_spmv(ctx, M, dev(x)).cpu().numpy()  # SELL-32 until a tuner says otherwise
    assert np.all(np.abs(y - ref) <= 1e-12 * bound)
    rep = sg.sait_mat_autotune(ctx, M).as_dict()
    assert rep["candidates"][0]["format"] == "sell32"
    y = sg.sait_spmv(ctx, M, dev(x)).cpu().numpy()
    assert np.all(np.abs(y - ref) <= 1e-12 * bound)


def test_exact_ilu_preconditioner(sg, ctx, oracle_lib):
    A = synth.convdiff3d(21)
    L, U = sg.sait_ilu0(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
    Lo, Uo = oracle_lib.ilu0(A)
    P = sg.sait_prec_create_ilu(ctx, L, U)
    assert sg.sait_prec_levels(P) == (3 * 21 - 2, 3 * 21 - 2)
    r = synth.uniform(4, A.n)
    z = sg.sait_prec_apply(ctx, P, dev(r)).cpu().numpy()
    zo = oracle_lib.trisolve(Uo, oracle_lib.trisolve(Lo, r, True), False)
    assert np.abs(z - zo).max() <= 1e-12 * np.abs(zo).max()


# ---- solvers -------------------------------------------------------------------
@pytest.fixture(scope="module")
def c1(oracle_lib):
    A = synth.poisson2d(64)
    xt = synth.uniform(synth.SEED_BASE + 1, A.n)
    b = oracle_lib.spmv(A, xt)
    Lo, Uo = oracle_lib.ilu0(A)
    return A, b, Lo, Uo


@pytest.mark.parametrize("prec", ["sait", "ilu", "none"])
def test_gmres_c1(sg, ctx, oracle_lib, c1, prec):
    A, b, Lo, Uo = c1
    Ag = mat(sg, ctx, A)
    L, U = sg.sait_ilu0(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
    if prec == "sait":
        P = sg.sait_prec_create_sait(ctx, sg.sait_build(ctx, L, True, 3, "rowrel", 1e-3),
                                     sg.sait_build(ctx, U, False, 3, "rowrel", 1e-3))
        lo, up = oracle_lib.sait(Lo, 3, "rowrel", 1e-3), oracle_lib.sait(Uo, 3, "rowrel", 1e-3)
    elif prec == "ilu":
        P = sg.sait_prec_create_ilu(ctx, L, U)
        lo, up = Lo, Uo
    else:
        P, lo, up = None, None, None
    x, info, st = sg.sait_gmres(ctx, Ag, P, dev(b), restart=30, tol=1e-8, maxit=5000)
    xo, ito, rro, sto = oracle_lib.gmres(A, b, prec, lo, up, restart=30, tol=1e-8, maxit=5000)
    xg = x.cpu().numpy()
    rel = np.linalg.norm(b - oracle_lib.spmv(A, xg)) / np.linalg.norm(b)
    assert st == 0 and sto == 0
    assert rel <= 1e-8 and abs(info.rel_resid - rel) <= 1e-3 * rel
    assert abs(info.iters - ito) <= max(2, 0.02 * ito), (info.iters, ito)


@pytest.mark.parametrize("prec", ["sait", "ilu"])
def test_bicgstab_convdiff(sg, ctx, oracle_lib, prec):
    A = synth.convdiff3d(20)
    xt = synth.uniform(9, A.n)
    b = oracle_lib.spmv(A, xt)
    Lo, Uo = oracle_lib.ilu0(A)
    L, U = sg.sait_ilu0(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
    if prec == "sait":
        P = sg.sait_prec_create_sait(ctx, sg.sait_build(ctx, L, True, 3, "rowrel", 1e-3),
                                     sg.sait_build(ctx, U, False, 3, "rowrel", 1e-3))
        lo, up = oracle_lib.sait(Lo, 3, "rowrel", 1e-3), oracle_lib.sait(Uo, 3, "rowrel", 1e-3)
    else:
        P = sg.sait_prec_create_ilu(ctx, L, U)
        lo, up = Lo, Uo
    x, info, st = sg.sait_bicgstab(ctx, mat(sg, ctx, A), P, dev(b), tol=1e-8, maxit=2000)
    xo, ito, rro, sto = oracle_lib.bicgstab(A, b, prec, lo, up, tol=1e-8, maxit=2000)
    rel = np.linalg.norm(b - oracle_lib.spmv(A, x.cpu().numpy())) / np.linalg.norm(b)
    assert st == 0 and sto == 0 and rel <= 1e-8
    assert abs(info.iters - ito) <= max(3, 0.1 * ito), (info.iters, ito)


@pytest.mark.parametrize("restart", [7, 30])
def test_gmres_ragged_n(sg, ctx, oracle_lib, restart):
    """n = 17^3 = 4913 (not a multiple of 4: the padded basis rows must stay inert)."""
    A = synth.convdiff3d(17)
    b = oracle_lib.spmv(A, synth.uniform(21, A.n, -1.0, 1.0))
    Lo, Uo = oracle_lib.ilu0(A)
    L, U = sg.sait_ilu0(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
    P = sg.sait_prec_create_sait(ctx, sg.sait_build(ctx, L, True, 3, "rowrel", 1e-3),
                                 sg.sait_build(ctx, U, False, 3, "rowrel", 1e-3))
    lo, up = oracle_lib.sait(Lo, 3, "rowrel", 1e-3), oracle_lib.sait(Uo, 3, "rowrel", 1e-3)
    x, info, st = sg.sait_gmres(ctx, mat(sg, ctx, A), P, dev(b), restart=restart, tol=1e-10, maxit=3000)
    xo, ito, rro, sto = oracle_lib.gmres(A, b, "sait", lo, up, restart=restart, tol=1e-10, maxit=3000)
    rel = np.linalg.norm(b - oracle_lib.spmv(A, x.cpu().numpy())) / np.linalg.norm(b)
    assert st == 0 and sto == 0 and rel <= 1e-10
    assert abs(info.iters - ito) <= max(2, 0.02 * ito), (info.iters, ito)


@pytest.mark.parametrize("restart", [1, 2, 3])
def test_gmres_short_restarts(sg, ctx, oracle_lib, restart):
    """The delayed reorthogonalization at its smallest cycles (the close step finalizes every column)."""
    A = synth.poisson2d(12)
    b = oracle_lib.spmv(A, synth.uniform(31, A.n, -1.0, 1.0))
    Lo, Uo = oracle_lib.ilu0(A)
    L, U = sg.sait_ilu0(ctx, A.n, dev(A.rp), dev(A.ci), dev(A.va))
    P = sg.sait_prec_create_sait(ctx, sg.sait_build(ctx, L, True, 3, "rowrel", 1e-3),
                                 sg.sait_build(ctx, U, False, 3, "rowrel", 1e-3))
    lo, up = oracle_lib.sait(Lo, 3, "rowrel", 1e-3), oracle_lib.sait(Uo, 3, "rowrel", 1e-3)
    x, info, st = sg.sait_gmres(ctx, mat(sg, ctx, A), P, dev(b), restart=restart, tol=1e-9, maxit=20000)
    xo, ito, rro, sto = oracle_lib.gmres(A, b, "sait", lo, up, restart=restart, tol=1e-9, maxit=20000)
    rel = np.linalg.norm(b - oracle_lib.spmv(A, x.cpu().numpy())) / np.linalg.norm(b)
    assert st == 0 and sto == 0 and rel <= 1e-9
    assert abs(info.iters - ito) <= max(3, 0.05 * ito), (info.iters, ito)


def test_gmres_nonconvergence_and_zero_rhs(sg, ctx, oracle_lib, c1):
    A, b, _, _ = c1
    Ag = mat(sg, ctx, A)
    x, info, st = sg.sait_gmres(ctx, Ag, None, dev(b), restart=5, tol=1e-12, maxit=7, check=False)
    assert st == 6 and info.iters == 7
    rel = np.linalg.norm(b - oracle_lib.spmv(A, x.cpu().numpy())) / np.linalg.norm(b)
    assert abs(info.rel_resid - rel) <= 1e-6 * rel
    x, info, st = sg.sait_gmres(ctx, Ag, None, torch.zeros(A.n, dtype=torch.float64, device="cuda"))
    assert st == 0 and float(x.abs().max()) == 0.0
