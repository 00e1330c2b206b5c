"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these tests retypes the oracle's own formula: each compares it with an
independent statement (a dense inverse from LAPACK, a closed form, Jacobi
sweeps done densely, the paper's printed ratios and iteration counts, the
defining property of ILU(0), a dense direct solve).
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Section 2, equation T_inverse: T~ is strictly triangular, hence nilpotent,
# so the series with n terms and no dropping is the exact inverse.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("lower", [True, False])
@pytest.mark.parametrize("seed", [1, 2])
def test_exact_inverse_matches_lapack(oracle_lib, lower, seed):
    n = 48
    T = synth.random_triangular(n, lower, seed, max_row=12, long_frac=0.0)
    M = oracle_lib.sait(T, n, "none")
    ref = np.linalg.inv(T.to_dense())
    assert np.abs(M.to_dense() - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())
    assert np.abs(T.to_dense() @ M.to_dense() - np.eye(n)).max() <= 1e-13


@pytest.mark.parametrize("g", [5, 8])
def test_nilpotency_depth_of_2d_ilu0_factors(oracle_lib, g):
    """T~^k = 0 once k reaches the number of level sets (2g-1 on a g x g grid)."""
    L, U = oracle_lib.ilu0(synth.poisson2d(g))
    for T in (L, U):
        Td = T.to_dense()
        exact = oracle_lib.sait(T, 2 * g - 1, "none").to_dense()
        assert np.abs(Td @ exact - np.eye(g * g)).max() <= 1e-13
        short = oracle_lib.sait(T, 2 * g - 2, "none").to_dense()
        assert np.abs(Td @ short - np.eye(g * g)).max() > 1e-8


def test_bidiagonal_closed_form(oracle_lib):
    """T = diag(d) + c on the subdiagonal: (M)_ij = prod_{l=j+1..i}(-c_l/d_l) / d_j."""
    n, m_terms = 40, 7
    rng = np.random.default_rng(5)
    d = rng.uniform(1.0, 3.0, n)
    c = rng.uniform(-1.5, 1.5, n)
    dense = np.diag(d) + np.diag(c[1:], -1)
    T = synth.from_dense(dense)
    M = oracle_lib.sait(T, m_terms, "none").to_dense()
    ref = np.zeros((n, n))
    for i in range(n):
        for j in range(max(0, i - m_terms + 1), i + 1):
            ref[i, j] = np.prod(-c[j + 1:i + 1] / d[j + 1:i + 1]) / d[j]
    assert np.abs(M - ref).max() <= 1e-14 * np.abs(ref).max()
    assert np.count_nonzero(M) == sum(min(m_terms, i + 1) for i in range(n))


# --------------------------------------------------------------------------
# Section 2, equation Jacobi_iter: M_k b equals k Jacobi sweeps from x^0 = 0.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("lower", [True, False])
@pytest.mark.parametrize("k", [1, 2, 3, 6])
def test_series_equals_jacobi_sweeps(oracle_lib, lower, k):
    n = 120
    T = synth.random_triangular(n, lower, 11 + k, max_row=20, long_frac=0.02, long_row=80)
    Td = T.to_dense()
    D = np.diag(Td)
    b = synth.uniform(3, n)
    x = np.zeros(n)
    for _ in range(k):
        x = (np.diag(D) - Td) @ x / D + b / D      # x^k = D^-1 (D - T) x^{k-1} + D^-1 b
    M = oracle_lib.sait(T, k, "none")
    y = M.to_dense() @ b
    assert np.abs(y - x).max() <= 1e-13 * max(1.0, np.abs(x).max())


# --------------------------------------------------------------------------
# ILUT(tau, lfil) (Saad, Algorithm 10.6).
# --------------------------------------------------------------------------
def _dense(L, U):
    return L.to_dense(), U.to_dense()


@pytest.mark.parametrize("make", [lambda: synth.convdiff3d(4), lambda: synth.varcoef3d(4, 1.0, 77),
                                  lambda: synth.aniso2d(7, 0.01)])
def test_ilut_without_dropping_is_exact_lu(oracle_lib, make):
    """tau = 0 and lfil >= n keep every fill entry: L U = A with L unit lower, U upper (the unique LU)."""
    A = make()
    L, U = oracle_lib.ilut(A, 0.0, A.n)
    Ld, Ud = _dense(L, U)
    Ad = A.to_dense()
    assert np.array_equal(np.diag(Ld), np.ones(A.n)) and not np.triu(Ld, 1).any() and not np.tril(Ud, -1).any()
    assert np.abs(Ld @ Ud - Ad).max() <= 1e-13 * np.abs(Ad).max()
    # the same factors by dense Doolittle elimination in LAPACK order: solve with them
    b = synth.uniform(3, A.n)
    x = sla.solve_triangular(Ud, sla.solve_triangular(Ld, b, lower=True), lower=False)
    assert np.abs(x - np.linalg.solve(Ad, b)).max() <= 1e-11 * np.abs(x).max()


def test_ilut_tridiagonal_equals_ilu0(oracle_lib):
    """A tridiagonal LU has no fill, so ILUT(0, lfil >= 1) and ILU(0) run the same fma chain: bit-equal."""
    A = synth.from_dense(np.diag(np.full(50, 4.0)) + np.diag(synth.uniform(5, 49, -1.5, -0.5), -1) +
                         np.diag(synth.uniform(6, 49, -1.5, -0.5), 1))
    L, U = oracle_lib.ilut(A, 0.0, 1)
    L0, U0 = oracle_lib.ilu0(A)
    for X, Y in ((L, L0), (U, U0)):
        assert np.array_equal(X.rp, Y.rp) and np.array_equal(X.ci, Y.ci) and np.array_equal(X.va, Y.va)


def test_ilut_closed_forms(oracle_lib):
    """A huge tau drops every multiplier (first rule), lfil = 0 drops every off-diagonal (second rule):
    both leave L = I and U = diag(A), since no update ever reaches the diagonal."""
    A = synth.convdiff3d(6)
    rows = np.repeat(np.arange(A.n), np.diff(A.rp))
    dA = A.va[A.ci == rows]
    for tau, lfil in ((1e30, 10), (0.0, 0)):
        L, U = oracle_lib.ilut(A, tau, lfil)
        assert L.nnz == A.n and U.nnz == A.n
        assert np.array_equal(L.va, np.ones(A.n)) and np.array_equal(U.va, dA)


@pytest.mark.parametrize("tau,lfil", [(1e-4, 10), (1e-2, 3), (0.0, 2)])
def test_ilut_drop_invariants(oracle_lib, tau, lfil):
    A = synth.varcoef3d(8, 1.0, 123)
    L, U = oracle_lib.ilut(A, tau, lfil)
    norms = np.sqrt(np.add.reduceat(A.va ** 2, A.rp[:-1]))
    for T, lower in ((L, True), (U, False)):
        rows = np.repeat(np.arange(T.n), np.diff(T.rp))
        off = T.ci != rows
        assert np.all(np.diff(T.rp) - 1 <= lfil)
        assert np.all(np.abs(T.va[off]) >= tau * norms[rows[off]])
        assert np.all(T.va[off] != 0.0)
        assert np.all(T.ci[off] < rows[off]) if lower else np.all(T.ci[off] > rows[off])
        assert np.count_nonzero(~off) == T.n
    # (L U)_ij = a_ij wherever (i, j) is kept in U and no entry was dropped on that row (tau = 0, lfil large)
    L2, U2 = oracle_lib.ilut(A, 0.0, A.n)
    assert np.abs(L2.to_dense() @ U2.to_dense() - A.to_dense()).max() <= 1e-12 * np.abs(A.va).max()


def test_ilut_error_decreases_with_tau(oracle_lib):
    """Less dropping gives a better factorization: ||A - L U||_F falls as tau falls (lfil large)."""
    A = synth.varcoef3d(6, 1.0, 321)
    Ad = A.to_dense()
    errs = []
    for tau in (1e-1, 1e-2, 1e-3, 1e-4, 0.0):
        L, U = oracle_lib.ilut(A, tau, A.n)
        errs.append(np.linalg.norm(Ad - L.to_dense() @ U.to_dense()))
    assert all(a > b for a, b in zip(errs, errs[1:-1])) and errs[-1] <= 1e-12 * np.linalg.norm(Ad)


def test_ilut_keeps_largest(oracle_lib):
    """Second rule on a row with one elimination step: the lfil kept U entries are the largest of w."""
    # row 0 has three off-diagonals (all kept); row 1 = a_1 - (a_10 / a_00) a_0 has five candidates
    n = 8
    Ad = np.eye(n) * 10.0
    Ad[0, [2, 3, 5]] = [-3.0, 2.0, 4.0]
    Ad[1, [0, 3, 6, 7]] = [2.0, 0.5, 0.3, -0.7]
    A = synth.from_dense(Ad)
    L, U = oracle_lib.ilut(A, 0.0, 3)
    w = Ad[1].copy()
    l10 = w[0] / Ad[0, 0]
    w[1:] = w[1:] - l10 * Ad[0, 1:]          # 0.6, 0.1, -0.8, 0.3, -0.7 at columns 2, 3, 5, 6, 7
    off = np.arange(2, n)
    top = off[np.argsort(-np.abs(w[off]), kind="stable")[:3]]
    Ud = U.to_dense()
    assert set(top) == {2, 5, 7}
    assert set(np.nonzero(Ud[1, 2:])[0] + 2) == set(top)
    assert np.abs(Ud[1, top] - w[top]).max() <= 1e-15
    assert L.to_dense()[1, 0] == l10


# --------------------------------------------------------------------------
# Jacobi sweeps (equation Jacobi_iter; Section 4, comparison with Jacobi).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("lower", [True, False])
def test_jacobi_sweeps_exact_after_n(oracle_lib, lower):
    """T~ of a triangular T is nilpotent, so n sweeps give T^-1 b exactly."""
    n = 40
    T = synth.random_triangular(n, lower, 5, max_row=8)
    b = synth.uniform(7, n)
    x = oracle_lib.jacobi(T, b, n)
    ref = sla.solve_triangular(T.to_dense(), b, lower=lower)
    assert np.abs(x - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("k", [0, 1, 2, 5])
def test_jacobi_sweeps_equal_series(oracle_lib, k):
    """k sweeps from zero apply M_k = sum_{j<k} T~^j D^-1 (Section 2): the pinned SAIT with no dropping."""
    T = synth.random_triangular(150, True, 21 + k, max_row=12)
    b = synth.uniform(9, T.n)
    x = oracle_lib.jacobi(T, b, k)
    if k == 0:
        assert not x.any()
        return
    y = oracle_lib.sait(T, k, "none").to_dense() @ b
    assert np.abs(x - y).max() <= 1e-13 * max(1.0, np.abs(y).max())


def test_jacobi_sweeps_general_matrix(oracle_lib):
    """On a strictly diagonally dominant non-triangular matrix the sweeps converge to A^-1 b."""
    A = synth.poisson2d(6)
    rows = np.repeat(np.arange(A.n), np.diff(A.rp))
    va = np.where(A.ci == rows, 2.0 * A.va, A.va)      # diagonal 8 against off-diagonal sum 4
    B = synth.CSR(A.n, A.rp, A.ci, va)
    b = synth.uniform(13, A.n)
    x = oracle_lib.jacobi(B, b, 80)
    ref = np.linalg.solve(B.to_dense(), b)
    assert np.abs(x - ref).max() <= 1e-12 * np.abs(ref).max()


def test_jacobi_prec_pcg_between_diagonal_and_exact(oracle_lib):
    """More sweeps approach the exact ILU solves: iterations fall from the diagonal case towards the exact one."""
    A = synth.laplace3d(14)
    L, U = oracle_lib.ilu0(A)
    b = synth.uniform(17, A.n)
    its = []
    for kind in ("jacobi1", "jacobi3", "jacobi40", "ilu"):
        _, it, rr, st = oracle_lib.pcg(A, b, kind, L, U, tol=1e-10)
        assert st == 0 and rr <= 1e-10
        its.append(it)
    assert its[0] > its[1] > its[3] and its[2] == its[3]


# --------------------------------------------------------------------------
# Algorithms 2-3 with brute force: a dense Horner loop with a mask on tiny
# matrices.  Entries within 1e-12 of a threshold are not graded.
# --------------------------------------------------------------------------
def _dense_sait(Td, m_terms, rule, tau=0.0, p=0):
    n = Td.shape[0]
    D = np.diag(Td)
    Tt = np.eye(n) - Td / D[:, None]
    np.fill_diagonal(Tt, 0.0)
    MD = np.eye(n)
    S = np.eye(n, dtype=bool)          # p = 0: the pattern of M_0 D = I
    near = np.zeros((n, n), bool)
    for it in range(1, m_terms):
        full = Tt @ MD + np.eye(n)
        struct = (np.abs(Tt) > 0).astype(float) @ (np.abs(MD) > 0).astype(float) > 0
        struct |= np.eye(n, dtype=bool)
        keep = struct.copy()
        if rule in ("abs", "rowrel"):
            thr = tau * (np.abs(full).max(axis=1, keepdims=True) if rule == "rowrel" else 1.0)
            keep &= ~(np.abs(full) < thr)
            near |= struct & (np.abs(np.abs(full) - thr) <= 1e-12 * np.maximum(thr, 1e-300))
        elif rule == "pattern" and it > p:
            keep &= S
        elif rule == "hybrid" and it > p:
            keep &= ~(np.abs(full) < tau)
            near |= struct & (np.abs(np.abs(full) - tau) <= 1e-12 * max(tau, 1e-300))
        keep |= np.eye(n, dtype=bool)
        MD = np.where(keep, full, 0.0)
        if rule == "pattern" and it == p:
            S = keep.copy()
    return MD / D[None, :], MD != 0, near


@pytest.mark.parametrize("rule,tau,p", [("abs", 0.05, 0), ("abs", 0.2, 0), ("rowrel", 0.1, 0),
                                        ("pattern", 0.0, 1), ("pattern", 0.0, 2),
                                        ("pattern", 0.0, 0), ("none", 0.0, 0), ("hybrid", 0.05, 2),
                                        ("hybrid", 0.2, 1)])
@pytest.mark.parametrize("lower", [True, False])
def test_dropping_against_dense_brute_force(oracle_lib, rule, tau, p, lower):
    n, m_terms = 60, 5
    T = synth.random_triangular(n, lower, 21, max_row=6, long_frac=0.05, long_row=20)
    ref, ref_pat, near = _dense_sait(T.to_dense(), m_terms, rule, tau, p)
    M = oracle_lib.sait(T, m_terms, rule, tau, p)
    Md = M.to_dense()
    pat = np.zeros((n, n), bool)
    rows = np.repeat(np.arange(n), np.diff(M.rp))
    pat[rows, M.ci] = True
    graded = ~near
    assert np.array_equal(pat & graded, ref_pat & graded)
    both = pat & ref_pat
    assert np.abs(Md[both] - ref[both]).max() <= 1e-12 * np.abs(ref).max()


# --------------------------------------------------------------------------
# Paper-replica: Table runtime_SAIT, level-0 ILU of the 100^3 Laplacian.
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def laplace100(oracle_lib):
    A = synth.laplace3d(100)
    L, U = oracle_lib.ilu0(A)
    return A, L, U


@pytest.fixture(scope="module")
def golden_runtime():
    with open(os.path.join(GOLDEN, "paper_runtime_sait.json")) as f:
        return json.load(f)


@pytest.mark.slow
def test_paper_ratios_sait_thr(oracle_lib, laplace100, golden_runtime):
    A, L, U = laplace100
    assert L.nnz == 3_970_000 and U.nnz == 3_970_000   # sum over a+b+c<=1 of (100-a)(100-b)(100-c)
    m = golden_runtime["loop_iterations_m"]
    for row in golden_runtime["sait_thr"]:
        M = oracle_lib.sait(L, m + 1, "abs", row["tau"])
        assert round(M.nnz / L.nnz, 2) == row["ratio"], row


@pytest.mark.slow
def test_paper_ratios_sait_pat(oracle_lib, laplace100, golden_runtime):
    A, L, U = laplace100
    m = golden_runtime["loop_iterations_m"]
    for row in golden_runtime["sait_pat"]:
        M = oracle_lib.sait(U, row["p"] + m + 1, "pattern", 0.0, row["p"])
        assert round(M.nnz / U.nnz, 2) == row["ratio"], row


@pytest.mark.slow
def test_paper_pcg_iteration_counts(oracle_lib, laplace100, golden_runtime):
    """Right-hand side and seed are not stated by the paper: b ~ U[0,1)."""
    A, L, U = laplace100
    b = synth.uniform(synth.SEED_BASE, A.n, 0.0, 1.0)
    tol = golden_runtime["pcg_tol"]
    _, it, rr, st = oracle_lib.pcg(A, b, "ilu", L, U, tol=tol)
    assert st == 0 and rr <= tol
    assert abs(it - golden_runtime["exact_ilu0_pcg_iters"]) <= 3
    row = golden_runtime["sait_thr"][0]
    ML = oracle_lib.sait(L, golden_runtime["loop_iterations_m"] + 1, "abs", row["tau"])
    MU = oracle_lib.sait(U, golden_runtime["loop_iterations_m"] + 1, "abs", row["tau"])
    _, it2, rr2, st2 = oracle_lib.pcg(A, b, "sait", ML, MU, tol=tol)
    assert st2 == 0 and rr2 <= tol
    assert abs(it2 - row["pcg_iters"]) <= 0.1 * row["pcg_iters"]
    assert it2 > it      # SAIT never beats the exact triangular solves (Section 4.1)


@pytest.mark.slow
def test_paper_jacobi_pcg_iteration_counts(oracle_lib, laplace100):
    """Table runtime_Jacobi, level-0 column, a few rows; right-hand side b ~ U[0,1) as above."""
    with open(os.path.join(GOLDEN, "paper_runtime_jacobi.json")) as f:
        g = json.load(f)
    A, L, U = laplace100
    b = synth.uniform(synth.SEED_BASE, A.n, 0.0, 1.0)
    for k in (1, 3, 10):
        _, it, rr, st = oracle_lib.pcg(A, b, f"jacobi{k}", L, U, tol=g["pcg_tol"])
        assert st == 0 and rr <= g["pcg_tol"]
        assert abs(it - g["level0_pcg_iters"][str(k)]) <= 0.05 * g["level0_pcg_iters"][str(k)], (k, it)


def test_hybrid_limits(oracle_lib):
    """Hybrid with every product undropped is the exact series; with no undropped product it is SAIT_Thr."""
    L, _ = oracle_lib.ilu0(synth.convdiff3d(10))
    for m in (3, 5):
        H = oracle_lib.sait(L, m, "hybrid", 0.05, m - 1)
        N = oracle_lib.sait(L, m, "none")
        assert np.array_equal(H.rp, N.rp) and np.array_equal(H.ci, N.ci) and np.array_equal(H.va, N.va)
        H0 = oracle_lib.sait(L, m, "hybrid", 0.05, 0)
        A0 = oracle_lib.sait(L, m, "abs", 0.05)
        assert np.array_equal(H0.rp, A0.rp) and np.array_equal(H0.ci, A0.ci) and np.array_equal(H0.va, A0.va)


def test_pattern_nnz_independent_of_m(oracle_lib):
    """Section 4.1: a fixed p gives a fixed pattern, so nnz does not change with m."""
    L, U = oracle_lib.ilu0(synth.laplace3d(12))
    for p in (1, 2, 3):
        counts = {oracle_lib.sait(L, p + m + 1, "pattern", 0.0, p).nnz for m in (1, 3, 6)}
        assert len(counts) == 1


def test_pattern_of_t_power(oracle_lib):
    """Section 3: pattern(T^p) = pattern(M_{p+1}) (structural, no cancellation)."""
    L, _ = oracle_lib.ilu0(synth.laplace3d(8))
    Ls = L.to_scipy()
    P = Ls.copy()
    for p in (1, 2, 3):
        M = oracle_lib.sait(L, p + 1, "none")
        Ms = M.to_scipy()
        assert (P != 0).astype(int).nnz == Ms.nnz
        assert abs(abs(P.sign()) - abs(Ms.sign())).nnz == 0
        P = P @ Ls


# --------------------------------------------------------------------------
# Drop-rule invariants (Section 3).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("rule,tau", [("abs", 0.01), ("abs", 0.05), ("rowrel", 0.02)])
def test_drop_invariants(oracle_lib, rule, tau):
    A = synth.convdiff3d(14)
    L, U = oracle_lib.ilu0(A)
    for T in (L, U):
        M = oracle_lib.sait(T, 5, rule, tau)
        rows = np.repeat(np.arange(T.n), np.diff(M.rp))
        d = T.to_scipy().diagonal()
        MD = M.va * d[M.ci]                     # undo the final column scaling
        diag = M.ci == rows
        assert np.allclose(MD[diag], 1.0, rtol=0, atol=1e-15)
        rowmax = np.zeros(T.n)
        np.maximum.at(rowmax, rows, np.abs(MD))
        thr = tau * (rowmax[rows] if rule == "rowrel" else np.ones(len(rows)))
        assert np.all(np.abs(MD[~diag]) >= thr[~diag] * (1 - 1e-12))
        assert np.all(M.va >= 0)               # M-matrix factors: T~ >= 0, so M >= 0


# --------------------------------------------------------------------------
# ILU(0): (LU)_ij = a_ij on the pattern of A; exact LU on a full pattern and
# on a tridiagonal matrix (closed form d_i = (i+2)/(i+1) for tridiag(-1,2,-1)).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("make", [lambda: synth.poisson2d(9), lambda: synth.convdiff3d(6),
                                  lambda: synth.varcoef3d(5, 1.0, 3)])
def test_ilu0_reproduces_a_on_its_pattern(oracle_lib, make):
    A = make()
    L, U = oracle_lib.ilu0(A)
    LU = (L.to_scipy() @ U.to_scipy()).toarray()
    Ad = A.to_dense()
    mask = Ad != 0
    assert np.abs(LU[mask] - Ad[mask]).max() <= 1e-13 * np.abs(Ad).max()
    assert np.allclose(np.diag(L.to_dense()), 1.0)
    assert np.count_nonzero(np.triu(L.to_dense(), 1)) == 0
    assert np.count_nonzero(np.tril(U.to_dense(), -1)) == 0


def test_ilu0_full_pattern_is_exact_lu(oracle_lib):
    rng = np.random.default_rng(4)
    n = 30
    Ad = rng.uniform(-1, 1, (n, n)) + n * np.eye(n)
    L, U = oracle_lib.ilu0(synth.from_dense(Ad))
    assert np.abs(L.to_dense() @ U.to_dense() - Ad).max() <= 1e-12 * n


def test_ilu0_tridiagonal_closed_form(oracle_lib):
    n = 50
    Ad = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    _, U = oracle_lib.ilu0(synth.from_dense(Ad))
    i = np.arange(n)
    assert np.allclose(np.diag(U.to_dense()), (i + 2) / (i + 1), rtol=1e-15, atol=0)


# --------------------------------------------------------------------------
# ILU(p) (level of fill, Saad Algorithm 10.5): p = 0 is ILU(0) bit for bit;
# p >= n is the complete LU; LU = A on the ILU(p) pattern; the level-1 fill of
# the 5- and 7-point stencils in closed form; the paper's level-1 columns.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("make", [lambda: synth.poisson2d(9), lambda: synth.convdiff3d(6),
                                  lambda: synth.varcoef3d(5, 1.0, 3), lambda: synth.aniso2d(11, 0.01)])
def test_iluk_level0_is_ilu0(oracle_lib, make):
    A = make()
    L0, U0 = oracle_lib.ilu0(A)
    L, U = oracle_lib.iluk(A, 0)
    for X, Y in ((L, L0), (U, U0)):
        assert np.array_equal(X.rp, Y.rp) and np.array_equal(X.ci, Y.ci)
        assert np.array_equal(X.va, Y.va)          # same fma chains


def test_iluk_complete_is_exact_lu(oracle_lib):
    rng = np.random.default_rng(5)
    n = 40
    Ad = np.where(rng.uniform(size=(n, n)) < 0.1, rng.uniform(-1, 1, (n, n)), 0.0) + n * np.eye(n)
    L, U = oracle_lib.iluk(synth.from_dense(Ad), n)
    assert np.abs(L.to_dense() @ U.to_dense() - Ad).max() <= 1e-12 * n
    y = sla.solve_triangular(L.to_dense(), np.ones(n), lower=True)
    x = sla.solve_triangular(U.to_dense(), y, lower=False)
    assert np.allclose(x, np.linalg.solve(Ad, np.ones(n)), rtol=1e-12, atol=0)


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("make", [lambda: synth.poisson2d(9), lambda: synth.convdiff3d(6),
                                  lambda: synth.varcoef3d(5, 1.0, 3)])
def test_iluk_reproduces_a_on_its_pattern(oracle_lib, make, p):
    """Incomplete LU on a pattern P leaves LU - A zero on P (Saad, Proposition 10.3's setting)."""
    A = make()
    L, U, LUc, lev = oracle_lib.iluk(A, p, levels=True)
    LU = L.to_dense() @ U.to_dense()
    Ad = A.to_dense()
    P = LUc.to_dense() != 0
    P[np.arange(A.n), np.arange(A.n)] = True
    assert np.abs(LU[P] - Ad[P]).max() <= 1e-13 * np.abs(Ad).max()
    # the levels: A's pattern is level 0, every other stored entry is fill of level 1..p
    rows = np.repeat(np.arange(A.n), np.diff(LUc.rp))
    in_a = Ad[rows, LUc.ci] != 0
    assert np.all(lev[in_a] == 0) and np.all((lev[~in_a] >= 1) & (lev[~in_a] <= p))


def test_iluk_level1_fill_closed_form(oracle_lib):
    """Level-1 fill of the natural-order 5-point (g x g) and 7-point (N^3) stencils:
    products of one L offset and one U offset, at grid points that exist."""
    g = 13
    L, U = oracle_lib.iluk(synth.poisson2d(g), 1)
    assert L.nnz == g * g + 2 * g * (g - 1) + (g - 1) ** 2     # diagonal, -1, -g, -(g-1)
    assert U.nnz == L.nnz
    rows = np.repeat(np.arange(L.n), np.diff(L.rp))
    assert set(np.unique(rows - L.ci)) == {0, 1, g, g - 1}
    N = 9
    L, U = oracle_lib.iluk(synth.laplace3d(N), 1)
    assert L.nnz == N ** 3 + 3 * N * N * (N - 1) + 3 * N * (N - 1) ** 2
    rows = np.repeat(np.arange(L.n), np.diff(L.rp))
    assert set(np.unique(rows - L.ci)) == {0, 1, N, N * N, N - 1, N * N - 1, N * N - N}


@pytest.fixture(scope="module")
def laplace100_level1(oracle_lib):
    A = synth.laplace3d(100)
    L, U = oracle_lib.iluk(A, 1)
    return A, L, U


@pytest.fixture(scope="module")
def golden_level1():
    with open(os.path.join(GOLDEN, "paper_runtime_sait_level1.json")) as f:
        return json.load(f)


@pytest.mark.slow
def test_paper_ratios_level1(oracle_lib, laplace100_level1, golden_level1):
    """Table runtime_SAIT, level-1 ILU columns: the nnz ratios of SAIT_Thr and SAIT_Pat."""
    A, L, U = laplace100_level1
    assert L.nnz == 100 ** 3 + 3 * 100 ** 2 * 99 + 3 * 100 * 99 ** 2 == 6_910_300
    m = golden_level1["loop_iterations_m"]
    for row in golden_level1["sait_thr"]:
        M = oracle_lib.sait(L, m + 1, "abs", row["tau"])
        assert round(M.nnz / L.nnz, 2) == row["ratio"], row
    for row in golden_level1["sait_pat"]:
        M = oracle_lib.sait(U, row["p"] + m + 1, "pattern", 0.0, row["p"])
        assert round(M.nnz / U.nnz, 2) == row["ratio"], row


@pytest.mark.slow
def test_paper_pcg_iteration_counts_level1(oracle_lib, laplace100_level1, golden_level1):
    """Exact ILU(1) substitution (the commented-out row of Table runtime_SAIT) and four
    Jacobi sweeps on the level-1 factors (Table runtime_Jacobi); b ~ U[0,1) as for level 0."""
    A, L, U = laplace100_level1
    b = synth.uniform(synth.SEED_BASE, A.n, 0.0, 1.0)
    tol = golden_level1["pcg_tol"]
    _, it, rr, st = oracle_lib.pcg(A, b, "ilu", L, U, tol=tol)
    assert st == 0 and rr <= tol
    assert abs(it - golden_level1["exact_ilu1_pcg_iters"]) <= 3
    _, it4, rr4, st4 = oracle_lib.pcg(A, b, "jacobi4", L, U, tol=tol)
    assert st4 == 0 and rr4 <= tol
    ref = golden_level1["jacobi_level1_pcg_iters"]["4"]
    assert abs(it4 - ref) <= 0.05 * ref
    assert it < it4      # the exact substitution needs the fewest iterations


# --------------------------------------------------------------------------
# Apply, substitution, SpMV, solvers against dense direct solves.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("lower", [True, False])
def test_trisolve_matches_lapack(oracle_lib, lower):
    T = synth.random_triangular(200, lower, 9, max_row=30, long_frac=0.05, long_row=150)
    b = synth.uniform(1, 200)
    x = oracle_lib.trisolve(T, b, lower)
    ref = sla.solve_triangular(T.to_dense(), b, lower=lower)
    assert np.abs(x - ref).max() <= 1e-13 * max(1, np.abs(ref).max())


def test_spmv_and_apply_match_dense(oracle_lib):
    L, U = oracle_lib.ilu0(synth.convdiff3d(7))
    ML = oracle_lib.sait(L, 4, "rowrel", 1e-3)
    MU = oracle_lib.sait(U, 4, "rowrel", 1e-3)
    r = synth.uniform(2, L.n)
    z = oracle_lib.apply(ML, MU, r)
    assert np.abs(z - MU.to_dense() @ (ML.to_dense() @ r)).max() <= 1e-13 * np.abs(z).max()
    # with the exact inverses, the apply equals the two substitutions
    MLx = oracle_lib.sait(L, L.n, "none")
    MUx = oracle_lib.sait(U, U.n, "none")
    ze = oracle_lib.apply(MLx, MUx, r)
    zt = oracle_lib.trisolve(U, oracle_lib.trisolve(L, r, True), False)
    assert np.abs(ze - zt).max() <= 1e-12 * np.abs(zt).max()


def _nonsym(n, seed):
    rng = np.random.default_rng(seed)
    Ad = np.zeros((n, n))
    for i in range(n):
        cols = rng.choice(n, size=5, replace=False)
        Ad[i, cols] = rng.uniform(-1, 1, 5)
        Ad[i, i] = 3.0 + rng.uniform(0, 1)
    return Ad


@pytest.mark.parametrize("prec", ["none", "sait", "ilu"])
def test_gmres_full_restart_matches_dense_solve(oracle_lib, prec):
    n = 60
    Ad = _nonsym(n, 3)
    A = synth.from_dense(Ad)
    L, U = oracle_lib.ilu0(A)
    ML, MU = oracle_lib.sait(L, 3, "rowrel", 1e-3), oracle_lib.sait(U, 3, "rowrel", 1e-3)
    lo, up = (ML, MU) if prec == "sait" else (L, U)
    b = synth.uniform(4, n)
    x, it, rr, st = oracle_lib.gmres(A, b, prec, lo, up, restart=n, tol=1e-12)
    ref = np.linalg.solve(Ad, b)
    assert st == 0 and rr <= 1e-12 and it <= n
    assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("restart", [5, 30])
def test_gmres_restarted_converges(oracle_lib, restart):
    A = synth.convdiff3d(10)
    L, U = oracle_lib.ilu0(A)
    ML, MU = oracle_lib.sait(L, 3, "rowrel", 1e-3), oracle_lib.sait(U, 3, "rowrel", 1e-3)
    xt = synth.uniform(5, A.n)
    b = A.to_scipy() @ xt
    x, it, rr, st = oracle_lib.gmres(A, b, "sait", ML, MU, restart=restart, tol=1e-8)
    assert st == 0 and rr <= 1e-8
    assert np.linalg.norm(b - A.to_scipy() @ x) <= 1e-8 * np.linalg.norm(b)


@pytest.mark.parametrize("prec", ["none", "sait", "ilu"])
def test_bicgstab_matches_dense_solve(oracle_lib, prec):
    n = 80
    Ad = _nonsym(n, 8)
    A = synth.from_dense(Ad)
    L, U = oracle_lib.ilu0(A)
    ML, MU = oracle_lib.sait(L, 3, "rowrel", 1e-3), oracle_lib.sait(U, 3, "rowrel", 1e-3)
    lo, up = (ML, MU) if prec == "sait" else (L, U)
    b = synth.uniform(6, n)
    x, it, rr, st = oracle_lib.bicgstab(A, b, prec, lo, up, tol=1e-12)
    assert st == 0 and rr <= 1e-12
    ref = np.linalg.solve(Ad, b)
    assert np.abs(x - ref).max() <= 1e-9 * np.abs(ref).max()


def test_pcg_matches_dense_solve(oracle_lib):
    A = synth.varcoef3d(6, 1.0, 2)
    L, U = oracle_lib.ilu0(A)
    b = synth.uniform(7, A.n)
    x, it, rr, st = oracle_lib.pcg(A, b, "ilu", L, U, tol=1e-12)
    ref = np.linalg.solve(A.to_dense(), b)
    assert st == 0 and rr <= 1e-12
    assert np.abs(x - ref).max() <= 1e-9 * np.abs(ref).max()


# --------------------------------------------------------------------------
# Error behaviour.
# --------------------------------------------------------------------------
def test_errors(oracle_lib):
    bad = synth.from_dense(np.array([[1.0, 2.0], [3.0, 4.0]]))
    with pytest.raises(oracle_lib.OracleError) as e:
        oracle_lib.sait(bad, 3)
    assert e.value.code == 2
    zero = synth.from_dense(np.array([[1.0, 0.0], [3.0, 0.0]]))
    with pytest.raises(oracle_lib.OracleError) as e:
        oracle_lib.sait(zero, 3)
    assert e.value.code == 3
    M = oracle_lib.sait(synth.from_dense(np.diag([2.0, 4.0])), 1)
    assert np.allclose(M.to_dense(), np.diag([0.5, 0.25]))


# --------------------------------------------------------------------------
# LOBPCG (Knyazev 2001; the paper's eigenvalue solver, Section 4.4) and its
# dense helper.
# --------------------------------------------------------------------------
def test_sym_eig_matches_lapack(oracle_lib):
    rng = np.random.default_rng(8)
    for m in (1, 2, 7, 31):
        B = rng.standard_normal((m, m))
        Cm = B + B.T
        w, V = oracle_lib.sym_eig(Cm)
        assert np.abs(w - np.linalg.eigvalsh(Cm)).max() <= 1e-13 * max(1.0, np.abs(w).max())
        assert np.abs(Cm @ V - V * w).max() <= 1e-12 * max(1.0, np.abs(w).max())
        assert np.abs(V.T @ V - np.eye(m)).max() <= 1e-13


def laplace_eigs(N, k):
    """Eigenvalues of the h^2-scaled 7-point Laplacian on N^3: sum_d 4 sin^2(j_d pi / (2(N+1)))."""
    j = np.arange(1, N + 1)
    l1 = 4 * np.sin(j * np.pi / (2 * (N + 1))) ** 2
    return np.sort((l1[:, None, None] + l1[None, :, None] + l1[None, None, :]).ravel())[:k]


@pytest.mark.parametrize("prec", ["none", "sait", "ilu"])
def test_lobpcg_laplace_closed_form(oracle_lib, prec):
    N, k = 10, 16                       # the 16th eigenvalue sits inside a degenerate cluster
    A = synth.laplace3d(N)
    L, U = oracle_lib.ilu0(A)
    lo, up = ((oracle_lib.sait(L, 3, "rowrel", 1e-3), oracle_lib.sait(U, 3, "rowrel", 1e-3))
              if prec == "sait" else (L, U))
    X0 = synth.uniform(5, (A.n, k))
    lam, X, it, rr, st = oracle_lib.lobpcg(A, X0, prec, lo, up, tol=1e-8, maxit=500)
    assert st == 0 and rr <= 1e-8
    assert np.abs(lam - laplace_eigs(N, k)).max() <= 1e-12 * lam.max()
    assert np.abs(X.T @ X - np.eye(k)).max() <= 1e-10
    R = A.to_scipy() @ X - X * lam
    assert np.all(np.linalg.norm(R, axis=0) <= 1e-8 * lam * 1.0001)


def test_lobpcg_variable_coefficients_dense(oracle_lib):
    A = synth.varcoef3d(7, 1.0, 3)
    k = 6
    lam, X, it, rr, st = oracle_lib.lobpcg(A, synth.uniform(6, (A.n, k)), tol=1e-9, maxit=1000)
    ref = np.linalg.eigvalsh(A.to_dense())[:k]
    assert st == 0
    assert np.abs(lam - ref).max() <= 1e-12 * ref.max()
