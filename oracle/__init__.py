"""SAIT oracle (test infrastructure only).

Plain FP64 CPU implementations, written from the paper (Z. Lu, arXiv
2106.12836) and the textbook algorithms it cites, of everything the GPU path
computes: ILU(0), level-of-fill ILU(p) and ILUT factors, the SAIT series with its dropping rules
(Algorithms 1-3), the preconditioner apply z = M_U (M_L r) (Section 3.1), exact
substitution, and the GMRES / BiCGSTAB / PCG solvers.  The arithmetic lives in
``sait_oracle.c`` (compiled with gcc, ``-ffp-contract=off``); this module only
marshals numpy arrays.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
and never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

from synth import CSR

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sait_oracle.c")
_LIB = os.path.join(_HERE, "libsait_oracle.so")

DROP = {"none": 0, "abs": 1, "rowrel": 2, "pattern": 3, "hybrid": 4}
STATUS = {0: "ok", 1: "invalid argument", 2: "not triangular", 3: "zero pivot",
          4: "out of memory", 5: "not converged", 6: "breakdown"}


class OracleError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn}: {STATUS.get(code, code)}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle's C source into a shared library next to it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Mat(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("cap", C.c_int64),
                ("rp", C.POINTER(C.c_int32)), ("ci", C.POINTER(C.c_int32)),
                ("va", C.POINTER(C.c_double))]


class _Prec(C.Structure):
    _fields_ = [("kind", C.c_int), ("n", C.c_int64),
                ("l_rp", C.c_void_p), ("l_ci", C.c_void_p), ("l_va", C.c_void_p),
                ("u_rp", C.c_void_p), ("u_ci", C.c_void_p), ("u_va", C.c_void_p),
                ("sweeps", C.c_int)]


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        i64, i32p, dp, vp = C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p
        _lib.ora_spmv.argtypes = [i64, i32p, i32p, dp, dp, dp]
        _lib.ora_trisolve.argtypes = [i64, i32p, i32p, dp, C.c_int, dp, dp]
        _lib.ora_ilu0.argtypes = [i64, i32p, i32p, dp]
        _lib.ora_sait.argtypes = [i64, i32p, i32p, dp, C.c_int, C.c_int, C.c_double, C.c_int,
                                  C.POINTER(_Mat)]
        _lib.ora_free.argtypes = [C.POINTER(_Mat)]
        _lib.ora_jacobi.argtypes = [i64, i32p, i32p, dp, C.c_int, dp, dp]
        _lib.ora_ilut.argtypes = [i64, i32p, i32p, dp, C.c_double, C.c_int, C.POINTER(_Mat)]
        _lib.ora_iluk.argtypes = [i64, i32p, i32p, dp, C.c_int, C.POINTER(_Mat),
                                  C.POINTER(C.POINTER(C.c_int32))]
        _lib.ora_free_i32.argtypes = [C.POINTER(C.c_int32)]
        solver = [i64, i32p, i32p, dp, C.POINTER(_Prec), dp, dp]
        _lib.ora_gmres.argtypes = solver + [C.c_int, C.c_double, C.c_int,
                                            C.POINTER(C.c_int), C.POINTER(C.c_double)]
        _lib.ora_bicgstab.argtypes = solver + [C.c_double, C.c_int,
                                               C.POINTER(C.c_int), C.POINTER(C.c_double)]
        _lib.ora_pcg.argtypes = solver + [C.c_double, C.c_int,
                                          C.POINTER(C.c_int), C.POINTER(C.c_double)]
        _lib.ora_lobpcg.argtypes = [i64, i32p, i32p, dp, C.POINTER(_Prec), C.c_int, dp, dp, C.c_double,
                                    C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)]
        _lib.ora_sym_eig.argtypes = [C.c_int, dp, dp, dp]
        for f in ("ora_trisolve", "ora_ilu0", "ora_sait", "ora_gmres", "ora_bicgstab", "ora_pcg",
                  "ora_lobpcg", "ora_sym_eig"):
            getattr(_lib, f).restype = C.c_int
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _csr_args(A: CSR):
    rp = np.ascontiguousarray(A.rp, dtype=np.int32)
    ci = np.ascontiguousarray(A.ci, dtype=np.int32)
    va = np.ascontiguousarray(A.va, dtype=np.float64)
    return rp, ci, va


def spmv(A: CSR, x: np.ndarray) -> np.ndarray:
    rp, ci, va = _csr_args(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(A.n)
    _L().ora_spmv(A.n, _p(rp), _p(ci), _p(va), _p(x), _p(y))
    return y


def trisolve(T: CSR, b: np.ndarray, lower: bool) -> np.ndarray:
    rp, ci, va = _csr_args(T)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty(T.n)
    st = _L().ora_trisolve(T.n, _p(rp), _p(ci), _p(va), int(lower), _p(b), _p(x))
    if st:
        raise OracleError("trisolve", st)
    return x


def ilu0(A: CSR) -> tuple[CSR, CSR]:
    """Level-0 ILU factors: L unit lower (diagonal 1 stored), U upper with diagonal."""
    rp, ci, va = _csr_args(A)
    lu = va.copy()
    st = _L().ora_ilu0(A.n, _p(rp), _p(ci), _p(lu))
    if st:
        raise OracleError("ilu0", st)
    return split_lu(CSR(A.n, rp, ci, lu))


def _take(out) -> CSR:
    try:
        n, nnz = out.n, out.nnz
        orp = np.ctypeslib.as_array(out.rp, shape=(n + 1,)).copy()
        if nnz:
            oci = np.ctypeslib.as_array(out.ci, shape=(nnz,)).copy()
            ova = np.ctypeslib.as_array(out.va, shape=(nnz,)).copy()
        else:
            oci, ova = np.zeros(0, np.int32), np.zeros(0)
    finally:
        _L().ora_free(C.byref(out))
    return CSR(int(n), orp, oci, ova)


def ilut(A: CSR, tau: float, lfil: int) -> tuple[CSR, CSR]:
    """ILUT(tau, lfil) factors (Saad, Algorithm 10.6), split as ilu0's."""
    rp, ci, va = _csr_args(A)
    out = _Mat()
    st = _L().ora_ilut(A.n, _p(rp), _p(ci), _p(va), float(tau), int(lfil), C.byref(out))
    if st:
        raise OracleError("ilut", st)
    return split_lu(_take(out))


def iluk(A: CSR, p: int, levels: bool = False):
    """Level-of-fill ILU(p) factors (Saad, Algorithm 10.5), split as ilu0's.

    With levels=True also returns the level of fill of every entry of the
    combined factor (strict L part, then U with its diagonal, CSR order)."""
    rp, ci, va = _csr_args(A)
    out = _Mat()
    lev = C.POINTER(C.c_int32)()
    st = _L().ora_iluk(A.n, _p(rp), _p(ci), _p(va), int(p), C.byref(out), C.byref(lev))
    if st:
        raise OracleError("iluk", st)
    nnz = int(out.nnz)
    try:
        lv = np.ctypeslib.as_array(lev, shape=(nnz,)).copy() if nnz else np.zeros(0, np.int32)
    finally:
        _L().ora_free_i32(lev)
    LU = _take(out)
    L, U = split_lu(LU)
    return (L, U, LU, lv) if levels else (L, U)


def split_lu(LU: CSR) -> tuple[CSR, CSR]:
    """Split combined ILU storage into L (strict part plus a stored unit diagonal) and U."""
    n = LU.n
    rows = np.repeat(np.arange(n), np.diff(LU.rp))
    lo = LU.ci < rows
    up = LU.ci >= rows
    # L: strict-lower entries, then the unit diagonal (columns stay ascending)
    lcnt = np.bincount(rows[lo], minlength=n) + 1
    lrp = np.zeros(n + 1, np.int64)
    lrp[1:] = np.cumsum(lcnt)
    lci = np.empty(lrp[-1], np.int32)
    lva = np.empty(lrp[-1])
    diag_pos = lrp[1:] - 1
    mask = np.ones(lrp[-1], bool)
    mask[diag_pos] = False
    lci[mask] = LU.ci[lo]
    lva[mask] = LU.va[lo]
    lci[diag_pos] = np.arange(n)
    lva[diag_pos] = 1.0
    ucnt = np.bincount(rows[up], minlength=n)
    urp = np.zeros(n + 1, np.int64)
    urp[1:] = np.cumsum(ucnt)
    L = CSR(n, lrp.astype(np.int32), lci, lva)
    U = CSR(n, urp.astype(np.int32), LU.ci[up].astype(np.int32), LU.va[up].copy())
    return L, U


def sait(T: CSR, m_terms: int, drop: str = "none", tau: float = 0.0, p: int = 0) -> CSR:
    """SAIT matrix M ~ T^-1 with ``m_terms`` series terms and the given dropping rule."""
    rp, ci, va = _csr_args(T)
    out = _Mat()
    st = _L().ora_sait(T.n, _p(rp), _p(ci), _p(va), int(m_terms), DROP[drop], float(tau),
                       int(p), C.byref(out))
    if st:
        raise OracleError("sait", st)
    try:
        n, nnz = out.n, out.nnz
        orp = np.ctypeslib.as_array(out.rp, shape=(n + 1,)).copy()
        if nnz:
            oci = np.ctypeslib.as_array(out.ci, shape=(nnz,)).copy()
            ova = np.ctypeslib.as_array(out.va, shape=(nnz,)).copy()
        else:
            oci, ova = np.zeros(0, np.int32), np.zeros(0)
    finally:
        _L().ora_free(C.byref(out))
    return CSR(int(n), orp, oci, ova)


def apply(ML: CSR, MU: CSR, r: np.ndarray) -> np.ndarray:
    """SAIT preconditioner apply z = M_U (M_L r) (Section 3.1)."""
    return spmv(MU, spmv(ML, r))


def _prec(kind: str, lo: CSR | None, up: CSR | None, n: int):
    """kind: "none", "sait", "ilu" or "jacobiK" (K Jacobi sweeps per triangle)."""
    P = _Prec()
    if kind.startswith("jacobi"):
        P.kind, P.sweeps = 3, int(kind[6:])
    else:
        P.kind = {"none": 0, "sait": 1, "ilu": 2}[kind]
    P.n = n
    keep = []
    if kind != "none":
        for pre, M in (("l", lo), ("u", up)):
            rp, ci, va = _csr_args(M)
            keep += [rp, ci, va]
            setattr(P, pre + "_rp", rp.ctypes.data)
            setattr(P, pre + "_ci", ci.ctypes.data)
            setattr(P, pre + "_va", va.ctypes.data)
    return P, keep


def _solve(fn, A: CSR, b, x0, prec, lo, up, *extra):
    rp, ci, va = _csr_args(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(A.n) if x0 is None else np.array(x0, dtype=np.float64)
    P, keep = _prec(prec, lo, up, A.n)
    it = C.c_int(0)
    rr = C.c_double(0.0)
    st = fn(A.n, _p(rp), _p(ci), _p(va), C.byref(P), _p(b), _p(x), *extra, C.byref(it), C.byref(rr))
    del keep
    return x, int(it.value), float(rr.value), int(st)


def gmres(A: CSR, b, prec: str = "none", lo: CSR | None = None, up: CSR | None = None,
          restart: int = 30, tol: float = 1e-8, maxit: int = 10000, x0=None):
    """Right-preconditioned GMRES(restart).  Returns (x, iterations, true relres, status)."""
    return _solve(_L().ora_gmres, A, b, x0, prec, lo, up, C.c_int(restart), C.c_double(tol),
                  C.c_int(maxit))


def bicgstab(A: CSR, b, prec: str = "none", lo: CSR | None = None, up: CSR | None = None,
             tol: float = 1e-8, maxit: int = 10000, x0=None):
    """Right-preconditioned BiCGSTAB.  Returns (x, iterations, true relres, status)."""
    return _solve(_L().ora_bicgstab, A, b, x0, prec, lo, up, C.c_double(tol), C.c_int(maxit))


def jacobi(T: CSR, b, sweeps: int) -> np.ndarray:
    """``sweeps`` Jacobi iterations for T x = b from x = 0 (equation Jacobi_iter)."""
    rp, ci, va = _csr_args(T)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(T.n)
    st = _L().ora_jacobi(T.n, _p(rp), _p(ci), _p(va), int(sweeps), _p(b), _p(x))
    if st:
        raise OracleError("jacobi", st)
    return x


def pcg(A: CSR, b, prec: str = "none", lo: CSR | None = None, up: CSR | None = None,
        tol: float = 1e-10, maxit: int = 10000, x0=None):
    """Preconditioned CG (the paper's solver).  Returns (x, iterations, true relres, status)."""
    return _solve(_L().ora_pcg, A, b, x0, prec, lo, up, C.c_double(tol), C.c_int(maxit))


def lobpcg(A: CSR, X0: np.ndarray, prec: str = "none", lo: CSR | None = None, up: CSR | None = None,
           tol: float = 1e-8, maxit: int = 500):
    """k smallest eigenpairs of SPD A by LOBPCG.  Returns (lambda, X, iterations, max residual, status)."""
    rp, ci, va = _csr_args(A)
    X = np.array(X0, dtype=np.float64, order="C")
    k = X.shape[1]
    lam = np.zeros(k)
    P, keep = _prec(prec, lo, up, A.n)
    it = C.c_int(0)
    rr = C.c_double(0.0)
    st = _L().ora_lobpcg(A.n, _p(rp), _p(ci), _p(va), C.byref(P), k, _p(X), _p(lam), C.c_double(tol),
                         C.c_int(maxit), C.byref(it), C.byref(rr))
    del keep
    return lam, X, int(it.value), float(rr.value), int(st)


def sym_eig(Cm: np.ndarray):
    """Eigenvalues (ascending) and eigenvectors of a small symmetric matrix (cyclic Jacobi)."""
    Cc = np.array(Cm, dtype=np.float64, order="C")
    m = Cc.shape[0]
    w = np.zeros(m)
    V = np.zeros((m, m))
    _L().ora_sym_eig(m, _p(Cc), _p(w), _p(V))
    return w, V
