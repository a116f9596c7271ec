"""CPU FP64 oracle for SLD-deflated Jacobi-PCG -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product path (the CUDA library and its binding) never loads it.

The arithmetic lives in ``sld_oracle.c`` (plain C, FP64, no FMA contraction);
this module compiles it with gcc and marshals numpy arrays through ctypes.
Paper: arXiv:1510.02148, Section 2 (pressure equation), Section 3.1
(Def. 3.1, eqs. (E), (deflops), (defsplit), (defsys), (projectback)),
Section 3.2.2 (eq. (domdefl), subdomain-levelset deflation).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sld_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_NOT_CONVERGED, ERR_BREAKDOWN, ERR_SINGULAR, ERR_OOM = 0, 1, 3, 4, 5, 7
BC_NOFLOW, BC_DIRICHLET = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle (OpenMP if the compiler supports it)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _SRC,
            "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            lib.oracle_assemble.argtypes = [C.c_int, C.c_int, C.c_int, P, P, P, P, P, P, P, P, P]
            lib.oracle_spmv.argtypes = [C.c_int64, P, P, P, P, P]
            lib.oracle_spmv.restype = None
            lib.oracle_labels.argtypes = [C.c_int, C.c_int, C.c_int, P, C.c_int, C.c_int,
                                          C.c_int, P, C.c_int, P]
            lib.oracle_coarse.argtypes = [C.c_int64, P, P, P, P, C.c_int, P, C.c_int, P, P]
            lib.oracle_restrict.argtypes = [C.c_int64, P, C.c_int, P, C.c_int, P, P]
            lib.oracle_cholesky.argtypes = [C.c_int, P, P]
            lib.oracle_dpcg.argtypes = [C.c_int64, P, P, P, P, P, C.c_int, P, C.c_int,
                                        C.c_double, C.c_int, P, P, P, P, P]
            lib.oracle_set_threads.argtypes = [C.c_int]
            lib.oracle_set_threads.restype = None
            lib.oracle_max_threads.restype = C.c_int
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def set_threads(t: int) -> None:
    _load().oracle_set_threads(int(t))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


class CSR:
    """The assembled pressure matrix (CSR, columns ascending) and rhs."""

    def __init__(self, n, rowptr, col, val, b, is_dirichlet, shape3):
        self.n, self.rowptr, self.col, self.val = n, rowptr, col, val
        self.b, self.is_dirichlet, self.shape3 = b, is_dirichlet, shape3

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))

    def dense(self):
        return self.to_scipy().toarray()

    def spmv(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(self.n)
        _load().oracle_spmv(self.n, _p(self.rowptr), _p(self.col), _p(self.val), _p(x), _p(y))
        return y

    def diag(self):
        d = np.zeros(self.n)
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        m = self.col == rows
        d[rows[m]] = self.val[m]
        return d


def assemble(K, q=None, bc_type=(1, 1, 0, 0, 0, 0), bc_value=(1.0, 0.0, 0, 0, 0, 0)) -> CSR:
    """TPFA assembly of -div(K grad p) = q on unit cells (K shaped (nz, ny, nx))."""
    K = np.ascontiguousarray(K, dtype=np.float64)
    nz, ny, nx = K.shape
    n = K.size
    qq = None if q is None else np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    bct = np.ascontiguousarray(bc_type, dtype=np.int32)
    bcv = np.ascontiguousarray(bc_value, dtype=np.float64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(7 * n, dtype=np.int32)
    val = np.zeros(7 * n, dtype=np.float64)
    b = np.zeros(n)
    isd = np.zeros(n, dtype=np.uint8)
    st = _load().oracle_assemble(nx, ny, nz, _p(K), _p(qq), _p(bct), _p(bcv), _p(rowptr),
                                 _p(col), _p(val), _p(b), _p(isd))
    if st != OK:
        raise ValueError(f"oracle_assemble failed with status {st}")
    nnz = int(rowptr[-1])
    return CSR(n, rowptr, col[:nnz].copy(), val[:nnz].copy(), b, isd, (nz, ny, nx))


def labels(K, S, tau, L) -> np.ndarray:
    """label = subdomain * L + levelset class (int32, flattened x-fastest)."""
    K = np.ascontiguousarray(K, dtype=np.float64)
    nz, ny, nx = K.shape
    Sx, Sy, Sz = S
    tau = np.ascontiguousarray(tau if len(tau) else [0.0], dtype=np.float64)
    out = np.zeros(K.size, dtype=np.int32)
    st = _load().oracle_labels(nx, ny, nz, _p(K), Sx, Sy, Sz, _p(tau), int(L), _p(out))
    if st != OK:
        raise ValueError(f"oracle_labels failed with status {st}")
    return out


def coarse(A: CSR, label, d, Zd=None):
    """E = Z^T A Z and its Cholesky factor (None if E is not SPD)."""
    k = 0 if Zd is None else Zd.shape[1]
    Zd = None if Zd is None else np.ascontiguousarray(Zd, dtype=np.float64)
    lab = None if label is None else np.ascontiguousarray(label, dtype=np.int32)
    m = d + k
    E = np.zeros((m, m))
    Lc = np.zeros((m, m))
    st = _load().oracle_coarse(A.n, _p(A.rowptr), _p(A.col), _p(A.val), _p(lab), d, _p(Zd), k,
                               _p(E), _p(Lc))
    if st not in (OK, ERR_SINGULAR):
        raise ValueError(f"oracle_coarse failed with status {st}")
    return E, (Lc if st == OK else None)


def restrict(label, d, v, Zd=None):
    """s = Z^T v."""
    k = 0 if Zd is None else Zd.shape[1]
    Zd = None if Zd is None else np.ascontiguousarray(Zd, dtype=np.float64)
    lab = None if label is None else np.ascontiguousarray(label, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.float64)
    s = np.zeros(d + k)
    st = _load().oracle_restrict(v.size, _p(lab), d, _p(Zd), k, _p(v), _p(s))
    if st != OK:
        raise ValueError(f"oracle_restrict failed with status {st}")
    return s


def cholesky(E):
    E = np.ascontiguousarray(E, dtype=np.float64)
    Lc = np.zeros_like(E)
    st = _load().oracle_cholesky(E.shape[0], _p(E), _p(Lc))
    return Lc if st == OK else None


class Result:
    def __init__(self, x, iterations, true_relres, status, hist, ztr_max):
        self.x, self.iterations, self.true_relres = x, iterations, true_relres
        self.status, self.hist, self.ztr_max = status, hist, ztr_max


def dpcg(A: CSR, label=None, d=0, b=None, tol=1e-9, maxiter=20000, Zd=None,
         history=False) -> Result:
    """Deflated Jacobi-PCG solve of A x = b (b defaults to the assembled rhs)."""
    b = A.b if b is None else np.ascontiguousarray(b, dtype=np.float64)
    k = 0 if Zd is None else Zd.shape[1]
    Zd = None if Zd is None else np.ascontiguousarray(Zd, dtype=np.float64)
    lab = None if label is None else np.ascontiguousarray(label, dtype=np.int32)
    x = np.zeros(A.n)
    it = C.c_int(0)
    rr = C.c_double(0)
    zt = C.c_double(0)
    hist = np.zeros(maxiter + 1) if history else None
    st = _load().oracle_dpcg(A.n, _p(A.rowptr), _p(A.col), _p(A.val), _p(b), _p(lab), d,
                             _p(Zd), k, float(tol), int(maxiter), _p(x), C.byref(it),
                             C.byref(rr), _p(hist), C.byref(zt))
    if st not in (OK, ERR_NOT_CONVERGED, ERR_BREAKDOWN):
        raise RuntimeError(f"oracle_dpcg failed with status {st}")
    # ERR_BREAKDOWN (p^T w <= 0) only happens at the roundoff floor of a
    # tolerance tighter than FP64 can reach; x is then the last iterate and
    # the caller sees the status.
    if hist is not None:
        hist = hist[: it.value + 1]
    return Result(x, it.value, rr.value, st, hist, zt.value)
