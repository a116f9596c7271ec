"""Python binding of libsld (include/sld.h): argument marshalling only.

Every array may be a numpy array (host) or a torch tensor (host or CUDA);
the library tells host and device pointers apart.  Nothing here computes
any step of the method: the library's kernels do.  If libsld.so is missing
or cannot load, every entry point raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsld.so")

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_NOT_CONVERGED, ERR_BREAKDOWN = 0, 1, 2, 3, 4
ZEXTRA_F64, ZEXTRA_F32 = 0, 1
ERR_COARSE_SINGULAR, ERR_TIMEOUT, ERR_OOM, ERR_STATE = 5, 6, 7, 8
STATUS_NAMES = {0: "SLD_OK", 1: "SLD_ERR_INVALID_ARG", 2: "SLD_ERR_CUDA", 3: "SLD_ERR_NOT_CONVERGED",
                4: "SLD_ERR_BREAKDOWN", 5: "SLD_ERR_COARSE_SINGULAR", 6: "SLD_ERR_TIMEOUT",
                7: "SLD_ERR_OOM", 8: "SLD_ERR_STATE"}
FP64, FP32_IR, BF16COEF_IR = 0, 1, 2
BC_NOFLOW, BC_DIRICHLET = 0, 1

EXPORTED = ["sld_default_options", "sld_build_system", "sld_make_labels", "sld_build_deflation",
            "sld_solve", "sld_destroy", "sld_last_error", "sld_get_operator", "sld_apply_A",
            "sld_restrict", "sld_get_coarse", "sld_batch_create", "sld_batch_solve",
            "sld_batch_describe", "sld_batch_destroy", "sld_solve_batched", "sld_deflation_info",
            "sld_net_num_params", "sld_net_create", "sld_net_set_params", "sld_net_get_params",
            "sld_net_get_grads", "sld_net_forward", "sld_net_backward", "sld_net_loss_backward",
            "sld_net_adam", "sld_net_destroy", "sld_lanczos_eigvecs", "sld_solve_gmres",
            "sld_make_labels_cc", "sld_harmonic_ritz", "sld_solve_rdgmres", "sld_default_train_options",
            "sld_learned_train", "sld_learned_infer"]


class SldError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int)]


class Bc(C.Structure):
    _fields_ = [("type", C.c_int * 6), ("value", C.c_double * 6)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("tol", C.c_double), ("inner_tol", C.c_double),
                ("maxiter", C.c_int), ("max_outer", C.c_int), ("ctas_per_sm", C.c_int),
                ("timeout_s", C.c_double), ("debug_skip_barrier", C.c_int), ("fwd_tol", C.c_double)]


class Result(C.Structure):
    _fields_ = [("iterations", C.c_int), ("outer_steps", C.c_int), ("true_relres", C.c_double),
                ("recursive_relres", C.c_double), ("solve_ms", C.c_double), ("kernel_path", C.c_int),
                ("fwd_err_estimate", C.c_double)]


class TrainOptions(C.Structure):
    _fields_ = [("epochs", C.c_int), ("lr", C.c_float), ("lr_decay", C.c_float), ("decay_every", C.c_int),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float), ("seed", C.c_uint64)]


class GmresInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("cycles", C.c_int), ("relres_estimate", C.c_double),
                ("true_relres", C.c_double), ("solve_ms", C.c_double)]


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load libsld.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libsld.so not found at {path}; build it first (no CPU fallback)")
        lib = C.CDLL(path)
        P = C.c_void_p
        lib.sld_default_options.argtypes = [C.POINTER(Options)]
        lib.sld_default_options.restype = None
        lib.sld_build_system.argtypes = [P, P, Grid, Bc, P, C.POINTER(P)]
        lib.sld_make_labels.argtypes = [P, C.c_int, C.c_int, C.c_int, P, C.c_int, P]
        lib.sld_build_deflation.argtypes = [P, P, C.c_int, P, C.c_int, C.c_int]
        lib.sld_solve.argtypes = [P, P, C.POINTER(Options), P, C.POINTER(Result)]
        lib.sld_destroy.argtypes = [P]
        lib.sld_destroy.restype = None
        lib.sld_last_error.restype = C.c_char_p
        lib.sld_get_operator.argtypes = [P, P, P, P, P, P]
        lib.sld_apply_A.argtypes = [P, P, P]
        lib.sld_restrict.argtypes = [P, P, P]
        lib.sld_get_coarse.argtypes = [P, P, P]
        lib.sld_batch_create.argtypes = [P, C.c_int, C.POINTER(Options), C.POINTER(P)]
        lib.sld_batch_solve.argtypes = [P, P, P, P]
        lib.sld_batch_describe.argtypes = [P]
        lib.sld_batch_describe.restype = C.c_char_p
        lib.sld_batch_destroy.argtypes = [P]
        lib.sld_batch_destroy.restype = None
        lib.sld_solve_batched.argtypes = [P, C.c_int, P, C.POINTER(Options), P, P]
        lib.sld_deflation_info.argtypes = [P, P, P, P]
        lib.sld_net_num_params.argtypes = []
        lib.sld_net_num_params.restype = C.c_int64
        lib.sld_net_create.argtypes = [C.c_int, C.c_int, C.c_int, P, C.POINTER(P)]
        lib.sld_net_set_params.argtypes = [P, P]
        lib.sld_net_get_params.argtypes = [P, P]
        lib.sld_net_get_grads.argtypes = [P, P]
        lib.sld_net_forward.argtypes = [P, P, P]
        lib.sld_net_backward.argtypes = [P, P]
        lib.sld_net_loss_backward.argtypes = [P, P, C.c_int, P, C.POINTER(C.c_double)]
        lib.sld_net_adam.argtypes = [P, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int]
        lib.sld_net_destroy.argtypes = [P]
        lib.sld_net_destroy.restype = None
        lib.sld_default_train_options.argtypes = [C.POINTER(TrainOptions)]
        lib.sld_default_train_options.restype = None
        lib.sld_learned_train.argtypes = [P, C.c_int, P, P, C.c_int, P, C.POINTER(TrainOptions), P]
        lib.sld_learned_infer.argtypes = [P, P, P]
        lib.sld_lanczos_eigvecs.argtypes = [P, C.c_int, C.c_int, P, P, P]
        lib.sld_make_labels_cc.argtypes = [P, C.c_int, C.c_int, C.c_int, P, C.c_int, P, C.POINTER(C.c_int)]
        lib.sld_solve_rdgmres.argtypes = [P, P, C.c_int, C.c_int, C.c_double, C.c_int, P, C.POINTER(GmresInfo)]
        lib.sld_harmonic_ritz.argtypes = [P, C.c_int, C.c_int, P, P, P]
        lib.sld_solve_gmres.argtypes = [P, P, C.c_int, C.c_int, C.c_double, C.c_int, P, C.POINTER(GmresInfo)]
        for name in ("sld_build_system", "sld_make_labels", "sld_build_deflation", "sld_solve",
                     "sld_get_operator", "sld_apply_A", "sld_restrict", "sld_get_coarse",
                     "sld_batch_create", "sld_batch_solve", "sld_solve_batched"):
            getattr(lib, name).restype = C.c_int
        _lib = lib
        return lib


def _check(st: int):
    if st != OK:
        raise SldError(st, load().sld_last_error().decode())


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype) -> Optional[int]:
    """Data pointer of a contiguous array of the given numpy dtype (or None)."""
    if a is None:
        return None
    if _is_torch(a):
        import torch
        want = {np.float64: torch.float64, np.int32: torch.int32, np.float32: torch.float32}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor")
        return a.data_ptr()
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous:
        raise TypeError(f"expected a C-contiguous numpy array of {np.dtype(dtype)}")
    return a.ctypes.data


def default_options(**kw) -> Options:
    o = Options()
    load().sld_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


@dataclass
class SolveInfo:
    iterations: int
    outer_steps: int
    true_relres: float
    recursive_relres: float
    solve_ms: float
    status: int
    kernel_path: int = 0
    fwd_err_estimate: float = -1.0


class System:
    """A handle on one assembled pressure system (sld_system)."""

    def __init__(self, K, q=None, bc_type=(1, 1, 0, 0, 0, 0), bc_value=(1.0, 0.0, 0, 0, 0, 0),
                 stream: Optional[int] = None, shape: Optional[Sequence[int]] = None):
        lib = load()
        if shape is None:
            shape = tuple(K.shape)
        nz, ny, nx = shape
        self.shape = (nz, ny, nx)
        self.n = nx * ny * nz
        bc = Bc()
        for f in range(6):
            bc.type[f] = int(bc_type[f])
            bc.value[f] = float(bc_value[f])
        h = C.c_void_p()
        self._keep = (K, q)
        _check(lib.sld_build_system(_ptr(K, np.float64), _ptr(q, np.float64), Grid(nx, ny, nz), bc,
                                    stream, C.byref(h)))
        self._h = h
        self.d = 0

    # -- lifetime -------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().sld_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- setup ------------------------------------------------------------
    def make_labels(self, S, tau, L, out=None):
        tau_a = np.ascontiguousarray(tau if len(tau) else [0.0], dtype=np.float64)
        if out is None:
            out = np.empty(self.n, dtype=np.int32)
        _check(load().sld_make_labels(self._h, int(S[0]), int(S[1]), int(S[2]), _ptr(tau_a, np.float64),
                                      int(L), _ptr(out, np.int32)))
        return out

    def make_labels_cc(self, S, tau, L, out=None):
        """Automatic subdomain-levelset labels (sld_make_labels_cc): the
        connected components of each subdomain's levelset classes.  Returns
        (labels, d); follow with build_deflation(d)."""
        tau_a = np.ascontiguousarray(tau if len(tau) else [0.0], dtype=np.float64)
        if out is None:
            out = np.empty(self.n, dtype=np.int32)
        d = C.c_int(0)
        st = load().sld_make_labels_cc(self._h, int(S[0]), int(S[1]), int(S[2]), _ptr(tau_a, np.float64), int(L),
                                       _ptr(out, np.int32), C.byref(d))
        self.cc_components = d.value
        _check(st)
        return out, d.value

    def build_deflation(self, d, labels=None, Zextra=None):
        """Z = [label columns, Zextra]: Zextra is n x k (k <= 8), row-major,
        float64 or float32 (numpy or a torch tensor, host or device)."""
        k, zp, zdt = 0, None, ZEXTRA_F64
        if Zextra is not None:
            if _is_torch(Zextra):
                import torch
                zdt = ZEXTRA_F32 if Zextra.dtype == torch.float32 else ZEXTRA_F64
            else:
                zdt = ZEXTRA_F32 if Zextra.dtype == np.float32 else ZEXTRA_F64
            if Zextra.ndim != 2 or Zextra.shape[0] != self.n:
                raise ValueError("Zextra must be n x k")
            k = int(Zextra.shape[1])
            zp = _ptr(Zextra, np.float32 if zdt == ZEXTRA_F32 else np.float64)
        _check(load().sld_build_deflation(self._h, _ptr(labels, np.int32), int(d), zp, k, zdt))
        self.d = int(d)

    def deflation_info(self):
        """(d, k_requested, k_used) of the deflation last built."""
        d, kr, ku = C.c_int(0), C.c_int(0), C.c_int(0)
        _check(load().sld_deflation_info(self._h, C.byref(d), C.byref(kr), C.byref(ku)))
        return d.value, kr.value, ku.value

    # -- solve ------------------------------------------------------------
    def solve(self, b=None, x=None, options: Optional[Options] = None, raise_on_error=True, **kw):
        o = options if options is not None else default_options(**kw)
        if x is None:
            x = np.empty(self.n, dtype=np.float64)
        r = Result()
        st = load().sld_solve(self._h, _ptr(b, np.float64), C.byref(o), _ptr(x, np.float64), C.byref(r))
        info = SolveInfo(r.iterations, r.outer_steps, r.true_relres, r.recursive_relres, r.solve_ms, st,
                         r.kernel_path, r.fwd_err_estimate)
        if st != OK and raise_on_error:
            _check(st)
        return x, info

    def solve_gmres(self, b=None, x=None, m=20, deflate=True, tol=1e-6, maxiter=5000, raise_on_error=True):
        """PDGMRES (sld_solve_gmres): deflated right-Jacobi GMRES(m), FP64.
        Returns (x, GmresInfo); status in info.status."""
        if x is None:
            x = np.empty(self.n, dtype=np.float64)
        r = GmresInfo()
        st = load().sld_solve_gmres(self._h, _ptr(b, np.float64), int(m), 1 if deflate else 0, float(tol),
                                    int(maxiter), _ptr(x, np.float64), C.byref(r))
        r.status = st
        if st != OK and raise_on_error:
            _check(st)
        return x, r

    def solve_rdgmres(self, b=None, x=None, m=30, d=3, tol=1e-6, maxiter=5000, raise_on_error=True):
        """RDGMRES (sld_solve_rdgmres): GMRES(m) deflated with the d harmonic
        Ritz vectors of its first cycle, FP64.  Returns (x, GmresInfo)."""
        if x is None:
            x = np.empty(self.n, dtype=np.float64)
        r = GmresInfo()
        st = load().sld_solve_rdgmres(self._h, _ptr(b, np.float64), int(m), int(d), float(tol), int(maxiter),
                                      _ptr(x, np.float64), C.byref(r))
        r.status = st
        if st != OK and raise_on_error:
            _check(st)
        return x, r

    # -- per-step access ------------------------------------------------------
    def get_operator(self):
        arrs = [np.empty(self.n) for _ in range(5)]
        _check(load().sld_get_operator(self._h, *[a.ctypes.data for a in arrs]))
        return dict(zip(("Tx", "Ty", "Tz", "diag", "b"), arrs))

    def apply_A(self, x, y=None):
        if y is None:
            y = np.empty(self.n)
        _check(load().sld_apply_A(self._h, _ptr(x, np.float64), _ptr(y, np.float64)))
        return y

    def restrict(self, v, out=None):
        if out is None:
            out = np.empty(self.d)
        _check(load().sld_restrict(self._h, _ptr(v, np.float64), _ptr(out, np.float64)))
        return out

    def get_coarse(self):
        _, _, ku = self.deflation_info()
        D = self.d + ku
        E = np.empty((D, D))
        Einv = np.empty((D, D))
        _check(load().sld_get_coarse(self._h, E.ctypes.data, Einv.ctypes.data))
        return E, Einv


def harmonic_ritz(Hbar, d):
    """(Y, theta) from sld_harmonic_ritz: Hbar (m+1) x m; Y m x d (real
    basis, a complex pair as real and imaginary parts), theta d complex."""
    H = np.ascontiguousarray(Hbar, dtype=np.float64)
    m = H.shape[1]
    if H.shape != (m + 1, m):
        raise ValueError("Hbar must be (m+1) x m")
    Y = np.empty((m, d))
    tr = np.empty(d)
    ti = np.empty(d)
    _check(load().sld_harmonic_ritz(H.ctypes.data, m, int(d), Y.ctypes.data, tr.ctypes.data, ti.ctypes.data))
    return Y, tr + 1j * ti


def from_problem(P, stream=None) -> System:
    """Build a System (with SLD labels and deflation) from a workloads.Problem."""
    s = System(np.ascontiguousarray(P.K, dtype=np.float64).reshape(-1),
               None if P.q is None else np.ascontiguousarray(P.q, dtype=np.float64).reshape(-1),
               P.bc_type, P.bc_value, stream=stream, shape=P.shape)
    s.make_labels(P.S, P.tau, P.L)
    s.build_deflation(P.d)
    return s


class Batch:
    """A batched-solve plan over several Systems (sld_batch): one persistent
    launch, one team of CTAs per system, captured in a CUDA graph."""

    def __init__(self, systems: Sequence[System], options: Optional[Options] = None, **kw):
        lib = load()
        self.systems = list(systems)
        o = options if options is not None else default_options(**kw)
        arr = (C.c_void_p * len(self.systems))(*[s._h.value for s in self.systems])
        h = C.c_void_p()
        _check(lib.sld_batch_create(arr, len(self.systems), C.byref(o), C.byref(h)))
        self._h = h
        self._arr = arr

    def describe(self) -> str:
        return load().sld_batch_describe(self._h).decode()

    def solve(self, bs=None, xs=None, raise_on_error=True):
        """bs, xs: sequences (one entry per system, None = assembled rhs /
        allocate a host array).  Returns (xs, infos)."""
        n = len(self.systems)
        if xs is None:
            xs = [np.empty(s.n, dtype=np.float64) for s in self.systems]
        bptr = None
        if bs is not None:
            bptr = (C.c_void_p * n)(*[None if b is None else _ptr(b, np.float64) for b in bs])
        xptr = (C.c_void_p * n)(*[_ptr(x, np.float64) for x in xs])
        res = (Result * n)()
        st = load().sld_batch_solve(self._h, bptr, xptr, res)
        infos = [SolveInfo(r.iterations, r.outer_steps, r.true_relres, r.recursive_relres, r.solve_ms, st,
                           r.kernel_path, r.fwd_err_estimate) for r in res]
        if st != OK and raise_on_error:
            _check(st)
        return xs, infos

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().sld_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass



# ---------------------------------------------------------------------------
# Deflation-vector network and the Lanczos targets (include/sld_net.h)
# ---------------------------------------------------------------------------
NET_K = 8


def net_num_params() -> int:
    return int(load().sld_net_num_params())


class Net:
    """The deflation-vector U-net for nx x ny x nz grids (multiples of 8).
    Arrays may be numpy (host) or torch tensors (device)."""

    def __init__(self, shape, stream=None):
        nz, ny, nx = shape
        h = C.c_void_p()
        _check(load().sld_net_create(int(nx), int(ny), int(nz), stream, C.byref(h)))
        self._h = h
        self.shape = (nz, ny, nx)
        self.n = nx * ny * nz
        self.np = net_num_params()

    def set_params(self, p):
        _check(load().sld_net_set_params(self._h, _ptr(p, np.float32)))

    def get_params(self, out=None):
        out = np.empty(self.np, dtype=np.float32) if out is None else out
        _check(load().sld_net_get_params(self._h, _ptr(out, np.float32)))
        return out

    def get_grads(self, out=None):
        out = np.empty(self.np, dtype=np.float32) if out is None else out
        _check(load().sld_net_get_grads(self._h, _ptr(out, np.float32)))
        return out

    def forward(self, K, out=None, keep=False):
        """n x 8 FP32 vectors for permeability K (n FP64 values)."""
        if keep:
            _check(load().sld_net_forward(self._h, _ptr(K, np.float64), None))
            return None
        out = np.empty((self.n, NET_K), dtype=np.float32) if out is None else out
        _check(load().sld_net_forward(self._h, _ptr(K, np.float64), _ptr(out, np.float32)))
        return out

    def backward(self, dout):
        _check(load().sld_net_backward(self._h, _ptr(dout, np.float32)))

    def loss_backward(self, V, D):
        """Subspace loss of the last forward output against V (n x m FP32)
        with weights D (n FP64); fills the parameter gradients."""
        loss = C.c_double(0.0)
        _check(load().sld_net_loss_backward(self._h, _ptr(V, np.float32), int(V.shape[1]), _ptr(D, np.float64),
                                            C.byref(loss)))
        return loss.value

    def adam(self, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(load().sld_net_adam(self._h, float(lr), float(beta1), float(beta2), float(eps), int(step)))

    def train(self, Ks, Vs, Ds, **opts):
        """sld_learned_train over the fields (Ks[i] n FP64, Vs[i] n x m FP32,
        Ds[i] n FP64; host or device each).  opts: fields of TrainOptions.
        Returns the mean loss of each epoch."""
        o = TrainOptions()
        load().sld_default_train_options(C.byref(o))
        for k, v in opts.items():
            if not hasattr(o, k):
                raise KeyError(k)
            setattr(o, k, v)
        nf = len(Ks)
        m = int(Vs[0].shape[1])
        kp = (C.c_void_p * nf)(*[_ptr(K, np.float64) for K in Ks])
        vp = (C.c_void_p * nf)(*[_ptr(V, np.float32) for V in Vs])
        dp = (C.c_void_p * nf)(*[_ptr(D, np.float64) for D in Ds])
        hist = np.zeros(o.epochs)
        _check(load().sld_learned_train(self._h, nf, kp, vp, m, dp, C.byref(o), hist.ctypes.data))
        return hist

    def infer(self, system, out=None):
        """sld_learned_infer: the network's vectors for the system's own K,
        appended to its labels (the deflation is rebuilt).  Returns `out`
        (n x 8 FP32) if given."""
        _check(load().sld_learned_infer(self._h, system._h, _ptr(out, np.float32) if out is not None else None))
        return out

    def close(self):
        if self._h:
            load().sld_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lanczos_eigvecs(system: System, k=8, m=40, vecs=None):
    """k smallest nonzero eigenpairs of M^{-1} P A (label deflation) by m
    shift-invert Lanczos steps: (values, n x k FP32 vectors, residuals)."""
    vals = np.empty(k)
    res = np.empty(k)
    vecs = np.empty((system.n, k), dtype=np.float32) if vecs is None else vecs
    _check(load().sld_lanczos_eigvecs(system._h, int(k), int(m), vals.ctypes.data, _ptr(vecs, np.float32),
                                      res.ctypes.data))
    return vals, vecs, res
