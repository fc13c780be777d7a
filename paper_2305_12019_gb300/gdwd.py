"""ctypes binding of libgdwd (include/gdwd.h).

Argument marshalling only: every step of the solver runs in the CUDA library.
The library is loaded on first use; if it cannot be loaded (not built, or no
CUDA driver) the calls raise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int32, c_int64, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgdwd.so")

F64, F32, BF16, F16, E4M3 = 0, 1, 2, 3, 4
DTYPES = {"f64": F64, "f32": F32, "bf16": BF16, "f16": F16, "e4m3": E4M3}
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ENOTPD", 4: "EMAXITER", 5: "ENUMERIC", 6: "ETIMEOUT",
          7: "ECUDA", 8: "EUNSUPPORTED"}
OK, EMAXITER = 0, 4


class Options(ctypes.Structure):
    _fields_ = [("mu", c_double), ("tau", c_double), ("tol", c_double), ("sigma0", c_double),
                ("timeout_s", c_double), ("max_iter", c_int32), ("store", c_int32), ("grid", c_int32),
                ("block_rows", c_int32), ("stream", c_void_p), ("refine", c_int32),
                ("cgrid_sequential", c_int32), ("gram_path", c_int32), ("stop_rule", c_int32),
                ("dots_every", c_int32), ("kernelized", c_int32), ("solver", c_int32),
                ("reserved_i32", c_int32), ("reserved", c_int64 * 4)]


class Result(ctypes.Structure):
    _fields_ = [("beta", c_double), ("primal_obj", c_double), ("dual_obj", c_double), ("kkt", c_double),
                ("eta_p", c_double), ("eta_d", c_double), ("eta_c", c_double), ("eta_gap", c_double),
                ("sigma", c_double), ("zscale", c_double), ("t_setup_ms", c_double), ("t_solve_ms", c_double),
                ("iters", c_int32), ("status", c_int32), ("reserved", c_int64 * 4)]

    def as_dict(self):
        out = {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}
        # quantized-stage iterations (refinement sweep); CG steps and Step 1c solves (inexact solver)
        out["quantized_iters"], out["cg_steps"], out["step1c_solves"] = (int(self.reserved[0]), int(self.reserved[1]),
                                                                        int(self.reserved[2]))
        return out


class Info(ctypes.Structure):
    _fields_ = [("d", c_int64), ("n", c_int64), ("store", c_int32), ("block_rows", c_int32), ("slabs", c_int32),
                ("grid", c_int32), ("z_bytes", c_int64), ("device_bytes", c_int64), ("zscale", c_double),
                ("t_setup_ms", c_double), ("t_ingest_ms", c_double), ("t_gram_ms", c_double),
                ("t_factor_ms", c_double), ("gram_tensor_cores", c_int32), ("kernelized", c_int32),
                ("solver", c_int32), ("reserved_", c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class Request(ctypes.Structure):
    _fields_ = [("Z", c_void_p), ("zdt", c_int32), ("z_on_device", c_int32), ("d", c_int64), ("n", c_int64),
                ("ldz", c_int64), ("y", c_void_p), ("q", c_double), ("C", c_double), ("opts", Options),
                ("w", c_void_p), ("alpha", c_void_p)]


EXPORTS = ["gdwd_default_options", "gdwd_create", "gdwd_solve", "gdwd_free", "gdwd_last_error", "gdwd_prox",
           "gdwd_apply", "gdwd_gram", "gdwd_get_info", "gdwd_get_phase_times", "gdwd_get_stored",
           "gdwd_server_create", "gdwd_server_submit", "gdwd_server_poll", "gdwd_server_destroy", "gdwd_solve_batch",
           "gdwd_set_weights", "gdwd_imbalance_weights", "gdwd_suggest_C"]
EAGAIN = 9
STORE_NP = {F64: "float64", F32: "float32", BF16: "uint16", F16: "float16", E4M3: "uint8"}
PHASES = ["warm_passes", "warm_passes_wait", "R", "R_wait", "N1_rows", "N1_wait", "N2_rows", "N2_wait", "B", "B_wait", "S_kkt",
          "N2_rhs", "N2_gemv", "S_sums", "N1_rhs", "N1_gemv", "B_prologue", "B_stream", "N1_prox", "spare"]

_lib = None


class GdwdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH):
    """Loads libgdwd.so (raises if it is missing) and declares the signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libgdwd.so not built at {path}: run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    lib.gdwd_default_options.argtypes = [POINTER(Options)]
    lib.gdwd_create.argtypes = [c_void_p, c_int32, c_int64, c_int64, c_int64, c_int32, POINTER(c_double), c_double,
                                c_double, POINTER(Options), POINTER(c_void_p)]
    lib.gdwd_solve.argtypes = [c_void_p, POINTER(c_double), c_int32, c_void_p, c_int32, c_void_p, POINTER(Result)]
    lib.gdwd_free.argtypes = [c_void_p]
    lib.gdwd_last_error.argtypes = [c_void_p]
    lib.gdwd_last_error.restype = ctypes.c_char_p
    lib.gdwd_prox.argtypes = [c_void_p, c_void_p, c_void_p, c_double, c_double, c_int64, c_void_p, c_void_p]
    lib.gdwd_apply.argtypes = [c_void_p, c_int32, c_void_p, c_void_p]
    lib.gdwd_gram.argtypes = [c_void_p, c_void_p]
    lib.gdwd_get_info.argtypes = [c_void_p, POINTER(Info)]
    lib.gdwd_get_phase_times.argtypes = [c_void_p, POINTER(c_double), c_int32]
    lib.gdwd_get_stored.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.gdwd_server_create.argtypes = [c_int32, ctypes.c_uint64, POINTER(c_void_p)]
    lib.gdwd_server_submit.argtypes = [c_void_p, POINTER(Request), POINTER(ctypes.c_uint64)]
    lib.gdwd_server_poll.argtypes = [c_void_p, ctypes.c_uint64, c_int32, POINTER(Result), POINTER(c_double)]
    lib.gdwd_server_destroy.argtypes = [c_void_p]
    lib.gdwd_solve_batch.argtypes = [POINTER(Request), c_int32, c_int32, POINTER(Result), POINTER(c_double)]
    lib.gdwd_gram_noalloc.argtypes = [c_void_p, c_int64, c_int64, c_int64, c_void_p, c_void_p]
    lib.gdwd_gram_noalloc.restype = c_int32
    lib.gdwd_set_weights.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.gdwd_imbalance_weights.argtypes = [c_void_p, c_int64, c_double, c_void_p]
    lib.gdwd_suggest_C.argtypes = [c_void_p, POINTER(c_double)]
    for name in EXPORTS:
        if name != "gdwd_last_error":
            getattr(lib, name).restype = c_int32
    _lib = lib
    return lib


def _check(status, handle=None):
    if status not in (OK,):
        msg = _lib.gdwd_last_error(handle).decode(errors="replace")
        raise GdwdError(status, msg)


def default_options() -> Options:
    o = Options()
    load().gdwd_default_options(ctypes.byref(o))
    return o


def _is_torch(x):
    return type(x).__module__.startswith("torch")


class Solver:
    """One gDWD data set on the device (gdwd_create) and its solves (gdwd_solve).

    Z is d x n with column i = y_i x_i: a numpy array (host; copied inside the
    call) or a torch tensor (CUDA or pinned host memory) laid out column-major,
    i.e. Z.stride(0) == 1 (for example ``X_rows.T`` of an n x d row-major tensor).
    """

    def __init__(self, Z, y, q, C, *, store="f32", mu=1.0, tau=1.618, tol=1e-6, sigma0=0.0, max_iter=20000,
                 timeout_s=2.0, grid=0, block_rows=0, stream=None, refine=0, cgrid_sequential=0, gram_path=0,
                 stop_rule=0, dots_every=0, kernelized=0, solver="smw"):
        lib = load()
        self._h = c_void_p()
        o = default_options()
        o.refine = int(refine)
        o.gram_path = int(gram_path)
        o.stop_rule = int(stop_rule)
        o.dots_every = int(dots_every)
        o.kernelized = int(kernelized)
        o.solver = {"smw": 0, "direct": 1, "inexact": 2}[solver] if isinstance(solver, str) else int(solver)
        self._direct = o.solver == 1
        o.cgrid_sequential = int(cgrid_sequential)
        o.mu, o.tau, o.tol, o.sigma0 = mu, tau, tol, sigma0
        o.max_iter, o.timeout_s = max_iter, timeout_s
        o.store = DTYPES[store] if isinstance(store, str) else int(store)
        o.grid, o.block_rows = grid, block_rows
        o.stream = stream
        self._stream = stream
        yv = np.ascontiguousarray(np.asarray(y, dtype=np.float64))
        if _is_torch(Z):
            if Z.dim() != 2 or Z.stride(0) != 1:
                raise ValueError("torch Z must be d x n column-major (stride(0) == 1)")
            zdt = F64 if str(Z.dtype) == "torch.float64" else F32
            if str(Z.dtype) not in ("torch.float64", "torch.float32"):
                raise ValueError("Z must be float32 or float64")
            d, n = Z.shape
            ldz = Z.stride(1) if n > 1 else d
            ptr, on_dev = Z.data_ptr(), int(Z.is_cuda)
            self._keep = Z
        else:
            Zn = np.asarray(Z)
            if Zn.dtype not in (np.float32, np.float64):
                Zn = Zn.astype(np.float64)
            Zn = np.asfortranarray(Zn)
            zdt = F64 if Zn.dtype == np.float64 else F32
            d, n = Zn.shape
            ldz = d
            ptr, on_dev = Zn.ctypes.data, 0
            self._keep = Zn
        self.d, self.n, self.q, self.C = int(d), int(n), float(q), float(C)
        st = lib.gdwd_create(c_void_p(ptr), zdt, d, n, ldz, on_dev, yv.ctypes.data_as(POINTER(c_double)), q, C,
                             ctypes.byref(o), ctypes.byref(self._h))
        self._keep = None
        _check(st, None)

    def solve(self, Cs=None, w_out=None, alpha=False):
        """Runs gdwd_solve.  Returns (results, w, alpha_or_None); w is a host (d, k)
        array unless w_out (a CUDA float64 tensor of d*k elements) is given."""
        Cs_arr = None if Cs is None else np.ascontiguousarray(np.atleast_1d(np.asarray(Cs, dtype=np.float64)))
        k = 1 if Cs_arr is None else Cs_arr.size
        res = (Result * k)()
        if w_out is not None:
            w_ptr, w_dev, w_host = w_out.data_ptr(), 1, None
        else:
            w_host = np.zeros((k, self.d), dtype=np.float64)
            w_ptr, w_dev = w_host.ctypes.data, 0
        a_host = np.zeros((k, self.n), dtype=np.float64) if alpha else None
        st = _lib.gdwd_solve(self._h, None if Cs_arr is None else Cs_arr.ctypes.data_as(POINTER(c_double)),
                             0 if Cs_arr is None else k, c_void_p(w_ptr), w_dev,
                             c_void_p(a_host.ctypes.data) if alpha else None, res)
        if st not in (OK, EMAXITER):
            _check(st, self._h)
        out = [r.as_dict() for r in res]
        return out, (w_out if w_host is None else w_host.T.copy()), (None if a_host is None else a_host.T.copy())

    def apply(self, x, out, trans):
        """out = Z~^T x (trans) or Z~ x on CUDA float64 tensors."""
        _check(_lib.gdwd_apply(self._h, int(bool(trans)), c_void_p(x.data_ptr()), c_void_p(out.data_ptr())), self._h)
        return out

    def gram(self):
        """G = I + Z~^T Z~ / mu (n x n); with solver="direct" the d x d I + Z~ Z~^T / mu."""
        m = self.d if self._direct else self.n
        G = np.zeros((m, m), dtype=np.float64)
        _check(_lib.gdwd_gram(self._h, c_void_p(G.ctypes.data)), self._h)
        return G

    def info(self):
        i = Info()
        _check(_lib.gdwd_get_info(self._h, ctypes.byref(i)), self._h)
        return i.as_dict()

    def stored(self):
        """(Zq, colscale): the stored data as raw codes (BF16 as uint16 bits, E4M3 as
        uint8 bits, FP16 as float16) in a d x n array, and the per-column scales."""
        i = self.info()
        Zq = np.zeros((self.n, self.d), dtype=STORE_NP[i["store"]])
        cs = np.zeros(self.n, dtype=np.float64)
        _check(_lib.gdwd_get_stored(self._h, c_void_p(Zq.ctypes.data), c_void_p(cs.ctypes.data)), self._h)
        return Zq.T, cs

    def set_weights(self, e=None, wt=None):
        """Weighted DWD (gdwd_set_weights): penalty weights e, r-term weights wt (n each)."""
        ev = None if e is None else np.ascontiguousarray(np.asarray(e, dtype=np.float64))
        wv = None if wt is None else np.ascontiguousarray(np.asarray(wt, dtype=np.float64))
        for v in (ev, wv):
            if v is not None and v.shape != (self.n,):
                raise ValueError("weights must have n entries")
        _check(_lib.gdwd_set_weights(self._h, None if ev is None else ev.ctypes.data,
                                     None if wv is None else wv.ctypes.data), self._h)

    def suggest_C(self):
        """The penalty parameter heuristic of Sec. 4.1 for the handle's data (gdwd_suggest_C)."""
        c = c_double()
        _check(_lib.gdwd_suggest_C(self._h, ctypes.byref(c)), self._h)
        return c.value

    def phase_times(self):
        """Per-phase device time (ns) of the last solve, CTA 0's view (gdwd_get_phase_times)."""
        buf = (c_double * len(PHASES))()
        _check(_lib.gdwd_get_phase_times(self._h, buf, len(PHASES)), self._h)
        return {PHASES[k]: buf[k] for k in range(len(PHASES))}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.gdwd_free(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def prox(a, sigma, q, r0=None, omega=None, out=None, stream=None):
    """Step-1b prox on CUDA float64 tensors (gdwd_prox)."""
    lib = load()
    import torch
    out = torch.empty_like(a) if out is None else out
    st = lib.gdwd_prox(c_void_p(a.data_ptr()), None if r0 is None else c_void_p(r0.data_ptr()),
                       None if omega is None else c_void_p(omega.data_ptr()), float(sigma), float(q), a.numel(),
                       c_void_p(out.data_ptr()), stream)
    _check(st, None)
    return out


def make_request(Z, y, q, C, *, store="f32", tol=1e-6, sigma0=0.0, max_iter=20000, mu=1.0, tau=1.618,
                 timeout_s=2.0, want_alpha=False, kernelized=0):
    """A gdwd_request for host data (numpy, column-major copy) with host outputs.

    Returns (request, keep) where keep holds the arrays that must outlive the
    request and keep["w"] / keep["alpha"] receive the results."""
    Zn = np.asfortranarray(np.asarray(Z))
    if Zn.dtype not in (np.float32, np.float64):
        Zn = Zn.astype(np.float64)
    yv = np.ascontiguousarray(np.asarray(y, dtype=np.float64))
    d, n = Zn.shape
    w = np.zeros(d)
    al = np.zeros(n) if want_alpha else None
    o = default_options()
    o.mu, o.tau, o.tol, o.sigma0, o.max_iter, o.timeout_s = mu, tau, tol, sigma0, max_iter, timeout_s
    o.store = DTYPES[store] if isinstance(store, str) else int(store)
    o.kernelized = int(kernelized)
    r = Request(Z=Zn.ctypes.data, zdt=F64 if Zn.dtype == np.float64 else F32, z_on_device=0, d=d, n=n, ldz=d,
                y=yv.ctypes.data, q=float(q), C=float(C), opts=o, w=w.ctypes.data,
                alpha=None if al is None else al.ctypes.data)
    return r, {"Z": Zn, "y": yv, "w": w, "alpha": al}


class Server:
    """gdwd_server: continuous batching of independent problems over `slots` streams."""

    def __init__(self, slots=4, hbm_budget=0):
        lib = load()
        self._s = c_void_p()
        _check(lib.gdwd_server_create(int(slots), int(hbm_budget), ctypes.byref(self._s)), None)
        self._keep = {}

    def submit(self, request, keep=None):
        t = ctypes.c_uint64()
        _check(_lib.gdwd_server_submit(self._s, ctypes.byref(request), ctypes.byref(t)), None)
        self._keep[t.value] = (request, keep)
        return t.value

    def poll(self, ticket, wait=True):
        """(result dict, latency_ms) or None while pending."""
        res = Result()
        lat = c_double()
        st = _lib.gdwd_server_poll(self._s, ticket, int(bool(wait)), ctypes.byref(res), ctypes.byref(lat))
        if st == EAGAIN:
            return None
        if st not in (OK, EMAXITER):
            raise GdwdError(st, _lib.gdwd_last_error(None).decode(errors="replace"))
        self._keep.pop(ticket, None)
        return res.as_dict(), lat.value

    def close(self):
        if getattr(self, "_s", None) is not None and self._s.value:
            _lib.gdwd_server_destroy(self._s)
            self._s = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def solve_batch(requests, slots=4):
    """gdwd_solve_batch over a list of Request structs: (results, latencies_ms, status)."""
    lib = load()
    k = len(requests)
    arr = (Request * k)(*requests)
    res = (Result * k)()
    lat = (c_double * k)()
    st = lib.gdwd_solve_batch(arr, k, int(slots), res, lat)
    return [r.as_dict() for r in res], list(lat), st


def imbalance_weights(y, q):
    """Class-balancing r-term weights of Sec. 4.5 (gdwd_imbalance_weights)."""
    lib = load()
    yv = np.ascontiguousarray(np.asarray(y, dtype=np.float64))
    wt = np.zeros(yv.size)
    _check(lib.gdwd_imbalance_weights(yv.ctypes.data, yv.size, float(q), wt.ctypes.data), None)
    return wt


def gram_noalloc(Z, K, stream=None):
    """K = Z^T Z (gdwd_gram_noalloc) for a CUDA float32 Z (d x n, column-major:
    Z.stride(0) == 1) into a CUDA float64 K (n x n, contiguous).  The library
    allocates nothing; its scratch is a fixed array inside the library (n <= 2048)."""
    import torch
    lib = load()
    if Z.dim() != 2 or Z.stride(0) != 1:
        raise ValueError("Z must be d x n column-major (stride(0) == 1)")
    if Z.dtype != torch.float32 or not Z.is_cuda:
        raise ValueError("Z must be a CUDA float32 tensor")
    d, n = Z.shape
    if K.dtype != torch.float64 or not K.is_cuda or not K.is_contiguous():
        raise ValueError("K must be a contiguous CUDA float64 tensor")
    if K.numel() < n * n:
        raise ValueError(f"K holds {K.numel()} elements, fewer than n * n = {n * n}")
    ldz = Z.stride(1) if n > 1 else d
    st = lib.gdwd_gram_noalloc(c_void_p(Z.data_ptr()), d, n, ldz, c_void_p(K.data_ptr()), stream)
    if st != OK:
        raise GdwdError(st, "gdwd_gram_noalloc failed (n <= 2048, float32 column-major input)")
    return K
