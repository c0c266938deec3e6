"""ctypes binding of libinfft.so (include/infft.h).

Argument marshalling only: every step of every transform runs in the CUDA
library.  The raw functions keep the C names (``infft_plan``, ``infft_adjoint``,
...) and take integer pointers; ``Plan`` and ``Batch`` wrap them for torch
tensors (device buffers) and numpy arrays (host buffers, staged by the library).
If the library is missing this module raises instead of falling back to
anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libinfft.so")

OK, EINVAL, ENOMEM, ECUDA, ENOTCONV, ETIMEOUT, ESTATE, EUNSUPPORTED = range(8)
FP32, FP64 = 1, 2
WIN_KB, WIN_BSPLINE, WIN_DIRICHLET = 0, 4, 8
POOLED = 16
MODE_PLAIN, MODE_DCF, MODE_BOPT = 0, 1, 2
BOPT_PATTERN_2M2, BOPT_PATTERN_PAPER, BOPT_REAL = 0, 1, 2
WEIGHTS_AUTO, WEIGHTS_NFFT, WEIGHTS_TOEPLITZ = 0, 1, 2
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ENOTCONV", "ETIMEOUT", "ESTATE", "EUNSUPPORTED"]


class InfftError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


_lib = None

_SIGS = {
    "infft_plan": (C.c_int, [C.c_int, C.c_int, C.c_int64, C.c_void_p, C.c_double, C.c_int, C.c_uint, C.c_void_p,
                             C.POINTER(C.c_void_p)]),
    "infft_plan_tuned": (C.c_int, [C.c_int, C.c_int, C.c_int64, C.c_void_p, C.c_double, C.c_int, C.c_uint,
                                   C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "infft_weights": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_double),
                                C.POINTER(C.c_int), C.c_void_p]),
    "infft_weights_opts": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_uint, C.POINTER(C.c_double),
                                     C.POINTER(C.c_int), C.c_void_p]),
    "infft_set_weights": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "infft_get_weights": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "infft_optimize_B": (C.c_int, [C.c_void_p, C.c_uint, C.POINTER(C.c_double), C.c_void_p]),
    "infft_get_bopt": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "infft_set_bopt": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "infft_adjoint": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "infft_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "infft_inverse_adjoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "infft_adjoint_batched": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.POINTER(C.c_void_p),
                                        C.POINTER(C.c_void_p), C.c_void_p]),
    "infft_adjoint_batched_slots": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.POINTER(C.c_void_p),
                                              C.POINTER(C.c_void_p), C.POINTER(C.c_int), C.c_void_p]),
    "infft_adjoint_batched_timed": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.POINTER(C.c_void_p),
                                              C.POINTER(C.c_void_p), C.c_void_p, C.POINTER(C.c_float)]),
    "infft_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.POINTER(C.c_void_p),
                                     C.POINTER(C.c_void_p), C.c_void_p, C.POINTER(C.c_void_p)]),
    "infft_batch_run": (C.c_int, [C.c_void_p, C.c_void_p]),
    "infft_adjoint_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "infft_spread_grid": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "infft_fft_axis": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_int64, C.c_int, C.c_void_p, C.c_void_p,
                                 C.c_void_p]),
    "infft_batch_destroy": (None, [C.c_void_p]),
    "infft_plan_N": (C.c_int64, [C.c_void_p]),
    "infft_plan_Msigma": (C.c_int, [C.c_void_p]),
    "infft_plan_work_items": (C.c_int, [C.c_void_p]),
    "infft_plan_device_bytes": (C.c_size_t, [C.c_void_p]),
    "infft_last_error": (C.c_char_p, []),
    "infft_destroy": (None, [C.c_void_p]),
    "infft_launch_count": (C.c_uint64, []),
    "infft_wait_timeouts": (C.c_uint, []),
    "infft_inject_faults": (None, [C.c_uint]),
    "infft_launch_count_reset": (None, []),
}

EXPORTED = tuple(_SIGS)


def load(path: str = LIB_PATH):
    """Load libinfft.so (built by ``paper_2302_00414_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2302_00414_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != OK:
        raise InfftError(status, load().infft_last_error().decode(errors="replace"))


def last_error() -> str:
    return load().infft_last_error().decode(errors="replace")


def launch_count() -> int:
    return int(load().infft_launch_count())


def wait_timeouts() -> int:
    """Bounded waits of the persistent batched kernel that gave up (infft_wait_timeouts)."""
    return int(load().infft_wait_timeouts())


def inject_faults(mask: int):
    """Host-side fault injection: 1 allocations fail, 2 launches report failure, 4 CG does
    not converge; 0 off."""
    load().infft_inject_faults(int(mask))


def launch_count_reset():
    load().infft_launch_count_reset()


# ---- raw entry points, same names as the C ABI (integer pointers) ----------------------

class Tune(C.Structure):
    """infft_tune_t: the plan's kernel choices (0 = the library's default)."""
    _fields_ = [("tile", C.c_int), ("item_cap", C.c_int), ("branches", C.c_int), ("prefetch", C.c_int),
                ("fused_fft", C.c_int)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


TUNE_FIELDS = tuple(k for k, _ in Tune._fields_)


def infft_plan(d, M, N, x_ptr, sigma, m, flags, stream=0):
    out = C.c_void_p()
    return load().infft_plan(d, M, N, x_ptr, sigma, m, flags, stream, C.byref(out)), out.value


def infft_plan_tuned(d, M, N, x_ptr, sigma, m, flags, tune=None, stream=0):
    """tune: a dict with keys of TUNE_FIELDS (missing keys 0), or None."""
    out = C.c_void_p()
    t = None
    if tune:
        t = Tune(**{k: int(tune.get(k, 0)) for k in TUNE_FIELDS})
    return load().infft_plan_tuned(d, M, N, x_ptr, sigma, m, flags, C.byref(t) if t is not None else None, stream,
                                   C.byref(out)), out.value


def infft_weights(plan, max_iter, rel_tol, m_cg=0, stream=0, opts=0):
    res = C.c_double(float("nan"))
    it = C.c_int(0)
    if opts:
        s = load().infft_weights_opts(plan, max_iter, rel_tol, m_cg, opts, C.byref(res), C.byref(it), stream)
    else:
        s = load().infft_weights(plan, max_iter, rel_tol, m_cg, C.byref(res), C.byref(it), stream)
    return s, res.value, it.value


def infft_optimize_B(plan, opts=0, stream=0):
    res = C.c_double(float("nan"))
    s = load().infft_optimize_B(plan, opts, C.byref(res), stream)
    return s, res.value


def infft_adjoint(plan, mode, f_ptr, fhat_ptr, stream=0):
    return load().infft_adjoint(plan, mode, f_ptr, fhat_ptr, stream)


def infft_adjoint_noalloc(plan, mode, f_ptr, fhat_ptr, stream=0):
    """The reconstruction of infft_adjoint with the per-call scratch in the library's
    fixed device array (device pointers only; see include/infft.h)."""
    return load().infft_adjoint_noalloc(plan, mode, f_ptr, fhat_ptr, stream)


def infft_spread_grid(plan, mode, f_ptr, grid_ptr, stream=0):
    """Step 1 of Algorithm 2.4 into a caller's M_sigma^d grid (device pointers)."""
    return load().infft_spread_grid(plan, mode, f_ptr, grid_ptr, stream)


def infft_fft_axis(plan, mode, A, B, nblk, in_ptr, out_ptr, stream=0):
    """Steps 2-3 of Algorithm 2.4 along the middle axis of an (A, M_sigma, B) tensor."""
    return load().infft_fft_axis(plan, mode, A, B, nblk, in_ptr, out_ptr, stream)


def infft_forward(plan, fhat_ptr, f_ptr, stream=0):
    return load().infft_forward(plan, fhat_ptr, f_ptr, stream)


def infft_adjoint_batched(plans, mode, f_ptrs, fhat_ptrs, stream=0):
    n = len(plans)
    P = (C.c_void_p * n)(*plans)
    F = (C.c_void_p * n)(*f_ptrs)
    H = (C.c_void_p * n)(*fhat_ptrs)
    return load().infft_adjoint_batched(P, n, mode, F, H, stream)


def infft_adjoint_batched_slots(plans, mode, f_ptrs, fhat_ptrs, slots, stream=0):
    n = len(plans)
    P = (C.c_void_p * n)(*plans)
    F = (C.c_void_p * n)(*f_ptrs)
    H = (C.c_void_p * n)(*fhat_ptrs)
    S = (C.c_int * n)(*slots)
    return load().infft_adjoint_batched_slots(P, n, mode, F, H, S, stream)


def infft_destroy(plan):
    load().infft_destroy(plan)


# ---- convenience wrappers ---------------------------------------------------------------

def _ptr(a):
    """Pointer of a torch tensor (device or host) or a numpy array (host), C-contiguous."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return a.data_ptr()


def _stream(stream):
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))   # a torch stream or a handle
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return 0


class Plan:
    """A plan for fixed points x (N x d, float64 numpy array or torch tensor)."""

    def __init__(self, x, M: int, sigma: float = 2.0, m: int = 4, precision: str = "fp32",
                 window: str = "kb", stream=None, pooled: bool = False, tune=None):
        """tune: optional dict of kernel choices (see infft_tune_t in include/infft.h)."""
        self.precision, self.window = precision, window
        self.tune = dict(tune) if tune else None
        self.has_weights = self.has_bopt = False
        flags = {"fp32": FP32, "fp64": FP64}[precision] | (POOLED if pooled else 0)
        flags |= {"kb": WIN_KB, "bspline": WIN_BSPLINE, "dirichlet": WIN_DIRICHLET}[window]
        if isinstance(x, np.ndarray):
            x = np.ascontiguousarray(x, dtype=np.float64)
            if x.ndim == 1:
                x = x[:, None]
            N, d = x.shape
        else:
            if x.dtype != __import__("torch").float64:
                raise ValueError("x must be float64")
            x = x.contiguous()
            if x.dim() == 1:
                x = x[:, None]
            N, d = x.shape
        self.d, self.M, self.N, self.m, self.sigma = int(d), int(M), int(N), int(m), float(sigma)
        if self.tune:
            s, h = infft_plan_tuned(self.d, self.M, self.N, _ptr(x), self.sigma, self.m, flags, self.tune,
                                    _stream(stream))
        else:
            s, h = infft_plan(self.d, self.M, self.N, _ptr(x), self.sigma, self.m, flags, _stream(stream))
        _check(s)
        self.handle = h
        self.Ms = int(load().infft_plan_Msigma(h))

    @property
    def complex_dtype(self):
        return np.complex64 if self.precision == "fp32" else np.complex128

    @property
    def work_items(self) -> int:
        """Number of work items (tile, point range) the plan's spreading kernels run."""
        return int(load().infft_plan_work_items(self.handle))

    @property
    def device_bytes(self) -> int:
        return int(load().infft_plan_device_bytes(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            infft_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def weights(self, max_iter: int = 1000, rel_tol: float = 1e-13, m_cg: int = 0, stream=None, check=True,
                method: str = "auto"):
        """Algorithm 3.6; method "nfft" (products by NFFTs), "toeplitz" (convolution form,
        second kind only) or "auto"."""
        opts = {"auto": WEIGHTS_AUTO, "nfft": WEIGHTS_NFFT, "toeplitz": WEIGHTS_TOEPLITZ}[method]
        s, res, it = infft_weights(self.handle, max_iter, rel_tol, m_cg, _stream(stream), opts)
        if check and s not in (OK, ENOTCONV):
            _check(s)
        self.has_weights = self.has_weights or s in (OK, ENOTCONV)
        return {"status": s, "residual_inf": res, "iters": it}

    def set_weights(self, w, stream=None):
        """N weights in the caller's point order: any numpy array (converted to complex128)
        or a complex128 torch tensor."""
        if isinstance(w, np.ndarray):
            w = np.ascontiguousarray(w, dtype=np.complex128).ravel()
            if w.size != self.N:
                raise ValueError(f"{w.size} weights for {self.N} points")
        else:
            import torch
            if w.dtype != torch.complex128 or w.numel() != self.N:
                raise ValueError("weights must be a complex128 tensor of N entries")
            w = w.contiguous()
        _check(load().infft_set_weights(self.handle, _ptr(w), _stream(stream)))
        self.has_weights = True

    def get_weights(self, stream=None) -> np.ndarray:
        w = np.empty(self.N, dtype=np.complex128)
        _check(load().infft_get_weights(self.handle, w.ctypes.data, _stream(stream)))
        return w

    def optimize_B(self, opts: int = 0, stream=None):
        s, res = infft_optimize_B(self.handle, opts, _stream(stream))
        _check(s)
        self.has_bopt = True
        return res

    def set_bopt(self, coeff, stream=None):
        """Restore B_opt coefficients from get_bopt (N x (2m+2)^d complex128)."""
        c = np.ascontiguousarray(coeff, dtype=np.complex128) if isinstance(coeff, np.ndarray) else coeff
        _check(load().infft_set_bopt(self.handle, _ptr(c), _stream(stream)))
        self.has_bopt = True

    def get_bopt(self, stream=None) -> np.ndarray:
        S = 2 * self.m + 2
        c = np.empty((self.N,) + (S,) * self.d, dtype=np.complex128)
        _check(load().infft_get_bopt(self.handle, c.ctypes.data, _stream(stream)))
        return c

    def adjoint(self, f, fhat=None, mode: int = MODE_PLAIN, stream=None):
        """fhat = D^* F^* B^* (W) f; f and fhat are torch tensors (device) or numpy arrays (host)."""
        if fhat is None:
            if isinstance(f, np.ndarray):
                fhat = np.empty((self.M,) * self.d, dtype=self.complex_dtype)
            else:
                import torch
                fhat = torch.empty((self.M,) * self.d, dtype=f.dtype, device=f.device)
        _check(infft_adjoint(self.handle, mode, _ptr(f), _ptr(fhat), _stream(stream)))
        return fhat

    def inverse_adjoint(self, h, f=None, stream=None):
        """f = B_opt F D h (Remark 4.6), an approximate solution of A^* f = h; needs optimize_B."""
        if f is None:
            if isinstance(h, np.ndarray):
                f = np.empty(self.N, dtype=self.complex_dtype)
            else:
                import torch
                f = torch.empty(self.N, dtype=h.dtype, device=h.device)
        _check(load().infft_inverse_adjoint(self.handle, _ptr(h), _ptr(f), _stream(stream)))
        return f

    def forward(self, fhat, f=None, stream=None):
        if f is None:
            if isinstance(fhat, np.ndarray):
                f = np.empty(self.N, dtype=self.complex_dtype)
            else:
                import torch
                f = torch.empty(self.N, dtype=fhat.dtype, device=fhat.device)
        _check(infft_forward(self.handle, _ptr(fhat), _ptr(f), _stream(stream)))
        return f


def adjoint_batched(plans, fs, fhats, mode: int = MODE_PLAIN, stream=None, slots=None):
    """Batched adjoint; `slots` (optional) picks the scratch set of each job."""
    if slots is None:
        _check(infft_adjoint_batched([p.handle for p in plans], mode, [_ptr(f) for f in fs],
                                     [_ptr(h) for h in fhats], _stream(stream)))
    else:
        _check(infft_adjoint_batched_slots([p.handle for p in plans], mode, [_ptr(f) for f in fs],
                                           [_ptr(h) for h in fhats], list(slots), _stream(stream)))


def adjoint_batched_timed(plans, fs, fhats, mode: int = MODE_PLAIN, stream=None):
    """Batched adjoint; returns device times (ms) of spread, merge and the FFT passes."""
    n = len(plans)
    P = (C.c_void_p * n)(*[p.handle for p in plans])
    F = (C.c_void_p * n)(*[_ptr(f) for f in fs])
    H = (C.c_void_p * n)(*[_ptr(h) for h in fhats])
    ms = (C.c_float * 5)()
    _check(load().infft_adjoint_batched_timed(P, n, mode, F, H, _stream(stream), ms))
    return {"spread": ms[0], "merge": ms[1], "fft": [ms[2 + t] for t in range(plans[0].d)]}


class Batch:
    """A CUDA graph of the batched adjoint over fixed plans and fixed buffers: device tensors,
    or page-locked host arrays (numpy views of pinned torch tensors), whose copies the graph
    then holds; after run() synchronise the stream before reading host results."""

    def __init__(self, plans, fs, fhats, mode: int = MODE_PLAIN, stream=None):
        n = len(plans)
        self._keep = (plans, fs, fhats)
        P = (C.c_void_p * n)(*[p.handle for p in plans])
        F = (C.c_void_p * n)(*[_ptr(f) for f in fs])
        H = (C.c_void_p * n)(*[_ptr(h) for h in fhats])
        out = C.c_void_p()
        _check(load().infft_batch_create(P, n, mode, F, H, _stream(stream), C.byref(out)))
        self.handle = out.value

    def run(self, stream=None):
        _check(load().infft_batch_run(self.handle, _stream(stream)))

    def close(self):
        if getattr(self, "handle", None):
            load().infft_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
