"""Python binding of the C ABI in ``include/lqcd.h`` (ctypes).

Argument marshalling only: every numerical step runs in the CUDA kernels of
``liblqcd.so``. Fields are complex128 arrays of length ``12*V`` in the order
``[site][spin][colour]`` (site ``x + Lx*(y + Ly*(z + Lz*t))``); a batch of
``k`` fields is a ``(k, 12*V)`` array. Host arrays (numpy, CPU torch) are
passed as host pointers; CUDA torch tensors are passed as device pointers and
must be contiguous complex128 on the library's device.

The library must have been built (``paper_0911_2285_gb300.build.build()``);
there is no fallback: a missing library raises ``RuntimeError``.
"""
from __future__ import annotations

import ctypes as C
import hashlib
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblqcd.so")

# lqcd_status
OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NOCONV, ERR_BREAKDOWN, ERR_TIMEOUT, ERR_STATE = range(8)
FP64, MIXED = 0, 1
MODE_AUTO, MODE_EIGBICG, MODE_DEFLATED, MODE_PLAIN = 0, 1, 2, 3
_MODES = {"auto": MODE_AUTO, "eigbicg": MODE_EIGBICG, "deflated": MODE_DEFLATED, "plain": MODE_PLAIN}
_PREC = {"fp64": FP64, "mixed": MIXED}


class Params(C.Structure):
    _fields_ = [
        ("dims", C.c_int * 4),
        ("kappa", C.c_double),
        ("nev", C.c_int),
        ("m", C.c_int),
        ("n1", C.c_int),
        ("tol", C.c_double),
        ("maxiter", C.c_int),
        ("precision", C.c_int),
        ("deftol", C.c_double),
        ("k_max", C.c_int),
        ("hbm_budget_bytes", C.c_size_t),
        ("n_def_max", C.c_int),
        ("delta", C.c_double),
        ("gamma5", C.c_int),
        ("bicgstab", C.c_int),
        ("evenodd", C.c_int),
        ("no_autotune", C.c_int),
    ]


class SolveInfo(C.Structure):
    _fields_ = [
        ("iters", C.c_int),
        ("matvecs", C.c_int),
        ("restarts", C.c_int),
        ("reliable_updates", C.c_int),
        ("outer_steps", C.c_int),
        ("true_resid", C.c_double),
        ("seconds", C.c_double),
        ("mode_used", C.c_int),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class LQCDError(RuntimeError):
    def __init__(self, status, where, msg=""):
        self.status = status
        super().__init__(f"{where}: {status_str(status)}" + (f" ({msg})" if msg else ""))


_lib = None


def lib():
    """The loaded ``liblqcd.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_0911_2285_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
        L.lqcd_eigbicg_init.argtypes = [C.POINTER(vp), C.POINTER(Params), vp, vp]
        L.lqcd_solve.argtypes = [vp, C.c_int, vp, vp, C.c_int, C.c_int, C.POINTER(SolveInfo)]
        L.lqcd_deflate.argtypes = [vp, C.c_int, vp, vp, C.c_int]
        L.lqcd_eigs.argtypes = [vp, ip, vp, vp, vp, vp]
        L.lqcd_apply.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp, vp, C.c_int]
        L.lqcd_eigspace_size.argtypes = [vp]
        L.lqcd_eigspace_size.restype = C.c_int
        L.lqcd_eigspace_get.argtypes = [vp, vp, vp, vp]
        L.lqcd_eigspace_set.argtypes = [vp, C.c_int, vp, vp]
        L.lqcd_last_window.argtypes = [vp, C.c_int, ip, vp, vp, ip]
        L.lqcd_small_eig.argtypes = [C.c_int, vp, vp, vp, vp]
        L.lqcd_restart_coefficients.argtypes = [C.c_int, C.c_int, vp, ip, vp, vp, vp]
        L.lqcd_status_str.argtypes = [C.c_int]
        L.lqcd_status_str.restype = C.c_char_p
        L.lqcd_last_error.restype = C.c_char_p
        L.lqcd_destroy.argtypes = [vp]
        L.lqcd_kernel_launches.restype = C.c_longlong
        L.lqcd_time_kernel.argtypes = [vp, C.c_int, C.c_int, C.c_int, dp]
        L.lqcd_time_kernel.restype = C.c_int
        L.lqcd_submit.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.POINTER(C.c_longlong)]
        L.lqcd_progress.argtypes = [vp, C.c_int, C.POINTER(C.c_int)]
        L.lqcd_poll.argtypes = [vp, C.c_longlong, C.POINTER(C.c_int), C.POINTER(SolveInfo), C.POINTER(C.c_int)]
        for name in ("lqcd_submit", "lqcd_progress", "lqcd_poll"):
            getattr(L, name).restype = C.c_int
        L.lqcd_set_tensor_cores.argtypes = [vp, C.c_int]
        L.lqcd_set_tensor_cores.restype = C.c_int
        L.lqcd_field_dots.argtypes = [C.c_int, vp, C.c_int, vp, C.c_longlong, C.c_int, C.c_int, vp,
                                      C.POINTER(C.c_double)]
        L.lqcd_field_dots.restype = C.c_int
        L.lqcd_small_eig_noalloc.argtypes = [C.c_int, vp, vp, vp, vp, vp]
        L.lqcd_small_eig_noalloc.restype = C.c_int
        L.lqcd_apply_pair.argtypes = [vp, C.c_int, C.c_int, vp, vp, vp, vp, vp]
        L.lqcd_apply_pair.restype = C.c_int
        L.lqcd_memory_info.argtypes = [vp, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t), ip]
        L.lqcd_memory_info.restype = C.c_int
        L.lqcd_batch_size.argtypes = [vp]
        L.lqcd_batch_size.restype = C.c_int
        L.lqcd_batch_timings.argtypes = [vp, dp]
        L.lqcd_batch_timings.restype = C.c_int
        L.lqcd_set_wait_limit.argtypes = [C.c_longlong]
        L.lqcd_set_wait_limit.restype = C.c_int
        L.lqcd_wait_flag.argtypes = [vp, vp]
        L.lqcd_wait_flag.restype = C.c_int
        L.lqcd_dslash_variant.argtypes = [vp]
        L.lqcd_dslash_variant.restype = C.c_int
        L.lqcd_set_dslash_variant.argtypes = [vp, C.c_int]
        L.lqcd_set_dslash_variant.restype = C.c_int
        for name in ("lqcd_eigbicg_init", "lqcd_solve", "lqcd_deflate", "lqcd_eigs", "lqcd_apply",
                     "lqcd_eigspace_get", "lqcd_eigspace_set", "lqcd_last_window", "lqcd_small_eig",
                     "lqcd_restart_coefficients"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def status_str(s):
    return lib().lqcd_status_str(int(s)).decode()


def last_error():
    return lib().lqcd_last_error().decode()


def _check(status, where, allow=()):
    if status != OK and status not in allow:
        raise LQCDError(status, where, last_error())
    return status


def _ptr(a, n_expected=None):
    """(pointer, on_device) of a contiguous complex128 array or tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.complex128 or not a.is_contiguous():
                raise TypeError("torch fields must be contiguous complex128")
            if n_expected is not None and a.numel() != n_expected:
                raise ValueError(f"expected {n_expected} complex numbers, got {a.numel()}")
            return C.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0
    except ImportError:  # pragma: no cover - torch is optional for the host path
        pass
    if not isinstance(a, np.ndarray) or a.dtype != np.complex128 or not a.flags.c_contiguous:
        raise TypeError("fields must be C-contiguous complex128 numpy arrays or torch tensors")
    if n_expected is not None and a.size != n_expected:
        raise ValueError(f"expected {n_expected} complex numbers, got {a.size}")
    return C.c_void_p(a.ctypes.data), 0


def _current_cuda_device():
    """Index of the current CUDA device if torch has initialised CUDA, else None (the
    context was then created on the CUDA runtime's current device, not known here)."""
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_device()
    except ImportError:  # pragma: no cover
        pass
    return None


def _fingerprint(a):
    """Digest of a whole gauge field (shape and every link entry), to refuse an
    eigenspace saved for another field. Hashes the contiguous buffer once per
    context (about a second at 24^3x64)."""
    a = np.ascontiguousarray(a)
    h = hashlib.sha256(repr(a.shape).encode())
    h.update(a.reshape(-1).view(np.uint8))
    return h.hexdigest()[:32]


def _npz_path(path):
    """``np.savez`` appends ``.npz`` to a path without it; use the same name on load."""
    path = os.fspath(path)
    return path if path.endswith(".npz") else path + ".npz"


class Solver:
    """One gauge field + parameter set (an ``lqcd_ctx``)."""

    def __init__(self, links, dims, kappa, nev=10, m=40, n1=4, tol=1e-10, maxiter=5000,
                 precision="mixed", deftol=0.0, k_max=0, hbm_budget_bytes=0, n_def_max=0,
                 delta=0.0, stream=None, gamma5=False, bicgstab=False, evenodd=False, autotune=True):
        links = np.ascontiguousarray(links, dtype=np.complex128)
        self.dims = tuple(int(d) for d in dims)
        self.kappa = float(kappa)
        self._links_fp = _fingerprint(links)
        self.volume = int(np.prod(self.dims))
        self.n = 12 * self.volume
        if links.size != 4 * self.volume * 9:
            raise ValueError("links must hold 4*V*9 complex numbers")
        p = Params()
        for i, d in enumerate(self.dims):
            p.dims[i] = d
        p.kappa = kappa
        p.nev, p.m, p.n1 = nev, m, n1
        p.tol, p.maxiter = tol, maxiter
        p.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
        p.deftol, p.k_max = deftol, k_max
        p.hbm_budget_bytes = hbm_budget_bytes
        p.n_def_max = n_def_max
        p.delta = delta
        p.gamma5 = 1 if gamma5 else 0
        p.bicgstab = 1 if bicgstab else 0
        p.evenodd = 1 if evenodd else 0
        p.no_autotune = 0 if autotune else 1
        self.evenodd = bool(evenodd)
        # field length of the solver's own space (eigenvectors, lqcd_apply): the odd
        # half lattice in an even-odd context; sources and solutions stay full (self.n)
        self.n_space = self.n // 2 if self.evenodd else self.n
        self.params = p
        self.gamma5 = bool(gamma5)
        self.precision = precision
        h = C.c_void_p()
        st = lib().lqcd_eigbicg_init(C.byref(h), C.byref(p), C.c_void_p(links.ctypes.data),
                                     C.c_void_p(stream) if stream else None)
        _check(st, "lqcd_eigbicg_init")
        self._h = h
        self.kmax = k_max or 8
        self._own_stream = not stream
        self._device = _current_cuda_device()

    def _fields(self, a, c, n_a=None, n_c=None):
        """Pointers of two fields of one call, both host or both device; device tensors
        must live on the context's GPU. A context on its private stream does not wait
        for work queued on torch's current stream, so that work (e.g. the zero fill of
        an initial guess) is finished first."""
        pa, da = _ptr(a, n_a)
        pc, dc = _ptr(c, n_c)
        if da != dc:
            raise ValueError("both fields must be host arrays or both device tensors")
        if da:
            import torch
            for t in (a, c):
                if self._device is not None and t.device.index != self._device:
                    raise ValueError(f"device tensors must be on cuda:{self._device}, got {t.device}")
            if self._own_stream:
                torch.cuda.current_stream(a.device).synchronize()
        return pa, pc, da

    def memory_info(self):
        """``(plan_bytes, window_bytes, windows_attached)``: the fixed device-memory plan,
        the size of one eigBiCG window and the windows held now."""
        plan, win, att = C.c_size_t(), C.c_size_t(), C.c_int()
        _check(lib().lqcd_memory_info(self._h, C.byref(plan), C.byref(win), C.byref(att)), "lqcd_memory_info")
        return plan.value, win.value, att.value

    def batch_size(self):
        """Right-hand sides per batched launch (``k_max``, or the autotuned size)."""
        return lib().lqcd_batch_size(self._h)

    def batch_timings(self):
        """ms of one BiCG iteration per batch size k (index k) as the batch-size autotuner
        timed it (``k_max = 0`` contexts only; else None)."""
        ms = (C.c_double * 9)()
        st = lib().lqcd_batch_timings(self._h, ms)
        return list(ms) if st == OK else None

    def close(self):
        if getattr(self, "_h", None):
            lib().lqcd_destroy(self._h)
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

    # ---------------------------------------------------------------- calls
    def solve(self, b, x0=None, mode="auto", raise_on_fail=True, out=None):
        """Solve ``A x = b`` for a batch; returns ``(x, infos, status)``.

        ``out`` (optional) receives the solutions in place and must already hold
        the initial guesses (``x0`` is then ignored).
        """
        b = _as_batch(b, self.n)
        k = b.shape[0]
        if out is not None:
            x = _as_batch(out, self.n)
        elif x0 is None:
            x = _zeros_like(b)
        else:
            x = _as_batch(x0, self.n)
            x = x.clone() if hasattr(x, "clone") else x.copy()
        pb, px, db = self._fields(b, x, k * self.n, k * self.n)
        infos = (SolveInfo * max(k, 1))()
        st = lib().lqcd_solve(self._h, k, pb, px, db, _MODES[mode] if isinstance(mode, str) else int(mode), infos)
        if raise_on_fail:
            _check(st, "lqcd_solve")
        return x, [infos[i].as_dict() for i in range(k)], st

    # ------------------------------------------------------ serving session
    def submit(self, b, x, mode="auto"):
        """Queue one source; ``x`` holds the initial guess and receives the solution.
        Both arrays must stay alive until :meth:`poll` reports the ticket done."""
        pb, px, db = self._fields(b, x, self.n, self.n)
        t = C.c_longlong()
        _check(lib().lqcd_submit(self._h, pb, px, db, _MODES[mode] if isinstance(mode, str) else int(mode),
                                 C.byref(t)), "lqcd_submit")
        return t.value

    def progress(self, wait=True):
        """Retire finished requests, admit queued ones, launch the next iterations;
        returns the number of requests still queued or running. With ``wait=False``
        it returns at once while the iterations in flight are still running."""
        n = C.c_int()
        _check(lib().lqcd_progress(self._h, 1 if wait else 0, C.byref(n)), "lqcd_progress")
        return n.value

    def poll(self, ticket):
        """``(done, info, status)`` of a submitted request (reported once)."""
        done = C.c_int()
        info = SolveInfo()
        res = C.c_int()
        _check(lib().lqcd_poll(self._h, int(ticket), C.byref(done), C.byref(info), C.byref(res)), "lqcd_poll")
        return bool(done.value), (info.as_dict() if done.value else None), res.value

    def deflate(self, b, x0):
        b = _as_batch(b, self.n)
        x = _as_batch(x0, self.n)
        x = x.clone() if hasattr(x, "clone") else x.copy()
        if b.shape != x.shape:
            raise ValueError("b and x0 must have the same shape")
        pb, px, db = self._fields(b, x)
        _check(lib().lqcd_deflate(self._h, b.shape[0], pb, px, db), "lqcd_deflate")
        return x

    def apply(self, v, dagger=False, precision="fp64"):
        """``A v`` (``A^+ v``) on the solver's space: the full lattice, or A_hat on the
        odd half lattice of an even-odd context."""
        v = _as_batch(v, self.n_space)
        out = _zeros_like(v)
        pv, po, dv = self._fields(v, out)
        _check(lib().lqcd_apply(self._h, int(dagger), _PREC[precision], v.shape[0], pv, po, dv), "lqcd_apply")
        return out

    def eigs(self, n=None, vectors=False):
        """Rayleigh-Ritz eigenpairs of the accumulated eigenspace."""
        size = self.eigspace_size()
        n = size if n is None else min(n, size)
        cnt = C.c_int(n)
        ev = np.zeros(max(n, 1), dtype=np.complex128)
        res = np.zeros(max(n, 1), dtype=np.float64)
        ur = np.zeros((n, self.n_space), dtype=np.complex128) if vectors else None
        ul = np.zeros((n, self.n_space), dtype=np.complex128) if vectors else None
        st = lib().lqcd_eigs(self._h, C.byref(cnt), C.c_void_p(ev.ctypes.data),
                             C.c_void_p(ur.ctypes.data) if vectors else None,
                             C.c_void_p(ul.ctypes.data) if vectors else None, C.c_void_p(res.ctypes.data))
        _check(st, "lqcd_eigs")
        k = cnt.value
        return ev[:k], res[:k], (ur[:k] if vectors else None), (ul[:k] if vectors else None)

    def reset_eigenspace(self):
        """Empty the eigenspace (AUTO mode starts over with eigBiCG)."""
        _check(lib().lqcd_eigspace_set(self._h, 0, None, None), "lqcd_eigspace_set")

    def time_kernel(self, kernel, k, reps=10):
        """Average device ms of one launch of an iteration kernel (see lqcd_time_kernel)."""
        ms = C.c_double()
        _check(lib().lqcd_time_kernel(self._h, int(kernel), int(k), int(reps), C.byref(ms)), "lqcd_time_kernel")
        return ms.value

    def apply_pair(self, p, phat, variant):
        """One launch of the operator-pair kernel shape ``variant``: ``(A p, A^+ phat, sigma)``."""
        p = np.ascontiguousarray(p, dtype=np.complex128).reshape(-1, self.n_space)
        phat = np.ascontiguousarray(phat, dtype=np.complex128).reshape(-1, self.n_space)
        k = p.shape[0]
        ap = np.zeros_like(p)
        ahp = np.zeros_like(phat)
        sig = np.zeros(k, dtype=np.complex128)
        _check(lib().lqcd_apply_pair(self._h, int(variant), k, C.c_void_p(p.ctypes.data), C.c_void_p(phat.ctypes.data),
                                     C.c_void_p(ap.ctypes.data), C.c_void_p(ahp.ctypes.data),
                                     C.c_void_p(sig.ctypes.data)), "lqcd_apply_pair")
        return ap, ahp, sig

    def set_tensor_cores(self, on):
        """Tensor-core (True, default) or CUDA-core (False) FP32 projections and restart products."""
        _check(lib().lqcd_set_tensor_cores(self._h, 1 if on else 0), "lqcd_set_tensor_cores")

    def dslash_variant(self):
        """Operator-kernel shape chosen by the autotuner (or pinned)."""
        return lib().lqcd_dslash_variant(self._h)

    def set_dslash_variant(self, variant):
        """Pin the operator-kernel shape (LQCDError if this context cannot use it)."""
        _check(lib().lqcd_set_dslash_variant(self._h, int(variant)), "lqcd_set_dslash_variant")

    def eigspace_size(self):
        return lib().lqcd_eigspace_size(self._h)

    def eigspace_get(self):
        n = self.eigspace_size()
        ur = np.zeros((n, self.n_space), dtype=np.complex128)
        ul = np.zeros((n, self.n_space), dtype=np.complex128)
        h = np.zeros((n, n), dtype=np.complex128)
        if n:
            _check(lib().lqcd_eigspace_get(self._h, C.c_void_p(ur.ctypes.data), C.c_void_p(ul.ctypes.data),
                                           C.c_void_p(h.ctypes.data)), "lqcd_eigspace_get")
        return ur, ul, h

    def eigspace_set(self, ur, ul):
        ur = np.ascontiguousarray(ur, dtype=np.complex128).reshape(-1, self.n_space)
        ul = np.ascontiguousarray(ul, dtype=np.complex128).reshape(-1, self.n_space)
        if ur.shape != ul.shape:
            raise ValueError("Ur and Ul must have the same shape")
        _check(lib().lqcd_eigspace_set(self._h, ur.shape[0], C.c_void_p(ur.ctypes.data),
                                       C.c_void_p(ul.ctypes.data)), "lqcd_eigspace_set")

    def save_eigenspace(self, path):
        """Checkpoint the accumulated eigenspace (U_r, U_l and H = U_l^H A U_r) with
        the lattice, kappa and a digest of the gauge field, as an ``.npz`` file."""
        ur, ul, h = self.eigspace_get()
        np.savez(_npz_path(path), Ur=ur, Ul=ul, H=h, dims=np.array(self.dims), kappa=np.float64(self.kappa),
                 links_fp=np.array(self._links_fp))

    def load_eigenspace(self, path):
        """Resume from :meth:`save_eigenspace`: the vectors are installed and H is
        recomputed on this context's operator (which must be the same gauge field,
        lattice and kappa, else ``ValueError``). The loaded vectors count as complete
        eigBiCG solves for AUTO mode. The recomputed H must agree with the stored
        one to ``h_rtol`` of its largest entry (FP32-stored vectors: their projections
        are FP32 sums; FP64: rounding), else ``ValueError``. Returns the largest
        relative difference."""
        with np.load(_npz_path(path)) as d:
            if tuple(int(x) for x in d["dims"]) != self.dims or float(d["kappa"]) != self.kappa:
                raise ValueError("eigenspace saved for another lattice or kappa")
            if str(d["links_fp"]) != self._links_fp:
                raise ValueError("eigenspace saved for another gauge field")
            ur, ul, h_saved = d["Ur"], d["Ul"], d["H"]
        self.eigspace_set(ur, ul)
        _, _, h = self.eigspace_get()
        scale = max(float(np.abs(h_saved).max()) if h_saved.size else 0.0, 1e-300)
        diff = float(np.abs(h - h_saved).max()) / scale if h.size else 0.0
        h_rtol = 1e-4 if self.precision in ("mixed", MIXED) else 1e-10
        if diff > h_rtol:
            raise ValueError(f"recomputed H differs from the stored one by {diff:.3g} (relative)")
        return diff

    def last_window(self, slot=0):
        m = self.params.m
        vs = C.c_int()
        rs = C.c_int()
        h = np.zeros(m * m, dtype=np.complex128)
        ritz = np.zeros(self.params.nev, dtype=np.complex128)
        _check(lib().lqcd_last_window(self._h, slot, C.byref(vs), C.c_void_p(h.ctypes.data),
                                      C.c_void_p(ritz.ctypes.data), C.byref(rs)), "lqcd_last_window")
        v = vs.value
        return h[: v * v].reshape(v, v), ritz[: min(v, self.params.nev)], rs.value


def _as_batch(a, n):
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return a.reshape(-1, n)
    except ImportError:  # pragma: no cover
        pass
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a.reshape(-1, n)


def _zeros_like(a):
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return torch.zeros_like(a)
    except ImportError:  # pragma: no cover
        pass
    return np.zeros_like(a)


def kernel_launches():
    """Kernels launched by the library in this process so far."""
    return int(lib().lqcd_kernel_launches())


def field_dots(X, Y, path=1, reps=0):
    """``C = X^H Y`` (a x b, complex128) of FP32 fields: ``X`` (a, n) and ``Y`` (b, n)
    contiguous complex64 CUDA tensors. ``path`` 0 = CUDA cores, 1 = tensor cores
    (3xTF32). Returns ``(C, avg_ms)``; ``avg_ms`` is the mean time of ``reps`` more
    calls (None when ``reps == 0``)."""
    import torch
    for t in (X, Y):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex64 and t.is_contiguous()
                and t.dim() == 2):
            raise TypeError("X and Y must be contiguous 2-D complex64 CUDA tensors")
    if X.shape[1] != Y.shape[1]:
        raise ValueError("X and Y fields must have the same length")
    a, n = X.shape
    b = Y.shape[0]
    out = np.zeros((a, b), dtype=np.complex128)
    ms = C.c_double()
    _check(lib().lqcd_field_dots(a, C.c_void_p(X.data_ptr()), b, C.c_void_p(Y.data_ptr()), n, int(path), int(reps),
                                 C.c_void_p(out.ctypes.data), C.byref(ms)), "lqcd_field_dots")
    return out, (ms.value if reps > 0 else None)


def small_eig(c):
    """Device eigen-solver on a small dense matrix: ``(lam, Y, Z)``, smallest |lambda| first."""
    c = np.ascontiguousarray(c, dtype=np.complex128)
    n = c.shape[0]
    lam = np.zeros(n, dtype=np.complex128)
    y = np.zeros((n, n), dtype=np.complex128)
    z = np.zeros((n, n), dtype=np.complex128)
    _check(lib().lqcd_small_eig(n, C.c_void_p(c.ctypes.data), C.c_void_p(lam.ctypes.data),
                                C.c_void_p(y.ctypes.data), C.c_void_p(z.ctypes.data)), "lqcd_small_eig")
    return lam, y, z


def restart_coefficients(h, nev):
    """Device Algorithm BiCG-eigen (coefficient part): ``(Yc, Zc, lam)``."""
    h = np.ascontiguousarray(h, dtype=np.complex128)
    m = h.shape[0]
    r = C.c_int()
    yc = np.zeros((m, 2 * nev), dtype=np.complex128)
    zc = np.zeros((m, 2 * nev), dtype=np.complex128)
    lam = np.zeros(2 * nev, dtype=np.complex128)
    _check(lib().lqcd_restart_coefficients(m, nev, C.c_void_p(h.ctypes.data), C.byref(r),
                                           C.c_void_p(yc.ctypes.data), C.c_void_p(zc.ctypes.data),
                                           C.c_void_p(lam.ctypes.data)), "lqcd_restart_coefficients")
    k = r.value
    return yc[:, :k].copy(), zc[:, :k].copy(), lam[:k].copy()
