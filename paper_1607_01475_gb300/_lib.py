"""ctypes binding of libpsd.so: argument marshalling only.

Tensors are torch CUDA tensors (float64, or float32 for psd_residual_f32),
contiguous, shaped (ny, nx) in 2D or (nz, ny, nx) in 3D (x fastest).  Work is
enqueued on torch's current CUDA stream unless a stream is given.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_NAME = "libpsd.so"

PSD_FP64 = 0
PSD_MIXED = 1
PSD_PROF_CLASSES = 13  # kernel classes of psd_profile_read

_STATUS = {0: "PSD_OK", 1: "PSD_ERR_INVALID", 2: "PSD_ERR_NOMEM", 3: "PSD_ERR_CUDA",
           4: "PSD_ERR_NOCONV", 5: "PSD_ERR_TIMEOUT", 6: "PSD_ERR_UNSUPPORTED",
           7: "PSD_ERR_NONFINITE"}


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class PSDParams(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("dim", ctypes.c_int), ("n", ctypes.c_int * 3),
                ("h", ctypes.c_double), ("p", ctypes.c_double), ("s", ctypes.c_double),
                ("eps", ctypes.c_double), ("lam", ctypes.c_double), ("precision", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("max_outer", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("inner_eta", ctypes.c_double), ("inner_stall", ctypes.c_int),
                ("alloc", ALLOC_FN), ("free_fn", FREE_FN), ("alloc_ctx", ctypes.c_void_p),
                ("report_energy", ctypes.c_int)]


class PSDInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer_iters", ctypes.c_int), ("res_l2", ctypes.c_double),
                ("res_linf", ctypes.c_double), ("energy", ctypes.c_double), ("last_alpha", ctypes.c_double),
                ("wall_ms", ctypes.c_double), ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# ctypes callback objects must outlive the handle that calls them
_callbacks = {}


def _allocator_callbacks(allocator):
    """(alloc(nbytes) -> int device pointer, free(int pointer)) -> ctypes pair."""
    if allocator is None:
        return ALLOC_FN(), FREE_FN()
    a, f = allocator
    return ALLOC_FN(lambda n, ctx: a(n)), FREE_FN(lambda ptr, ctx: f(ptr))


class PSDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib_path():
    return os.path.join(HERE, _LIB_NAME)


def load_library(build_if_missing=True):
    """Load libpsd.so (building it with nvcc if absent).  Raises on failure."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path) and build_if_missing:
        from . import build as _build
        _build.build()
    if not os.path.exists(path):
        raise PSDError(3, f"{path} not found; build it with paper_1607_01475_gb300/build.py")
    lib = ctypes.CDLL(path)
    P, H, D, F = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p
    lib.psd_create.argtypes = [ctypes.POINTER(PSDParams), ctypes.POINTER(ctypes.c_void_p)]
    lib.psd_destroy.argtypes = [H]
    lib.psd_residual.argtypes = [H, D, D, D, D, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.psd_precond_solve.argtypes = [H, D, D]
    lib.psd_solve.argtypes = [H, D, D, D, D, ctypes.POINTER(PSDInfo)]
    lib.psd_set_history.argtypes = [H, P, P, ctypes.c_int]
    lib.psd_residual_f32.argtypes = [H, F, F, F]
    lib.psd_residual_fixed.argtypes = [H, D, D, D, ctypes.POINTER(ctypes.c_int)]
    lib.psd_thinfilm_steps.argtypes = [H, D, ctypes.c_int, ctypes.POINTER(PSDInfo)]
    lib.psd_spfc_steps.argtypes = [H, D, ctypes.c_double, ctypes.c_int, ctypes.POINTER(PSDInfo)]
    lib.psd_thinfilm_adjoint.argtypes = [H, D, ctypes.c_int, D, D, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                         ctypes.c_double, ctypes.c_int, ctypes.POINTER(PSDInfo)]
    lib.psd_precond_solve_f32.argtypes = [H, F, F]
    lib.psd_theta_ff.argtypes = [H, D, D]
    lib.psd_autotune.argtypes = [H, P]
    lib.psd_energy.argtypes = [H, D, D, D, ctypes.POINTER(ctypes.c_double)]
    lib.psd_last_error.argtypes = [H, ctypes.c_char_p, ctypes.c_size_t]
    lib.psd_profile.argtypes = [H, ctypes.c_int]
    lib.psd_profile_classes.argtypes = [H, ctypes.c_uint]
    lib.psd_profile_read.argtypes = [H, P, P, P, P, ctypes.c_double, ctypes.c_int]
    lib.psd_profile_class_name.argtypes = [ctypes.c_int]
    lib.psd_profile_class_name.restype = ctypes.c_char_p
    lib.psd_hvp.argtypes = [H, D, D, D, ctypes.POINTER(ctypes.c_double)]
    lib.psd_adjoint.argtypes = [H, D, D, D, ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.c_int,
                                ctypes.POINTER(PSDInfo)]
    lib.psd_batch_create.argtypes = [ctypes.POINTER(PSDParams), ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_void_p)]
    lib.psd_batch_solve.argtypes = [H, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                    ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(PSDInfo)]
    lib.psd_batch_destroy.argtypes = [H]
    lib.psd_batch_last_error.argtypes = [H, ctypes.c_char_p, ctypes.c_size_t]
    lib.psd_batch_mode.argtypes = [H]
    lib.psd_batch_mode.restype = ctypes.c_int
    lib.psd_batch_set_mode.argtypes = [H, ctypes.c_int]
    lib.psd_batch_set_mode.restype = ctypes.c_int
    lib.psd_residual_noalloc.argtypes = [ctypes.POINTER(PSDParams), D, D, D, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double)]
    lib.psd_noalloc_last_error.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    lib.psd_status_string.argtypes = [ctypes.c_int]
    lib.psd_status_string.restype = ctypes.c_char_p
    for name in ("psd_create", "psd_destroy", "psd_residual", "psd_precond_solve", "psd_solve",
                 "psd_set_history", "psd_residual_f32", "psd_residual_fixed", "psd_theta_ff", "psd_autotune", "psd_thinfilm_steps", "psd_spfc_steps", "psd_thinfilm_adjoint", "psd_last_error",
                 "psd_profile",
                 "psd_profile_read", "psd_profile_classes", "psd_residual_noalloc", "psd_noalloc_last_error",
                 "psd_precond_solve_f32", "psd_energy",
                 "psd_hvp",
                 "psd_adjoint", "psd_batch_create", "psd_batch_solve", "psd_batch_destroy",
                 "psd_batch_last_error"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def psd_status_string(status):
    return load_library().psd_status_string(int(status)).decode()


def _last_error(handle):
    buf = ctypes.create_string_buffer(512)
    load_library().psd_last_error(handle, buf, len(buf))
    return buf.value.decode()


def _check(status, handle, allow=()):
    if status != 0 and status not in allow:
        raise PSDError(status, _last_error(handle))
    return status


def _ptr(t, dtype_name="float64"):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous() or str(t.dtype) != f"torch.{dtype_name}":
        raise PSDError(1, f"expected a contiguous CUDA {dtype_name} tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# ------------------------------------------------------------ C-named calls

def psd_create(order, shape, h, p, s, eps, lam=0.0, precision=PSD_FP64, tol=1e-10,
               max_iter=10000, max_outer=20, stream=None, inner_eta=0.0, inner_stall=0, allocator=None,
               report_energy=False):
    """Create a solver handle for a grid of ``shape`` ((ny, nx) or (nz, ny, nx)).
    ``allocator``: optional (alloc(nbytes) -> device pointer, free(pointer))."""
    lib = load_library()
    dim = len(shape)
    n = (shape[-1], shape[-2], shape[0] if dim == 3 else 1)
    cb_alloc, cb_free = _allocator_callbacks(allocator)
    prm = PSDParams(order=order, dim=dim, n=(ctypes.c_int * 3)(*n), h=h, p=p, s=s, eps=eps, lam=lam,
                    precision=precision, tol=tol, max_iter=max_iter, max_outer=max_outer,
                    stream=_stream_handle(stream) if stream is not False else None,
                    inner_eta=inner_eta, inner_stall=inner_stall, alloc=cb_alloc, free_fn=cb_free,
                    report_energy=1 if report_energy else 0)
    out = ctypes.c_void_p()
    _check(lib.psd_create(ctypes.byref(prm), ctypes.byref(out)), None)
    if allocator is not None:
        _callbacks[out.value] = (cb_alloc, cb_free)
    return out


def psd_destroy(handle):
    st = load_library().psd_destroy(handle)
    _callbacks.pop(getattr(handle, "value", handle), None)
    return st


def psd_residual(handle, u, f, g=None, r=None):
    l2, linf = ctypes.c_double(), ctypes.c_double()
    _check(load_library().psd_residual(handle, _ptr(u), _ptr(f), _ptr(g), _ptr(r),
                                       ctypes.byref(l2), ctypes.byref(linf)), handle)
    return l2.value, linf.value


def psd_precond_solve(handle, r, d):
    _check(load_library().psd_precond_solve(handle, _ptr(r), _ptr(d)), handle)


def psd_solve(handle, f, u, g=None, w=None, allow_noconv=False):
    info = PSDInfo()
    allow = (4,) if allow_noconv else ()
    _check(load_library().psd_solve(handle, _ptr(f), _ptr(g), _ptr(u), _ptr(w), ctypes.byref(info)),
           handle, allow)
    return info.as_dict()


def psd_hvp(handle, u, v, y):
    """y = H v (Hessian of the discrete energy at u, Euclidean); returns h^d v.y."""
    dot = ctypes.c_double()
    _check(load_library().psd_hvp(handle, _ptr(u), _ptr(v), _ptr(y), ctypes.byref(dot)), handle)
    return dot.value


def psd_adjoint(handle, u, grad_u, grad_f, tol_rel=1e-12, max_iter=1000):
    """grad_f <- dJ/df; returns (dJ/ds, info)."""
    gs = ctypes.c_double()
    info = PSDInfo()
    _check(load_library().psd_adjoint(handle, _ptr(u), _ptr(grad_u), _ptr(grad_f), ctypes.byref(gs),
                                      tol_rel, max_iter, ctypes.byref(info)), handle)
    return gs.value, info.as_dict()


def psd_energy(handle, u, f, g=None):
    e = ctypes.c_double()
    _check(load_library().psd_energy(handle, _ptr(u), _ptr(f), _ptr(g), ctypes.byref(e)), handle)
    return e.value


def psd_precond_solve_f32(handle, r, d):
    _check(load_library().psd_precond_solve_f32(handle, _ptr(r, "float32"), _ptr(d, "float32")), handle)


def psd_residual_f32(handle, u, f, r):
    _check(load_library().psd_residual_f32(handle, _ptr(u, "float32"), _ptr(f, "float32"),
                                           _ptr(r, "float32")), handle)


def psd_thinfilm_steps(handle, u, nsteps, allow_noconv=False):
    """nsteps thin-film convex-splitting steps in place on u (see
    include/psd.h); returns the accumulated info as a dict."""
    info = PSDInfo()
    allow = (4,) if allow_noconv else ()
    _check(load_library().psd_thinfilm_steps(handle, _ptr(u), int(nsteps), ctypes.byref(info)), handle, allow)
    return info.as_dict()


def psd_spfc_steps(handle, u, gamma1, nsteps, allow_noconv=False):
    """nsteps SPFC convex-splitting steps in place on u (see include/psd.h);
    returns the accumulated info as a dict."""
    info = PSDInfo()
    allow = (4,) if allow_noconv else ()
    _check(load_library().psd_spfc_steps(handle, _ptr(u), float(gamma1), int(nsteps), ctypes.byref(info)), handle,
           allow)
    return info.as_dict()


def psd_thinfilm_adjoint(handle, u0, nsteps, grad_uN, grad_u0, checkpoints=0, tol_rel=1e-12, max_iter=1000):
    """grad_u0 <- dJ/du^0 through nsteps thin-film steps from u0, given
    grad_uN = dJ/du^N (see include/psd.h); returns (dJ/ds, info)."""
    gs = ctypes.c_double()
    info = PSDInfo()
    _check(load_library().psd_thinfilm_adjoint(handle, _ptr(u0), int(nsteps), _ptr(grad_uN), _ptr(grad_u0),
                                                ctypes.byref(gs), int(checkpoints), float(tol_rel), int(max_iter),
                                                ctypes.byref(info)), handle)
    return gs.value, info.as_dict()


def psd_residual_fixed(handle, u, f, r):
    """FP64 residual by the fixed-point / float-float kernel variant; returns
    the fixed-point scale S (0: the variant does not apply, r untouched)."""
    scale = ctypes.c_int()
    _check(load_library().psd_residual_fixed(handle, _ptr(u), _ptr(f), _ptr(r), ctypes.byref(scale)), handle)
    return scale.value


def psd_theta_ff(handle, x, theta):
    """theta += H[T_h x] by the float-float transform passes (see include/psd.h)."""
    _check(load_library().psd_theta_ff(handle, _ptr(x), _ptr(theta)), handle)


def psd_residual_noalloc(shape, h, p, s, eps, u, f, r, stream=None):
    """Fourth-order residual and norms without a handle or any device
    allocation (see include/psd.h).  Returns (||r||_2, max|r|)."""
    lib = load_library()
    dim = len(shape)
    n = (shape[-1], shape[-2], shape[0] if dim == 3 else 1)
    prm = PSDParams(order=4, dim=dim, n=(ctypes.c_int * 3)(*n), h=h, p=p, s=s, eps=eps, lam=0.0,
                    precision=0, tol=0.0, max_iter=0, max_outer=0, stream=_stream_handle(stream))
    l2, linf = ctypes.c_double(), ctypes.c_double()
    st = lib.psd_residual_noalloc(ctypes.byref(prm), _ptr(u), _ptr(f), _ptr(r), ctypes.byref(l2),
                                  ctypes.byref(linf))
    if st != 0:
        buf = ctypes.create_string_buffer(256)
        lib.psd_noalloc_last_error(buf, len(buf))
        raise PSDError(st, buf.value.decode())
    return l2.value, linf.value


def _params(order, shape, h, p, s, eps, lam=0.0, precision=PSD_FP64, tol=1e-10, max_iter=10000,
            max_outer=20, stream=None, inner_eta=0.0, inner_stall=0):
    dim = len(shape)
    n = (shape[-1], shape[-2], shape[0] if dim == 3 else 1)
    return PSDParams(order=order, dim=dim, n=(ctypes.c_int * 3)(*n), h=h, p=p, s=s, eps=eps, lam=lam,
                     precision=precision, tol=tol, max_iter=max_iter, max_outer=max_outer, stream=stream,
                     inner_eta=inner_eta, inner_stall=inner_stall)


class Batch:
    """Many independent instances solved concurrently (psd_batch_*).
    ``instances``: list of dicts with keys order, shape, h, p, s, eps and
    optionally lam, precision, tol, max_iter, max_outer."""

    def __init__(self, instances, workers=0):
        lib = load_library()
        self.n = len(instances)
        arr = (PSDParams * self.n)(*[_params(**inst) for inst in instances])
        out = ctypes.c_void_p()
        st = lib.psd_batch_create(arr, self.n, workers, ctypes.byref(out))
        if st != 0:
            buf = ctypes.create_string_buffer(512)
            lib.psd_batch_last_error(None, buf, len(buf))
            raise PSDError(st, buf.value.decode())
        self.handle = out

    def solve(self, fs, us, gs=None, allow_noconv=False, check=True):
        """Solve every instance; returns the per-instance info dicts.  With
        check=False a failing batch does not raise: (status, message, infos)
        is returned instead, so that the other instances can be inspected."""
        lib = load_library()
        P = ctypes.c_void_p * self.n
        fp = P(*[_ptr(t).value for t in fs])
        up = P(*[_ptr(t).value for t in us])
        gp = P(*[(_ptr(t).value if t is not None else None) for t in gs]) if gs is not None else None
        infos = (PSDInfo * self.n)()
        st = lib.psd_batch_solve(self.handle, fp, gp, up, infos)
        msg = ""
        if st != 0:
            buf = ctypes.create_string_buffer(512)
            lib.psd_batch_last_error(self.handle, buf, len(buf))
            msg = buf.value.decode()
        if not check:
            return st, msg, [i.as_dict() for i in infos]
        if st != 0 and not (allow_noconv and st == 4):
            raise PSDError(st, msg)
        return [i.as_dict() for i in infos]

    def mode(self):
        """Schedule of the last solve: 1 one graph, 2 per-instance graphs, 3 host threads."""
        return load_library().psd_batch_mode(self.handle)

    def set_mode(self, mode):
        """0 default, 1 one graph, 2 per-instance graphs on their streams, 3 host threads."""
        st = load_library().psd_batch_set_mode(self.handle, int(mode))
        if st != 0:
            raise PSDError(st, "invalid batch mode")

    def close(self):
        if self.handle:
            load_library().psd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------- convenience

class Solver:
    """Owns one handle.  ``shape`` is (ny, nx) or (nz, ny, nx)."""

    def __init__(self, order, shape, h, p, s, eps, lam=0.0, precision=PSD_FP64, tol=1e-10,
                 max_iter=10000, max_outer=20, stream=None, inner_eta=0.0, inner_stall=0, allocator=None,
                 report_energy=False):
        self.shape = tuple(shape)
        self.handle = psd_create(order, shape, h, p, s, eps, lam, precision, tol, max_iter,
                                 max_outer, stream, inner_eta, inner_stall, allocator, report_energy)
        self._hist = None

    def close(self):
        if self.handle:
            psd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def residual(self, u, f, g=None, r=None):
        return psd_residual(self.handle, u, f, g, r)

    def precond_solve(self, r, d):
        psd_precond_solve(self.handle, r, d)

    def residual_f32(self, u, f, r):
        psd_residual_f32(self.handle, u, f, r)

    def residual_fixed(self, u, f, r):
        return psd_residual_fixed(self.handle, u, f, r)

    def autotune(self):
        """Tile widths of the FP32 transform passes (see include/psd.h);
        returns the three chosen caps."""
        caps = (ctypes.c_int * 3)()
        _check(load_library().psd_autotune(self.handle, caps), self.handle)
        return list(caps)

    def theta_ff(self, x, theta):
        psd_theta_ff(self.handle, x, theta)

    def thinfilm_steps(self, u, nsteps):
        return psd_thinfilm_steps(self.handle, u, nsteps)

    def spfc_steps(self, u, gamma1, nsteps):
        return psd_spfc_steps(self.handle, u, gamma1, nsteps)

    def thinfilm_adjoint(self, u0, nsteps, grad_uN, grad_u0, checkpoints=0, tol_rel=1e-12, max_iter=1000):
        return psd_thinfilm_adjoint(self.handle, u0, nsteps, grad_uN, grad_u0, checkpoints, tol_rel, max_iter)

    def precond_solve_f32(self, r, d):
        psd_precond_solve_f32(self.handle, r, d)

    def energy(self, u, f, g=None):
        return psd_energy(self.handle, u, f, g)

    def set_history(self, cap):
        import numpy as np
        if cap <= 0:
            self._hist = None
            _check(load_library().psd_set_history(self.handle, None, None, 0), self.handle)
            return
        a = np.full(cap, np.nan)
        r = np.full(cap, np.nan)
        _check(load_library().psd_set_history(self.handle, a.ctypes.data_as(ctypes.c_void_p),
                                              r.ctypes.data_as(ctypes.c_void_p), cap), self.handle)
        self._hist = (a, r)

    def history(self):
        return self._hist

    def solve(self, f, u, g=None, w=None, allow_noconv=False):
        return psd_solve(self.handle, f, u, g, w, allow_noconv)

    def hvp(self, u, v, y):
        return psd_hvp(self.handle, u, v, y)

    def adjoint(self, u, grad_u, grad_f, tol_rel=1e-12, max_iter=1000):
        return psd_adjoint(self.handle, u, grad_u, grad_f, tol_rel, max_iter)

    def profile(self, enable=True, classes=None):
        """Bracket kernel launches with events: all classes, or only the
        class names in ``classes``."""
        lib = load_library()
        if classes is None or not enable:
            _check(lib.psd_profile(self.handle, 1 if enable else 0), self.handle)
            return
        names = [lib.psd_profile_class_name(k).decode() for k in range(PSD_PROF_CLASSES)]
        mask = 0
        for c in classes:
            mask |= 1 << names.index(c)
        _check(lib.psd_profile_classes(self.handle, mask), self.handle)

    def profile_read(self, eff_us=8.0):
        """{class name: (ms, launches, effective ms, effective launches)}."""
        import numpy as np
        n = PSD_PROF_CLASSES
        ms = np.zeros(n)
        cnt = np.zeros(n, dtype=np.int64)
        ems = np.zeros(n)
        ecnt = np.zeros(n, dtype=np.int64)
        ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        lib = load_library()
        _check(lib.psd_profile_read(self.handle, ptr(ms), ptr(cnt), ptr(ems), ptr(ecnt), eff_us, n),
               self.handle)
        return {lib.psd_profile_class_name(k).decode(): (float(ms[k]), int(cnt[k]), float(ems[k]), int(ecnt[k]))
                for k in range(n)}
