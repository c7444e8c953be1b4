"""GB300 (sm_103a) kinetic DG library -- thin Python binding of include/kin.h.

The functions below carry the C ABI's names and only marshal arguments
(numpy arrays for host buffers, torch tensors for device or pinned host
buffers); every step of the method runs in the CUDA kernels of ``libkin.so``.
There is no CPU fallback: if the library cannot be loaded, importing a
function raises.

Method (arXiv:2212.11010): one step S(dt) = R_omega o T_CN(dt) -- an implicit
upwind DG Crank-Nicolson transport of every kinetic population, solved by
downwind sweeps inside subdomains coupled by the lagged iteration of Sec. 5.1,
followed by the over-relaxation f <- omega M(W) + (1 - omega) f (Sec. 2.2).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkin.so")

KIN_OK, KIN_EINVAL, KIN_ENOMEM, KIN_EBUDGET, KIN_ECUDA, KIN_ETIMEOUT, KIN_ESTATE = range(7)
KIN_ADVECTION, KIN_EULER, KIN_MAXWELL = 0, 1, 2
KIN_D1Q2, KIN_D2Q4, KIN_D3Q6, KIN_D2Q3, KIN_D3Q4 = 1, 2, 3, 4, 5
KIN_FP64, KIN_FP32 = 0, 1
KIN_DEBUG_STALL_LOAD = 1

STATUS_NAMES = {0: "KIN_OK", 1: "KIN_EINVAL", 2: "KIN_ENOMEM", 3: "KIN_EBUDGET",
                4: "KIN_ECUDA", 5: "KIN_ETIMEOUT", 6: "KIN_ESTATE"}

EXPORTED = ["kin_create", "kin_set_state", "kin_set_kinetic", "kin_step", "kin_get_state",
            "kin_get_kinetic", "kin_set_kinetic_async", "kin_get_kinetic_async", "kin_diag", "kin_sync", "kin_query", "kin_destroy", "kin_last_error",
            "kin_step_noalloc", "kin_batch_create", "kin_batch_create_ex", "kin_batch_step", "kin_batch_sync",
            "kin_batch_destroy", "kin_batch_last_error", "kin_set_boundary", "kin_batch_info", "kin_create_tet"]


class KinError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class kin_mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3), ("inflow", ctypes.c_int * 3)]


class kin_model(ctypes.Structure):
    _fields_ = [("system", ctypes.c_int), ("velset", ctypes.c_int), ("lam", ctypes.c_double),
                ("gamma", ctypes.c_double), ("adv", ctypes.c_double * 3), ("omega", ctypes.c_double),
                ("sigma", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class kin_opts(ctypes.Structure):
    _fields_ = [("tiles", ctypes.c_int * 3), ("iters", ctypes.c_int), ("precision", ctypes.c_int),
                ("block", ctypes.c_int * 3), ("mem_budget", ctypes.c_size_t),
                ("stream", ctypes.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_user", ctypes.c_void_p), ("wait_timeout_s", ctypes.c_double),
                ("debug_flags", ctypes.c_int), ("threads", ctypes.c_int), ("stages", ctypes.c_int)]


class kin_tetmesh(ctypes.Structure):
    _fields_ = [("ncells", ctypes.c_int), ("xyz", ctypes.POINTER(ctypes.c_double)),
                ("vid", ctypes.POINTER(ctypes.c_longlong)), ("nbr", ctypes.POINTER(ctypes.c_longlong)),
                ("sub", ctypes.POINTER(ctypes.c_int)), ("wrap", ctypes.POINTER(ctypes.c_int))]


class kin_info(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("degree", ctypes.c_int), ("m", ctypes.c_int),
                ("nvel", ctypes.c_int), ("npop", ctypes.c_int), ("nodes_per_cell", ctypes.c_int),
                ("cells", ctypes.c_size_t), ("nodes", ctypes.c_size_t),
                ("kinetic_values", ctypes.c_size_t), ("state_values", ctypes.c_size_t),
                ("device_bytes", ctypes.c_size_t), ("precision", ctypes.c_int),
                ("block", ctypes.c_int * 3), ("smem_bytes", ctypes.c_int), ("grid", ctypes.c_int),
                ("threads", ctypes.c_int), ("stages", ctypes.c_int), ("steps_done", ctypes.c_longlong),
                ("specialised", ctypes.c_int)]


_lib = None


def load_library():
    """Load libkin.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    sz = ctypes.c_size_t
    dp = ctypes.POINTER(ctypes.c_double)
    lib.kin_create.argtypes = [ctypes.POINTER(kin_mesh), ctypes.POINTER(kin_model), ctypes.c_int,
                               ctypes.c_double, ctypes.POINTER(kin_opts), ctypes.POINTER(vp)]
    lib.kin_create_tet.argtypes = [ctypes.POINTER(kin_tetmesh), ctypes.POINTER(kin_model), ctypes.c_double,
                                   ctypes.POINTER(kin_opts), ctypes.POINTER(vp)]
    lib.kin_set_state.argtypes = [vp, vp, sz, ctypes.c_int]
    lib.kin_set_kinetic.argtypes = [vp, vp, sz, ctypes.c_int]
    lib.kin_set_boundary.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp, sz]
    lib.kin_step.argtypes = [vp, ctypes.c_int]
    lib.kin_get_state.argtypes = [vp, vp, sz, ctypes.c_int]
    lib.kin_get_kinetic.argtypes = [vp, vp, sz, ctypes.c_int]
    lib.kin_set_kinetic_async.argtypes = [vp, vp, sz, vp]
    lib.kin_get_kinetic_async.argtypes = [vp, vp, sz, vp]
    lib.kin_diag.argtypes = [vp, dp, dp, dp]
    lib.kin_sync.argtypes = [vp]
    lib.kin_query.argtypes = [vp, ctypes.POINTER(kin_info)]
    lib.kin_destroy.argtypes = [vp]
    lib.kin_step_noalloc.argtypes = [ctypes.POINTER(kin_mesh), ctypes.POINTER(kin_model), ctypes.c_int,
                                     ctypes.c_double, ctypes.POINTER(kin_opts), vp, ctypes.c_int,
                                     ctypes.c_char_p, sz]
    lib.kin_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp, ctypes.POINTER(vp)]
    lib.kin_batch_create_ex.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp, ctypes.c_int, ctypes.POINTER(vp)]
    lib.kin_batch_step.argtypes = [vp, ctypes.c_int]
    lib.kin_batch_sync.argtypes = [vp]
    lib.kin_batch_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.kin_batch_destroy.argtypes = [vp]
    lib.kin_batch_last_error.argtypes = [vp]
    lib.kin_batch_last_error.restype = ctypes.c_char_p
    lib.kin_last_error.argtypes = [vp]
    lib.kin_last_error.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name not in ("kin_last_error", "kin_batch_last_error"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(ctx, status):
    if status != KIN_OK:
        msg = load_library().kin_last_error(ctx).decode()
        raise KinError(status, msg)


def _ptr(buf):
    """(pointer, on_device) of a numpy array or torch tensor (contiguous)."""
    if isinstance(buf, np.ndarray):
        assert buf.flags.c_contiguous
        return buf.ctypes.data, 0
    import torch
    assert isinstance(buf, torch.Tensor) and buf.is_contiguous()
    return buf.data_ptr(), 1 if buf.is_cuda else 0


def _elem_check(ctx, buf, want):
    """The C calls copy n_values elements of a fixed size (f: the context
    precision, W: FP64); a buffer of another element size would be overrun."""
    size = buf.itemsize if isinstance(buf, np.ndarray) else buf.element_size()
    if size != want:
        raise ValueError(f"expected {want}-byte values, got {buf.dtype}")


def _f_bytes(ctx):
    return 4 if kin_query(ctx).precision == KIN_FP32 else 8


# torch caching-allocator hooks (PyTorch owns the device memory)
_hooks = {}


def torch_allocator_hooks(device=None):
    import torch
    dev = torch.cuda.current_device() if device is None else device
    if dev in _hooks:
        return _hooks[dev]

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))
        except Exception:
            return None

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    _hooks[dev] = (ALLOC_FN(_alloc), FREE_FN(_free))
    return _hooks[dev]


# ---------------------------------------------------------------------------
# C ABI, same names
# ---------------------------------------------------------------------------

def kin_create(mesh: kin_mesh, model: kin_model, degree: int, dt: float, opts: kin_opts):
    lib = load_library()
    ctx = ctypes.c_void_p()
    st = lib.kin_create(ctypes.byref(mesh), ctypes.byref(model), degree, dt, ctypes.byref(opts),
                        ctypes.byref(ctx))
    _check(None, st)
    return ctx


def kin_create_tet(mesh: kin_tetmesh, model: kin_model, dt: float, opts: kin_opts):
    lib = load_library()
    ctx = ctypes.c_void_p()
    st = lib.kin_create_tet(ctypes.byref(mesh), ctypes.byref(model), dt, ctypes.byref(opts), ctypes.byref(ctx))
    _check(None, st)
    return ctx


def kin_set_state(ctx, W, n_values=None):
    _elem_check(ctx, W, 8)
    p, dev = _ptr(W)
    n = W.size if isinstance(W, np.ndarray) else W.numel()
    _check(ctx, load_library().kin_set_state(ctx, p, n if n_values is None else n_values, dev))


def kin_set_boundary(ctx, axis, side, W):
    W = np.ascontiguousarray(np.asarray(W, dtype=np.float64).reshape(-1))
    _check(ctx, load_library().kin_set_boundary(ctx, int(axis), int(side),
                                                W.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), W.size))


def kin_set_kinetic(ctx, f, n_values=None):
    _elem_check(ctx, f, _f_bytes(ctx))
    p, dev = _ptr(f)
    n = f.size if isinstance(f, np.ndarray) else f.numel()
    _check(ctx, load_library().kin_set_kinetic(ctx, p, n if n_values is None else n_values, dev))


def _host_ptr(ctx, a):
    """Address and size of a page-locked host torch tensor whose element size
    is the context's (the async copies move n_values elements of the context
    precision; a pageable numpy array would make the copy synchronous)."""
    if not (hasattr(a, "is_pinned") and a.is_pinned() and a.is_contiguous()):
        raise ValueError("the asynchronous host copies take a contiguous page-locked torch tensor")
    want = 4 if kin_query(ctx).precision == KIN_FP32 else 8
    if a.element_size() != want:
        raise ValueError(f"the context holds {want}-byte values; got a {a.dtype} tensor")
    return ctypes.c_void_p(a.data_ptr()), a.numel()


def kin_set_kinetic_async(ctx, f, stream=None):
    p, n = _host_ptr(ctx, f)
    _check(ctx, load_library().kin_set_kinetic_async(ctx, p, n, stream))


def kin_get_kinetic_async(ctx, f, stream=None):
    p, n = _host_ptr(ctx, f)
    _check(ctx, load_library().kin_get_kinetic_async(ctx, p, n, stream))


def kin_step(ctx, nsteps: int):
    _check(ctx, load_library().kin_step(ctx, nsteps))


def kin_get_state(ctx, W, n_values=None):
    _elem_check(ctx, W, 8)
    p, dev = _ptr(W)
    n = W.size if isinstance(W, np.ndarray) else W.numel()
    _check(ctx, load_library().kin_get_state(ctx, p, n if n_values is None else n_values, dev))


def kin_get_kinetic(ctx, f, n_values=None):
    _elem_check(ctx, f, _f_bytes(ctx))
    p, dev = _ptr(f)
    n = f.size if isinstance(f, np.ndarray) else f.numel()
    _check(ctx, load_library().kin_get_kinetic(ctx, p, n if n_values is None else n_values, dev))


def kin_diag(ctx, m: int, defect: bool = True):
    """(mass per variable, next-step interface defect, iteration residual);
    defect=False asks for the mass only (the defect and residual are None)."""
    mass = np.zeros(m)
    dfc = np.zeros(m)
    resid = np.zeros(1)
    dp = ctypes.POINTER(ctypes.c_double)
    null = ctypes.POINTER(ctypes.c_double)()
    _check(ctx, load_library().kin_diag(ctx, mass.ctypes.data_as(dp),
                                        dfc.ctypes.data_as(dp) if defect else null,
                                        resid.ctypes.data_as(dp) if defect else null))
    return (mass, dfc, float(resid[0])) if defect else (mass, None, None)


def kin_sync(ctx):
    _check(ctx, load_library().kin_sync(ctx))


def kin_query(ctx) -> kin_info:
    info = kin_info()
    _check(ctx, load_library().kin_query(ctx, ctypes.byref(info)))
    return info


def kin_destroy(ctx):
    _check(None, load_library().kin_destroy(ctx))


def kin_step_noalloc(mesh: kin_mesh, model: kin_model, degree: int, dt: float, opts: kin_opts,
                     f, nsteps: int):
    """Advance the caller's device kinetic state f (a CUDA tensor, updated in
    place) by nsteps steps without any device allocation by the library; its
    scratch is a static 16 MiB device array shared by all calls on a device,
    so calls must not overlap on the GPU.  For callers whose device memory is
    owned by their own allocator or fixed memory plan."""
    p, dev = _ptr(f)
    if not dev:
        raise ValueError("kin_step_noalloc needs a device buffer")
    err = ctypes.create_string_buffer(512)
    st = load_library().kin_step_noalloc(ctypes.byref(mesh), ctypes.byref(model), degree, dt,
                                         ctypes.byref(opts), p, nsteps, err, len(err))
    if st != KIN_OK:
        raise KinError(st, err.value.decode())


def _bcheck(batch, status):
    if status != KIN_OK:
        raise KinError(status, load_library().kin_batch_last_error(batch).decode())


KIN_BATCH_DIRECT = 1
KIN_BATCH_MIXED = 2


def kin_batch_create(ctxs, stream=None):
    """Batch of contexts stepped together (one launch per kernel type per step)."""
    lib = load_library()
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    out = ctypes.c_void_p()
    _bcheck(None, lib.kin_batch_create(arr, len(ctxs), stream, ctypes.byref(out)))
    return out


def kin_batch_create_ex(ctxs, stream=None, flags=0):
    """kin_batch_create with flags (KIN_BATCH_DIRECT: no CUDA graphs)."""
    lib = load_library()
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    out = ctypes.c_void_p()
    _bcheck(None, lib.kin_batch_create_ex(arr, len(ctxs), stream, int(flags), ctypes.byref(out)))
    return out


def kin_batch_step(batch, nsteps: int):
    _bcheck(batch, load_library().kin_batch_step(batch, nsteps))


def kin_batch_sync(batch):
    _bcheck(batch, load_library().kin_batch_sync(batch))


def kin_batch_destroy(batch):
    _bcheck(None, load_library().kin_batch_destroy(batch))


def kin_batch_info(batch):
    """(launches per batch step, members in the mixed-degree launch)."""
    n = ctypes.c_int(0)
    mixed = ctypes.c_int(0)
    _bcheck(batch, load_library().kin_batch_info(batch, ctypes.byref(n), ctypes.byref(mixed)))
    return n.value, mixed.value


def kin_batch_last_error(batch=None) -> str:
    return load_library().kin_batch_last_error(batch).decode()


def kin_last_error(ctx=None) -> str:
    return load_library().kin_last_error(ctx).decode()


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def make_args(dim, n, lo, hi, system, lam, omega=2.0, gamma=1.4, adv=(0.0, 0.0, 0.0),
              tiles=(1, 1, 1), iters=3, precision=KIN_FP64, block=(0, 0, 0), mem_budget=0,
              stream=None, torch_alloc=False, wait_timeout_s=0.0, debug_flags=0, threads=0, stages=0,
              velset=None, sigma=0.0, inflow=(0, 0, 0)):
    pad = lambda t, fill: tuple(t) + (fill,) * (3 - len(tuple(t)))
    mesh = kin_mesh(dim, (ctypes.c_int * 3)(*pad(n, 1)), (ctypes.c_double * 3)(*pad(lo, 0.0)),
                    (ctypes.c_double * 3)(*pad(hi, 1.0)), (ctypes.c_int * 3)(*pad(inflow, 0)))
    model = kin_model(system, dim if velset is None else velset, lam, gamma,
                      (ctypes.c_double * 3)(*pad(adv, 0.0)), omega, sigma)
    opts = kin_opts()
    opts.tiles = (ctypes.c_int * 3)(*pad(tiles, 1))
    opts.iters = iters
    opts.precision = precision
    opts.block = (ctypes.c_int * 3)(*pad(block, 0))
    opts.mem_budget = mem_budget
    opts.stream = stream
    opts.wait_timeout_s = wait_timeout_s
    opts.debug_flags = debug_flags
    opts.threads = threads
    opts.stages = stages
    if torch_alloc:
        a, f = torch_allocator_hooks()
        opts.alloc = a
        opts.free = f
    return mesh, model, opts


class Batch:
    """Owning wrapper of a kin_batch over Context objects (which must outlive it)."""

    def __init__(self, contexts, stream=None, graphs=True, mixed=False):
        self.contexts = list(contexts)
        flags = (0 if graphs else KIN_BATCH_DIRECT) | (KIN_BATCH_MIXED if mixed else 0)
        self.handle = kin_batch_create_ex([c.ctx for c in self.contexts], stream, flags)
        self.launches_per_step, self.mixed_members = kin_batch_info(self.handle)

    def step(self, n=1):
        kin_batch_step(self.handle, n)

    def sync(self):
        kin_batch_sync(self.handle)

    def close(self):
        if self.handle is not None:
            kin_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Context:
    """Owning wrapper of a kin_ctx (create / destroy); the methods call the
    C ABI functions above."""

    def __init__(self, dim, n, lo, hi, degree, system, lam, dt, **kw):
        self.mesh, self.model, self.opts = make_args(dim, n, lo, hi, system, lam, **kw)
        self.ctx = kin_create(self.mesh, self.model, degree, dt, self.opts)
        self.info = kin_query(self.ctx)

    @classmethod
    def from_workload(cls, w, precision=None, **kw):
        prec = precision if precision is not None else (KIN_FP32 if w.precision == "f32" else KIN_FP64)
        vs = {2: KIN_D2Q3, 3: KIN_D3Q4}.get(w.dim) if getattr(w, "velset", 0) == 1 else None
        inflow = tuple(getattr(w, "inflow", (0, 0, 0)))
        ctx = cls(w.dim, w.n, w.lo, w.hi, w.degree, w.system, w.lam, w.dt, omega=w.omega,
                  gamma=w.gamma, adv=w.adv, tiles=w.tiles, iters=w.iters, precision=prec, velset=vs,
                  sigma=getattr(w, "sigma", 0.0), inflow=inflow, **kw)
        if any(inflow):
            Wb = np.asarray(w.Wb, dtype=np.float64)
            for a in range(w.dim):
                if inflow[a]:
                    for side in (0, 1):
                        ctx.set_boundary(a, side, Wb[a, side, :w.m])
        return ctx

    @property
    def dtype(self):
        return np.float32 if self.info.precision == KIN_FP32 else np.float64

    def set_state(self, W):
        kin_set_state(self.ctx, W)

    def set_kinetic(self, f):
        kin_set_kinetic(self.ctx, f)

    def set_boundary(self, axis, side, W):
        kin_set_boundary(self.ctx, axis, side, W)

    def step(self, n=1):
        kin_step(self.ctx, n)

    def get_state(self, out=None):
        if out is None:
            out = np.zeros(self.info.state_values)
        kin_get_state(self.ctx, out)
        return out

    def get_kinetic(self, out=None):
        if out is None:
            out = np.zeros(self.info.kinetic_values, dtype=self.dtype)
        kin_get_kinetic(self.ctx, out)
        return out

    def diag(self):
        return kin_diag(self.ctx, self.info.m)

    def sync(self):
        kin_sync(self.ctx)

    def close(self):
        if self.ctx is not None:
            kin_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class TetContext(Context):
    """Owning wrapper of a kin_ctx on a tetrahedral mesh (kin_create_tet);
    the state and step methods are Context's."""

    def __init__(self, xyz, vid, nbr, sub, wrap, system, velset, lam, dt, omega=2.0, gamma=1.4,
                 adv=(0.0, 0.0, 0.0), sigma=0.0, iters=3, precision=KIN_FP64, mem_budget=0, stream=None,
                 torch_alloc=False):
        self._arrays = [np.ascontiguousarray(xyz, dtype=np.float64), np.ascontiguousarray(vid, dtype=np.int64),
                        np.ascontiguousarray(nbr, dtype=np.int64), np.ascontiguousarray(sub, dtype=np.int32),
                        np.ascontiguousarray(wrap, dtype=np.int32)]
        x, v, nb, sb, wr = self._arrays
        self.mesh = kin_tetmesh(v.shape[0], x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                v.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                                nb.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                                sb.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                wr.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        _, self.model, self.opts = make_args(3, (1, 1, 1), (0, 0, 0), (1, 1, 1), system, lam, omega=omega,
                                             gamma=gamma, adv=adv, iters=iters, precision=precision,
                                             mem_budget=mem_budget, stream=stream, torch_alloc=torch_alloc,
                                             velset=velset, sigma=sigma)
        self.ctx = kin_create_tet(self.mesh, self.model, dt, self.opts)
        self.info = kin_query(self.ctx)

    @classmethod
    def from_workload(cls, w, precision=None, **kw):
        prec = precision if precision is not None else (KIN_FP32 if w.precision == "f32" else KIN_FP64)
        m = w.mesh
        return cls(m.xyz, m.vid, m.nbr, w.subdomains(), m.wrap, w.system, KIN_D3Q4 if w.velset == 1 else KIN_D3Q6,
                   w.lam, w.dt, omega=w.omega, gamma=w.gamma, adv=w.adv, sigma=w.sigma, iters=w.iters,
                   precision=prec, **kw)
