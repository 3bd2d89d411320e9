"""GB300-native N-body hot path (softened gravity and the Lennard-Jones law):
Python binding of libnbody.

Argument marshalling only: every step of the path (staging, all-pairs forces,
KDK leapfrog, reductions, adjoint) runs in the sm_103a kernels of
``libnbody.so`` through its C ABI (``include/nbody.h``). PyTorch supplies
device memory and streams. There is no CPU fallback: if the library is
missing, ``load()`` raises.

Functions carry the C names: ``nbody_init``, ``nbody_forces``, ``nbody_step``,
``nbody_energy``, ``nbody_virial``, ``nbody_adjoint``, ``nbody_adjoint_params``,
``nbody_step_host``, ``nbody_forces_noalloc``, ``nbody_sync``, ``nbody_get_tuning``,
``nbody_profile``, ``nbody_kernel_time``, ``nbody_launch_count``, ``nbody_last_error``,
``nbody_destroy``, ``nbody_version``. ``NBodyAdjoint`` wraps the forward
``nbody_step`` and the reverse ``nbody_adjoint`` as a torch.autograd.Function.
"""

from __future__ import annotations

import ctypes
import os
import threading

__all__ = [
    "FP64", "MIXED", "GRAVITY", "LENNARD_JONES", "FLAG_GRAPH", "FLAG_NOCHECK", "NBodyError", "Context", "load", "lib_path",
    "nbody_init", "nbody_forces", "nbody_step", "nbody_energy", "nbody_virial", "nbody_adjoint",
    "nbody_adjoint_params",
    "nbody_step_host",
    "nbody_sync", "nbody_get_tuning", "nbody_get_slicing", "nbody_launch_count", "nbody_last_error", "nbody_destroy",
    "nbody_version", "nbody_build_flags", "nbody_profile", "nbody_kernel_time", "nbody_forces_noalloc", "NOALLOC_MAX_BODIES",
    "NBodyAdjoint", "ENERGY_FIELDS",
]

FP64, MIXED = 0, 1
GRAVITY, LENNARD_JONES = 0, 1
FLAG_GRAPH, FLAG_NOCHECK = 1, 2
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENONFINITE", 6: "EUNSUPPORTED",
          7: "EINTERNAL"}
ENERGY_FIELDS = ("E", "K", "U", "Px", "Py", "Pz", "Lx", "Ly", "Lz")

_HERE = os.path.dirname(os.path.abspath(__file__))
# NBODY_DEBUG_LIB=1 selects the build with device-side index checks (build.build(debug=True))
_LIB_PATH = os.path.join(_HERE, "libnbody_debug.so" if os.environ.get("NBODY_DEBUG_LIB") == "1" else "libnbody.so")
_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _LIB_PATH


class NBodyError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class _Config(ctypes.Structure):
    _fields_ = [
        ("G", ctypes.c_double), ("eps", ctypes.c_double), ("dt", ctypes.c_double),
        ("precision", ctypes.c_int32), ("energy_every", ctypes.c_int32), ("block", ctypes.c_int32),
        ("i_per_thread", ctypes.c_int32), ("j_tile", ctypes.c_int32), ("slice", ctypes.c_int32),
        ("flags", ctypes.c_uint32), ("variant", ctypes.c_int32), ("law", ctypes.c_int32),
        ("reserved", ctypes.c_int32), ("lj_epsilon", ctypes.c_double), ("lj_sigma", ctypes.c_double),
        ("box", ctypes.c_double),
    ]


def load():
    """Loads libnbody.so (built by ``paper_2511_02655_gb300.build``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{os.path.basename(_LIB_PATH)} not found at {_LIB_PATH}: run "
                               "paper_2511_02655_gb300.build.build()")
        try:  # let the library resolve the CUDA runtime torch already loaded
            import torch  # noqa: F401
        except Exception:
            pass
        lib = ctypes.CDLL(_LIB_PATH)
        p, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        sigs = {
            "nbody_init": (i32, [ctypes.POINTER(p), ctypes.POINTER(_Config), i64, p, p]),
            "nbody_set_stream": (i32, [p, p]),
            "nbody_forces": (i32, [p, p, p, p, p]),
            "nbody_step": (i32, [p, p, p, p, p, i32, i32, p]),
            "nbody_energy": (i32, [p, p, p, p, p]),
            "nbody_virial": (i32, [p, p, p, p, p]),
            "nbody_adjoint": (i32, [p, p, p, p, i32, i32, p, p, p, p, p]),
            "nbody_adjoint_params": (i32, [p, p, p, p, i32, i32, p, p, p, p, p, p]),
            "nbody_step_host": (i32, [p, p, p, p, p, i32, i32, p]),
            "nbody_sync": (i32, [p]),
            "nbody_get_tuning": (i32, [p] + [ctypes.POINTER(i32)] * 6),
            "nbody_get_slicing": (i32, [p] + [ctypes.POINTER(i32)] * 3),
            "nbody_launch_count": (i64, [p]),
            "nbody_profile": (i32, [p, i32]),
            "nbody_kernel_time": (i32, [p, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]),
            "nbody_last_error": (ctypes.c_char_p, [p]),
            "nbody_forces_noalloc": (i32, [p, p, i64, ctypes.c_double, ctypes.c_double, p, p, p]),
            "nbody_destroy": (None, [p]),
            "nbody_version": (i32, []),
            "nbody_build_flags": (i32, []),
        }
        for name, (res, args) in sigs.items():
            f = getattr(lib, name)
            f.restype, f.argtypes = res, args
        _lib = lib
        return lib


def nbody_version() -> int:
    return int(load().nbody_version())


def nbody_build_flags() -> int:
    """Build options of the loaded library (bit 0: NBODY_DEBUG device-side index checks)."""
    return int(load().nbody_build_flags())


def nbody_last_error(ctx=None) -> str:
    h = ctx._h if isinstance(ctx, Context) else None
    return load().nbody_last_error(h).decode()


class Context:
    """Owns one ``nbody_ctx``; freed by ``nbody_destroy`` / ``close`` / garbage collection."""

    def __init__(self, handle, cfg: _Config, offsets, stream_ptr):
        self._h = handle
        self.cfg = cfg
        self.offsets = [int(o) for o in offsets]
        self.n_systems = len(self.offsets) - 1
        self.n_total = self.offsets[-1]
        self.precision = cfg.precision
        self._stream = stream_ptr

    def close(self):
        if self._h:
            load().nbody_destroy(self._h)
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


def _check(status: int, ctx=None):
    if status != 0:
        raise NBodyError(status, nbody_last_error(ctx))


def _torch():
    import torch
    return torch


def _bind_stream(ctx: Context):
    torch = _torch()
    s = torch.cuda.current_stream().cuda_stream
    if s != ctx._stream:
        _check(load().nbody_set_stream(ctx._h, ctx_ptr(s)), ctx)
        ctx._stream = s


def ctx_ptr(v):
    return ctypes.c_void_p(v) if v else None


def _dev(t, name, shape, ctx: Context, allow_none=False):
    """Validates a CUDA float64 C-contiguous tensor and returns its address."""
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctx_ptr(t.data_ptr())


def nbody_init(*, G=1.0, eps=0.0, dt=0.0, precision=MIXED, offsets=None, n=None, energy_every=0, block=0,
               i_per_thread=0, j_tile=0, slice=0, flags=0, variant=0, law=GRAVITY, lj_epsilon=1.0, lj_sigma=1.0,
               box=0.0, stream=None) -> Context:
    """Creates a context for systems with row ranges ``offsets`` (or one system of ``n`` bodies).

    Tile parameters (and the mixed kernel ``variant``: 1 scalar, 2 packed, 3 packed under
    a register cap: 4 CTAs per SM for gravity, 6 for Lennard-Jones) left at 0 are chosen by
    the autotuner during init. ``law``: GRAVITY (G, eps) or
    LENNARD_JONES (lj_epsilon, lj_sigma; eps softens r^2); ``box`` > 0 adds
    reflecting walls of the cube [0, box]^3.
    ``stream``: a torch.cuda.Stream (default: the current stream).
    """
    torch = _torch()
    lib = load()
    if offsets is None:
        if n is None:
            raise ValueError("give offsets or n")
        offsets = [0, int(n)]
    offs = (ctypes.c_int64 * len(offsets))(*[int(o) for o in offsets])
    cfg = _Config(float(G), float(eps), float(dt), int(precision), int(energy_every), int(block),
                  int(i_per_thread), int(j_tile), int(slice), int(flags), int(variant), int(law), 0,
                  float(lj_epsilon), float(lj_sigma), float(box))
    s = (stream or torch.cuda.current_stream()).cuda_stream
    h = ctypes.c_void_p()
    _check(lib.nbody_init(ctypes.byref(h), ctypes.byref(cfg), len(offsets) - 1, offs, ctx_ptr(s)))
    return Context(h, cfg, offsets, s)


def nbody_forces(ctx: Context, x, m, a=None, phi=None, with_phi=True):
    """a [N,3], phi [N] (or None) for positions x [N,3] and masses m [N]."""
    torch = _torch()
    n = ctx.n_total
    if a is None:
        a = torch.empty((n, 3), dtype=torch.float64, device=x.device)
    if phi is None and with_phi:
        phi = torch.empty((n,), dtype=torch.float64, device=x.device)
    args = (_dev(x, "x", (n, 3), ctx), _dev(m, "m", (n,), ctx), _dev(a, "a", (n, 3), ctx),
            _dev(phi, "phi", (n,), ctx, allow_none=True))
    _bind_stream(ctx)
    _check(load().nbody_forces(ctx._h, *args), ctx)
    return a, phi


def nbody_step(ctx: Context, x, v, m, a, a_valid: bool, n_steps: int, energy_log=None):
    """In-place KDK steps on (x, v, a); returns energy_log (allocated if energy_every > 0 and None given)."""
    torch = _torch()
    n = ctx.n_total
    every = ctx.cfg.energy_every
    nrec = n_steps // every if every > 0 else 0
    if energy_log is None and nrec > 0:
        energy_log = torch.empty((nrec, ctx.n_systems, 9), dtype=torch.float64, device=x.device)
    elog = _dev(energy_log, "energy_log", (nrec, ctx.n_systems, 9), ctx, allow_none=True) if nrec > 0 else None
    args = (_dev(x, "x", (n, 3), ctx), _dev(v, "v", (n, 3), ctx), _dev(m, "m", (n,), ctx), _dev(a, "a", (n, 3), ctx))
    _bind_stream(ctx)
    _check(load().nbody_step(ctx._h, *args, int(bool(a_valid)), int(n_steps), elog), ctx)
    return energy_log


def nbody_energy(ctx: Context, x, v, m, out=None):
    """[n_systems, 9] = (E, K, U, Px, Py, Pz, Lx, Ly, Lz) per system."""
    torch = _torch()
    n = ctx.n_total
    if out is None:
        out = torch.empty((ctx.n_systems, 9), dtype=torch.float64, device=x.device)
    args = (_dev(x, "x", (n, 3), ctx), _dev(v, "v", (n, 3), ctx), _dev(m, "m", (n,), ctx),
            _dev(out, "out", (ctx.n_systems, 9), ctx))
    _bind_stream(ctx)
    _check(load().nbody_energy(ctx._h, *args), ctx)
    return out


def nbody_virial(ctx: Context, x, v, m, out=None):
    """[n_systems, 3] = (K, W, Q): kinetic energy, Clausius virial sum m x.a, ratio -2K/W."""
    torch = _torch()
    n = ctx.n_total
    if out is None:
        out = torch.empty((ctx.n_systems, 3), dtype=torch.float64, device=x.device)
    args = (_dev(x, "x", (n, 3), ctx), _dev(v, "v", (n, 3), ctx), _dev(m, "m", (n,), ctx),
            _dev(out, "out", (ctx.n_systems, 3), ctx))
    _bind_stream(ctx)
    _check(load().nbody_virial(ctx._h, *args), ctx)
    return out


def nbody_adjoint(ctx: Context, x0, v0, m, n_steps: int, checkpoint_every: int, lam_xT, lam_vT, g_x0=None,
                  g_v0=None, g_m=None):
    """(dL/dx0, dL/dv0, dL/dm) given dL/dx_T and dL/dv_T after n_steps KDK steps from (x0, v0)."""
    torch = _torch()
    n = ctx.n_total
    dev = x0.device
    g_x0 = torch.empty((n, 3), dtype=torch.float64, device=dev) if g_x0 is None else g_x0
    g_v0 = torch.empty((n, 3), dtype=torch.float64, device=dev) if g_v0 is None else g_v0
    g_m = torch.empty((n,), dtype=torch.float64, device=dev) if g_m is None else g_m
    args = (_dev(x0, "x0", (n, 3), ctx), _dev(v0, "v0", (n, 3), ctx), _dev(m, "m", (n,), ctx), int(n_steps),
            int(checkpoint_every), _dev(lam_xT, "lam_xT", (n, 3), ctx), _dev(lam_vT, "lam_vT", (n, 3), ctx),
            _dev(g_x0, "g_x0", (n, 3), ctx), _dev(g_v0, "g_v0", (n, 3), ctx), _dev(g_m, "g_m", (n,), ctx))
    _bind_stream(ctx)
    _check(load().nbody_adjoint(ctx._h, *args), ctx)
    return g_x0, g_v0, g_m


def nbody_adjoint_params(ctx: Context, x0, v0, m, n_steps: int, checkpoint_every: int, lam_xT, lam_vT):
    """``nbody_adjoint`` plus g_params [n_systems, 2] = (dL/dG, dL/deps) per system."""
    torch = _torch()
    n = ctx.n_total
    dev = x0.device
    g_x0 = torch.empty((n, 3), dtype=torch.float64, device=dev)
    g_v0 = torch.empty((n, 3), dtype=torch.float64, device=dev)
    g_m = torch.empty((n,), dtype=torch.float64, device=dev)
    g_p = torch.empty((ctx.n_systems, 2), dtype=torch.float64, device=dev)
    args = (_dev(x0, "x0", (n, 3), ctx), _dev(v0, "v0", (n, 3), ctx), _dev(m, "m", (n,), ctx), int(n_steps),
            int(checkpoint_every), _dev(lam_xT, "lam_xT", (n, 3), ctx), _dev(lam_vT, "lam_vT", (n, 3), ctx),
            _dev(g_x0, "g_x0", (n, 3), ctx), _dev(g_v0, "g_v0", (n, 3), ctx), _dev(g_m, "g_m", (n,), ctx),
            _dev(g_p, "g_params", (ctx.n_systems, 2), ctx))
    _bind_stream(ctx)
    _check(load().nbody_adjoint_params(ctx._h, *args), ctx)
    return g_x0, g_v0, g_m, g_p


def _host(t, name, shape):
    import numpy as np
    torch = _torch()
    if isinstance(t, torch.Tensor):
        if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} must be a contiguous CPU float64 tensor of shape {tuple(shape)}")
        return ctx_ptr(t.data_ptr())
    if isinstance(t, np.ndarray):
        if t.dtype != np.float64 or not t.flags.c_contiguous or t.shape != tuple(shape):
            raise ValueError(f"{name} must be a C-contiguous float64 array of shape {tuple(shape)}")
        return ctx_ptr(t.ctypes.data)
    raise TypeError(f"{name} must be a CPU tensor or numpy array")


def nbody_step_host(ctx: Context, x, v, m, a, a_valid: bool, n_steps: int, energy_log=None):
    """nbody_step on host arrays (CPU tensors, ideally pinned, or numpy); synchronises before returning."""
    n = ctx.n_total
    every = ctx.cfg.energy_every
    nrec = n_steps // every if every > 0 else 0
    elog = _host(energy_log, "energy_log", (nrec, ctx.n_systems, 9)) if (energy_log is not None and nrec) else None
    args = (_host(x, "x", (n, 3)), _host(v, "v", (n, 3)), _host(m, "m", (n,)), _host(a, "a", (n, 3)))
    _bind_stream(ctx)
    _check(load().nbody_step_host(ctx._h, *args, int(bool(a_valid)), int(n_steps), elog), ctx)
    return energy_log


def nbody_sync(ctx: Context):
    _check(load().nbody_sync(ctx._h), ctx)


def nbody_get_tuning(ctx: Context) -> dict:
    """Tiling in use (nbody_get_tuning) and the work list's shape (nbody_get_slicing)."""
    vals = [ctypes.c_int32() for _ in range(6)]
    _check(load().nbody_get_tuning(ctx._h, *[ctypes.byref(v) for v in vals]), ctx)
    out = dict(zip(("block", "i_per_thread", "j_tile", "slice", "n_ctas", "variant"), (v.value for v in vals)))
    out.update(nbody_get_slicing(ctx))
    return out


def nbody_get_slicing(ctx: Context) -> dict:
    """Work-list shape of the force pass: tail (0 equal slices, 1 halving tail), n_items, max_slices."""
    sl = [ctypes.c_int32() for _ in range(3)]
    _check(load().nbody_get_slicing(ctx._h, *[ctypes.byref(v) for v in sl]), ctx)
    return dict(zip(("tail", "n_items", "max_slices"), (v.value for v in sl)))


def nbody_launch_count(ctx: Context) -> int:
    return int(load().nbody_launch_count(ctx._h))


def nbody_profile(ctx: Context, enable: bool = True):
    """Starts (clearing the counters) or stops event timing of the all-pairs kernel launches."""
    _check(load().nbody_profile(ctx._h, int(bool(enable))), ctx)


def nbody_kernel_time(ctx: Context, which: int = 0):
    """(summed milliseconds, launches) of the timed force (which=0) or VJP (which=1) kernels."""
    ms, k = ctypes.c_double(), ctypes.c_int64()
    _check(load().nbody_kernel_time(ctx._h, int(which), ctypes.byref(ms), ctypes.byref(k)), ctx)
    return ms.value, k.value


NOALLOC_MAX_BODIES = 1048576


def nbody_forces_noalloc(x, m, G, eps, a=None, phi=None):
    """Forces of one system through the allocation-free entry point (no context).

    For callers that cannot allocate device memory at this point: the library
    uses a fixed static device array as scratch (the first call on a device
    loads it; make that call early). Output tensors are allocated here by torch
    only when not supplied. Calls overlapping on the GPU race on the shared
    scratch.
    """
    torch = _torch()
    n = int(m.shape[0])

    def check(t, name, shape):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
                and tuple(t.shape) == shape and t.device == x.device):
            raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of shape {shape} on {x.device}")

    if not isinstance(x, torch.Tensor):
        raise ValueError("x must be a CUDA tensor")
    check(x, "x", (n, 3))
    check(m, "m", (n,))
    if a is None:
        a = torch.empty((n, 3), dtype=torch.float64, device=x.device)
    check(a, "a", (n, 3))
    if phi is not None:
        check(phi, "phi", (n,))
    stream = torch.cuda.current_stream(x.device).cuda_stream
    with torch.cuda.device(x.device):
        st = load().nbody_forces_noalloc(ctx_ptr(x.data_ptr()), ctx_ptr(m.data_ptr()), n, float(G), float(eps),
                                         ctx_ptr(a.data_ptr()), ctx_ptr(phi.data_ptr()) if phi is not None else None,
                                         ctx_ptr(stream))
    _check(st)
    return a, phi


def nbody_destroy(ctx: Context):
    ctx.close()


def _make_adjoint_function():
    torch = _torch()

    class NBodyAdjoint(torch.autograd.Function):
        """(x_T, v_T) = KDK^n(x0, v0; m) with a hand-written reverse pass.

        forward runs ``nbody_step``; backward runs ``nbody_adjoint``, which
        recomputes the trajectory from checkpoints every ``checkpoint_every``
        steps and applies the force-VJP kernel in reverse.
        """

        @staticmethod
        def forward(fctx, ctx: Context, x0, v0, m, n_steps: int, checkpoint_every: int):
            x = x0.detach().clone()
            v = v0.detach().clone()
            a = torch.empty_like(x)
            nbody_step(ctx, x, v, m.detach(), a, False, n_steps)
            fctx.save_for_backward(x0.detach(), v0.detach(), m.detach())
            fctx.nb = (ctx, int(n_steps), int(checkpoint_every))
            return x, v

        @staticmethod
        def backward(fctx, gx, gv):
            x0, v0, m = fctx.saved_tensors
            ctx, n_steps, k = fctx.nb
            gx = torch.zeros_like(x0) if gx is None else gx.contiguous()
            gv = torch.zeros_like(v0) if gv is None else gv.contiguous()
            g_x0, g_v0, g_m = nbody_adjoint(ctx, x0, v0, m, n_steps, k, gx, gv)
            return None, g_x0, g_v0, g_m, None, None

    return NBodyAdjoint


class _LazyAdjoint:
    _cls = None

    def __getattr__(self, item):
        if _LazyAdjoint._cls is None:
            _LazyAdjoint._cls = _make_adjoint_function()
        return getattr(_LazyAdjoint._cls, item)


NBodyAdjoint = _LazyAdjoint()
