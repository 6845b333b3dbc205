"""Thin ctypes binding of liblbm.so (C-ABI declared in include/lbm.h).

Argument marshalling only: every step of the method runs in the CUDA library.  Arrays are
passed as raw pointers -- torch tensors (CUDA or CPU) or numpy arrays, float32 and
C-contiguous -- and the library tells device from host memory itself.  A missing library is an
error (there is no CPU fallback): build it with ``python -m paper_1311_7239_gb300.build``.
"""
from __future__ import annotations

import ctypes
import math
import os

PKG = os.path.dirname(os.path.abspath(__file__))
# LBM_LIBRARY selects another build of the library (e.g. liblbm_debug.so, with kernel index checks)
LIB_PATH = os.environ.get("LBM_LIBRARY") or os.path.join(PKG, "liblbm.so")

ABI_VERSION = 2
FP32, FP16_DEV, BF16_DEV = 0, 1, 2
PERIODIC, WALL, PRESSURE, NEE = 0, 1, 2, 3
STREAM_AB, STREAM_INPLACE = 0, 1
OPT_NO_RESIDUAL_RECORD = 1
TILING_ROWS, TILING_FLAT = 0, 1
LEFT, RIGHT, BOTTOM, TOP = 0, 1, 2, 3
CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy
LOSS_OUTLET_FLUX, LOSS_VELOCITY_MISFIT = 0, 1
OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ETIMEOUT, EABI, ESTATE = 0, -1, -2, -3, -4, -5, -6, -7

# Every function the header declares, with its ctypes signature.
_c_ctx = ctypes.c_void_p
_f32p = ctypes.c_void_p


class Config(ctypes.Structure):
    """Mirror of ``lbm_config`` (field order and types as in include/lbm.h)."""

    _fields_ = [
        ("abi_version", ctypes.c_uint32),
        ("nx", ctypes.c_uint32),
        ("ny", ctypes.c_uint32),
        ("precision", ctypes.c_uint32),
        ("bc_x", ctypes.c_uint32),
        ("bc_y", ctypes.c_uint32),
        ("forchheimer", ctypes.c_int32),
        ("thermal", ctypes.c_int32),
        ("nu", ctypes.c_double),
        ("J", ctypes.c_double),
        ("rho0", ctypes.c_double),
        ("s_e", ctypes.c_double),
        ("s_q", ctypes.c_double),
        ("ax", ctypes.c_double),
        ("ay", ctypes.c_double),
        ("phi", ctypes.c_double),
        ("K", ctypes.c_double),
        ("u_wall", (ctypes.c_double * 2) * 4),
        ("p_in", ctypes.c_double),
        ("p_out", ctypes.c_double),
        ("p_rest", ctypes.c_double),
        ("dev_scale_log2", ctypes.c_int32),
        ("tau_T", ctypes.c_double),
        ("zeta3", ctypes.c_double),
        ("zeta4", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("g_beta", ctypes.c_double),
        ("T0", ctypes.c_double),
        ("T_wall", ctypes.c_double * 4),
        ("stream", ctypes.c_void_p),
        ("streaming", ctypes.c_uint32),
        ("options", ctypes.c_uint32),
    ]


SIGNATURES = {
    "lbm_config_defaults": (None, [ctypes.POINTER(Config)]),
    "lbm_config_size": (ctypes.c_uint32, []),
    "lbm_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(_c_ctx)]),
    "lbm_destroy": (None, [_c_ctx]),
    "lbm_set_medium": (ctypes.c_int, [_c_ctx, _f32p, _f32p]),
    "lbm_set_medium_log": (ctypes.c_int, [_c_ctx, _f32p, _f32p]),
    "lbm_set_viscosity_ratio": (ctypes.c_int, [_c_ctx, _f32p]),
    "lbm_init_equilibrium": (ctypes.c_int, [_c_ctx, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int]),
    "lbm_init_temperature": (ctypes.c_int, [_c_ctx, ctypes.c_double]),
    "lbm_step": (ctypes.c_int, [_c_ctx, ctypes.c_int]),
    "lbm_set_walls": (ctypes.c_int, [_c_ctx, _f32p]),
    "lbm_probe": (ctypes.c_int, [_c_ctx, ctypes.c_int, ctypes.c_int, _f32p]),
    "lbm_probe_async": (ctypes.c_int, [_c_ctx, ctypes.c_int, ctypes.c_int, _f32p]),
    "lbm_macros": (ctypes.c_int, [_c_ctx, _f32p, _f32p, _f32p, _f32p]),
    "lbm_get_populations": (ctypes.c_int, [_c_ctx, _f32p, _f32p]),
    "lbm_set_populations": (ctypes.c_int, [_c_ctx, _f32p, _f32p]),
    "lbm_residual": (ctypes.c_int, [_c_ctx, ctypes.POINTER(ctypes.c_double)]),
    "lbm_nusselt": (ctypes.c_int, [_c_ctx, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "lbm_adjoint": (ctypes.c_int, [_c_ctx, ctypes.c_int, ctypes.c_int, _f32p, _f32p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p]),
    "lbm_adjoint_step": (ctypes.c_int, [_c_ctx, ctypes.c_int, ctypes.c_int, _f32p, _f32p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "lbm_release_workspace": (ctypes.c_int, [_c_ctx]),
    "lbm_residual_noalloc": (ctypes.c_int, [_f32p, _f32p, _f32p, _f32p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "lbm_sync": (ctypes.c_int, [_c_ctx]),
    "lbm_save": (ctypes.c_int, [_c_ctx, ctypes.c_char_p]),
    "lbm_load": (ctypes.c_int, [_c_ctx, ctypes.c_char_p]),
    "lbm_step_count": (ctypes.c_int, [_c_ctx, ctypes.POINTER(ctypes.c_int64)]),
    "lbm_memory_bytes": (ctypes.c_int, [_c_ctx, ctypes.POINTER(ctypes.c_uint64)]),
    "lbm_batch_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "lbm_create_batch": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "lbm_batch_destroy": (None, [ctypes.c_void_p]),
    "lbm_batch_set_medium": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _f32p, _f32p]),
    "lbm_batch_init_equilibrium": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_double, ctypes.c_int]),
    "lbm_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lbm_batch_step_each": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lbm_batch_set_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "lbm_batch_get_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "lbm_batch_set_items_per_cta": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lbm_batch_get_items_per_cta": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "lbm_batch_set_tiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lbm_batch_get_tiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "lbm_batch_tune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_float)]),
    "lbm_batch_macros": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _f32p, _f32p, _f32p]),
    "lbm_batch_get_populations": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _f32p]),
    "lbm_batch_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_uint64)]),
    "lbm_batch_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "lbm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "lbm_last_error": (ctypes.c_char_p, []),
}

_LIB = None


class LbmError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {msg} (status {code})")
        self.code = code


def lib():
    """The loaded liblbm.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1311_7239_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        if L.lbm_config_size() != ctypes.sizeof(Config):
            raise RuntimeError("lbm_config layout of the binding differs from the library's")
        _LIB = L
    return _LIB


def _check(rc: int, where: str):
    if rc != OK:
        L = lib()
        raise LbmError(rc, where, L.lbm_last_error().decode() or L.lbm_strerror(rc).decode())


def _ptr(a, writable=False):
    """Raw address of a float32 C-contiguous torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch
        import torch

        if a.dtype != torch.float32 or not a.is_contiguous():
            raise TypeError("expected a contiguous float32 tensor")
        return a.data_ptr()
    import numpy as np

    if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("expected a C-contiguous float32 array")
    if writable and not a.flags["WRITEABLE"]:
        raise TypeError("output array is read-only")
    return a.ctypes.data


def default_config(**kw) -> Config:
    cfg = Config()
    lib().lbm_config_defaults(ctypes.byref(cfg))
    for k, v in kw.items():
        if k == "u_wall":
            for w, (ux, uy) in enumerate(v):
                cfg.u_wall[w][0], cfg.u_wall[w][1] = float(ux), float(uy)
        elif k == "T_wall":
            for w, t in enumerate(v):
                cfg.T_wall[w] = math.nan if t is None else float(t)
        else:
            setattr(cfg, k, v)
    return cfg


class Lattice:
    """One lattice context (``lbm_ctx``) on the current CUDA device.

    Outputs of the read-out methods are torch tensors on the context's device unless ``out``
    arrays are given.  By default the context runs on torch's current CUDA stream.  Keyword
    arguments are ``lbm_config`` fields, e.g. ``streaming=STREAM_INPLACE`` for one population
    buffer updated in place (every side kind; ``options=OPT_NO_RESIDUAL_RECORD`` also drops the
    residual's velocity record).
    """

    def __init__(self, cfg: Config | None = None, **kw):
        import torch

        if cfg is None:
            cfg = default_config(**kw)
        if not cfg.stream:
            # torch's default stream is the legacy default stream (handle 0); pass
            # cudaStreamLegacy (handle 1) so the library orders its work with torch's.
            cfg.stream = torch.cuda.current_stream().cuda_stream or CUDA_STREAM_LEGACY
        self.cfg = cfg
        self.nx, self.ny = int(cfg.nx), int(cfg.ny)
        self.thermal = bool(cfg.thermal)
        self.device = torch.device("cuda", torch.cuda.current_device())
        h = ctypes.c_void_p()
        _check(lib().lbm_create(ctypes.byref(cfg), ctypes.byref(h)), "lbm_create")
        self._h = h

    # lifetime -----------------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_destroy(self._h)
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

    # set-up -------------------------------------------------------------------------------
    def set_medium(self, eps=None, K=None):
        _check(lib().lbm_set_medium(self._h, _ptr(eps), _ptr(K)), "lbm_set_medium")

    def set_viscosity_ratio(self, J=None):
        _check(lib().lbm_set_viscosity_ratio(self._h, _ptr(J)), "lbm_set_viscosity_ratio")

    def set_medium_log(self, eps=None, logK=None):
        _check(lib().lbm_set_medium_log(self._h, _ptr(eps), _ptr(logK)), "lbm_set_medium_log")

    def init_equilibrium(self, p0=1.0, ux0=0.0, uy0=0.0, phi_p_uniform=False):
        _check(lib().lbm_init_equilibrium(self._h, p0, ux0, uy0, int(bool(phi_p_uniform))), "lbm_init_equilibrium")

    def init_temperature(self, T_init):
        _check(lib().lbm_init_temperature(self._h, T_init), "lbm_init_temperature")

    # time stepping --------------------------------------------------------------------------
    def step(self, n=1):
        _check(lib().lbm_step(self._h, int(n)), "lbm_step")

    def sync(self):
        _check(lib().lbm_sync(self._h), "lbm_sync")

    def save(self, path):
        _check(lib().lbm_save(self._h, os.fsencode(path)), "lbm_save")

    def load(self, path):
        _check(lib().lbm_load(self._h, os.fsencode(path)), "lbm_load")

    def step_count(self):
        v = ctypes.c_int64()
        _check(lib().lbm_step_count(self._h, ctypes.byref(v)), "lbm_step_count")
        return v.value

    def memory_bytes(self):
        v = ctypes.c_uint64()
        _check(lib().lbm_memory_bytes(self._h, ctypes.byref(v)), "lbm_memory_bytes")
        return v.value

    def set_walls(self, u_wall):
        """u_wall: float32 [4, 2] (left, right, bottom, top), torch tensor or numpy array."""
        _check(lib().lbm_set_walls(self._h, _ptr(u_wall)), "lbm_set_walls")

    # read-outs ------------------------------------------------------------------------------
    def probe(self, x, y, out=None):
        """(p, ux, uy, T) of cell (x, y); out: float32 [4] host or device array."""
        import numpy as np

        out = np.empty(4, np.float32) if out is None else out
        _check(lib().lbm_probe(self._h, int(x), int(y), _ptr(out, True)), "lbm_probe")
        return out

    def probe_async(self, x, y, out):
        """Enqueue the read of (p, ux, uy, T) of cell (x, y) into out (float32 [4]: pinned host or
        device tensor) on the context's stream without waiting; out is valid once the stream has
        passed this point (``sync``, or an event recorded after the call)."""
        _check(lib().lbm_probe_async(self._h, int(x), int(y), _ptr(out, True)), "lbm_probe_async")
        return out

    def _new(self, *shape):
        import torch

        return torch.empty(shape, dtype=torch.float32, device=self.device)

    def macros(self, p=None, ux=None, uy=None, T=None, want_T=None):
        """(p, ux, uy[, T]) of the current pre-collision state; [ny, nx] float32 each."""
        want_T = self.thermal if want_T is None else want_T
        p = self._new(self.ny, self.nx) if p is None else p
        ux = self._new(self.ny, self.nx) if ux is None else ux
        uy = self._new(self.ny, self.nx) if uy is None else uy
        if want_T and T is None:
            T = self._new(self.ny, self.nx)
        _check(lib().lbm_macros(self._h, _ptr(p, True), _ptr(ux, True), _ptr(uy, True), _ptr(T, True)), "lbm_macros")
        return (p, ux, uy, T) if want_T else (p, ux, uy)

    def write_fields(self, path):
        """Write p, ux, uy (and T) of the current state to a NumPy .npz file (float32 [ny, nx] arrays,
        row 0 at the bottom), with the step count."""
        import numpy as np

        fields = self.macros()
        names = ("p", "ux", "uy", "T")[: len(fields)]
        np.savez(path, step=np.int64(self.step_count()), **{k: v.cpu().numpy() for k, v in zip(names, fields)})

    def get_populations(self, f=None, g=None):
        f = self._new(8, self.ny, self.nx) if f is None else f
        if self.thermal and g is None:
            g = self._new(5, self.ny, self.nx)
        _check(lib().lbm_get_populations(self._h, _ptr(f, True), _ptr(g, True)), "lbm_get_populations")
        return (f, g) if self.thermal else f

    def set_populations(self, f=None, g=None):
        _check(lib().lbm_set_populations(self._h, _ptr(f), _ptr(g)), "lbm_set_populations")

    def residual(self):
        r = ctypes.c_double()
        _check(lib().lbm_residual(self._h, ctypes.byref(r)), "lbm_residual")
        return r.value

    def adjoint(self, T, loss="flux", target=None):
        """(L, dL/dlogK, dL/deps) of T steps from the current initial state (float64 [ny, nx] tensors)."""
        import torch

        kind = {"flux": LOSS_OUTLET_FLUX, "misfit": LOSS_VELOCITY_MISFIT}[loss]
        gk = torch.zeros(self.ny, self.nx, dtype=torch.float64, device=self.device)
        ge = torch.zeros(self.ny, self.nx, dtype=torch.float64, device=self.device)
        L = torch.zeros(1, dtype=torch.float64, device=self.device)
        tx, ty = (None, None) if target is None else target
        _check(lib().lbm_adjoint(self._h, int(T), kind, _ptr(tx), _ptr(ty), gk.data_ptr(), ge.data_ptr(), L.data_ptr()),
               "lbm_adjoint")
        return float(L.item()), gk, ge

    def release_workspace(self):
        """Free the adjoint workspace kept between adjoint calls."""
        _check(lib().lbm_release_workspace(self._h), "lbm_release_workspace")

    def nusselt(self, side=LEFT):
        v = ctypes.c_double()
        _check(lib().lbm_nusselt(self._h, int(side), ctypes.byref(v)), "lbm_nusselt")
        return v.value


class Batch:
    """Ensemble of independent lattices advanced together (``lbm_batch``)."""

    def __init__(self, cfgs):
        import torch

        arr = (Config * len(cfgs))(*cfgs)
        if not arr[0].stream:
            arr[0].stream = torch.cuda.current_stream().cuda_stream or CUDA_STREAM_LEGACY
        self.cfgs = list(arr)
        self.shapes = [(int(c.ny), int(c.nx)) for c in arr]
        self.device = torch.device("cuda", torch.cuda.current_device())
        h = ctypes.c_void_p()
        _check(lib().lbm_batch_create(arr, len(cfgs), ctypes.byref(h)), "lbm_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_batch_destroy(self._h)
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

    def __len__(self):
        return len(self.shapes)

    def set_medium(self, d, eps=None, K=None):
        _check(lib().lbm_batch_set_medium(self._h, int(d), _ptr(eps), _ptr(K)), "lbm_batch_set_medium")

    def init_equilibrium(self, d=-1, p0=1.0, ux0=0.0, uy0=0.0, phi_p_uniform=False):
        _check(lib().lbm_batch_init_equilibrium(self._h, int(d), p0, ux0, uy0, int(bool(phi_p_uniform))),
               "lbm_batch_init_equilibrium")

    def step(self, n=1):
        _check(lib().lbm_batch_step(self._h, int(n)), "lbm_batch_step")

    def step_each(self, n=1):
        _check(lib().lbm_batch_step_each(self._h, int(n)), "lbm_batch_step_each")

    def set_launch(self, threads_per_cta, ctas_per_sm):
        _check(lib().lbm_batch_set_launch(self._h, int(threads_per_cta), int(ctas_per_sm)), "lbm_batch_set_launch")

    def get_launch(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(lib().lbm_batch_get_launch(self._h, ctypes.byref(a), ctypes.byref(b)), "lbm_batch_get_launch")
        return a.value, b.value

    def set_items_per_cta(self, items_per_cta):
        """Work items per CTA of the one-CTA form (ctas_per_sm = 0): 1, 2, 4 or 8 (4 x that many
        cells per thread)."""
        _check(lib().lbm_batch_set_items_per_cta(self._h, int(items_per_cta)), "lbm_batch_set_items_per_cta")

    def get_items_per_cta(self):
        k = ctypes.c_int()
        _check(lib().lbm_batch_get_items_per_cta(self._h, ctypes.byref(k)), "lbm_batch_get_items_per_cta")
        return k.value

    def set_tiling(self, tiling):
        _check(lib().lbm_batch_set_tiling(self._h, int(tiling)), "lbm_batch_set_tiling")

    def get_tiling(self):
        t = ctypes.c_int()
        _check(lib().lbm_batch_get_tiling(self._h, ctypes.byref(t)), "lbm_batch_get_tiling")
        return t.value

    def tune(self, steps=20):
        a, b, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        _check(lib().lbm_batch_tune(self._h, int(steps), ctypes.byref(a), ctypes.byref(b), ctypes.byref(ms)), "lbm_batch_tune")
        return a.value, b.value, ms.value

    def tune_cached(self, path=None, steps=20):
        """Launch shape, work items per CTA and tiling from a JSON cache on disk (keyed by GPU, storage
        precision, lattice count and total cells rounded to a power of two); a miss runs ``tune`` and
        records the result."""
        import json

        import torch

        path = path or os.environ.get("LBM_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "lbm_gb300_tune.json")
        cells = sum(a * b for a, b in self.shapes)
        key = f"{torch.cuda.get_device_name()}|prec{int(self.cfgs[0].precision)}|n{len(self)}|cells2^{int(math.log2(max(cells, 1)))}"
        try:
            with open(path) as fh:
                cache = json.load(fh)
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            nt, k = cache[key]["threads_per_cta"], cache[key]["ctas_per_sm"]
            self.set_tiling(cache[key].get("tiling", TILING_FLAT))
            self.set_items_per_cta(cache[key].get("items_per_cta", 1))
            self.set_launch(nt, k)
            return nt, k, cache[key]["ms_per_step"], True
        nt, k, ms = self.tune(steps)
        cache[key] = {"threads_per_cta": nt, "ctas_per_sm": k, "tiling": self.get_tiling(), "items_per_cta": self.get_items_per_cta(),
                      "ms_per_step": ms}
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1)
        os.replace(tmp, path)
        return nt, k, ms, False

    def macros(self, d):
        import torch

        ny, nx = self.shapes[d]
        out = [torch.empty(ny, nx, dtype=torch.float32, device=self.device) for _ in range(3)]
        _check(lib().lbm_batch_macros(self._h, int(d), *(o.data_ptr() for o in out)), "lbm_batch_macros")
        return tuple(out)

    def get_populations(self, d):
        import torch

        ny, nx = self.shapes[d]
        f = torch.empty(8, ny, nx, dtype=torch.float32, device=self.device)
        _check(lib().lbm_batch_get_populations(self._h, int(d), f.data_ptr()), "lbm_batch_get_populations")
        return f

    def info(self):
        c, s, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_uint64()
        _check(lib().lbm_batch_info(self._h, ctypes.byref(c), ctypes.byref(s), ctypes.byref(b)), "lbm_batch_info")
        return {"cells": c.value, "steps": s.value, "bytes": b.value}

    def sync(self):
        _check(lib().lbm_batch_sync(self._h), "lbm_batch_sync")


def _autograd_function():
    import torch

    class PorousFlowLoss(torch.autograd.Function):
        """loss = L(u(T; log K, eps)) of T steps of the porous flow from the equilibrium initial
        state, with d loss / d(log K, eps) from the discrete adjoint (lbm_adjoint).

        apply(logK, eps, cfg, T, loss="flux", target=None, p0=1.0, phi_p_uniform=False):
        logK, eps: float32 CUDA tensors [ny, nx]; cfg: a ``Config`` (copied); target: (ux*, uy*)
        for the misfit loss.  The forward call already runs the adjoint and keeps the gradient.
        """

        @staticmethod
        def forward(ctx, logK, eps, cfg, T, loss="flux", target=None, p0=1.0, phi_p_uniform=False):
            lat = Lattice(Config.from_buffer_copy(cfg))
            try:
                lat.set_medium_log(eps.detach().contiguous(), logK.detach().contiguous())
                lat.init_equilibrium(p0, 0.0, 0.0, phi_p_uniform)
                L, gk, ge = lat.adjoint(T, loss, target)
            finally:
                lat.close()
            ctx.save_for_backward(gk, ge)
            return torch.tensor(L, dtype=torch.float64, device=logK.device)

        @staticmethod
        def backward(ctx, gout):
            gk, ge = ctx.saved_tensors
            return (gout * gk).to(torch.float32), (gout * ge).to(torch.float32), None, None, None, None, None, None

    return PorousFlowLoss


def __getattr__(name):
    if name == "PorousFlowLoss":
        cls = _autograd_function()
        globals()[name] = cls
        return cls
    raise AttributeError(name)
