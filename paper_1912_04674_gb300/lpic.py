"""Python binding of the C ABI in ``include/lpic.h`` (argument marshalling only).

Every function of the header is exposed under the same name; each returns normally on
``LPIC_OK`` and raises :class:`LpicError` otherwise.  Every computation runs in the CUDA
library ``_build/liblpic.so``; there is no Python or CPU fallback, and loading fails
loudly when the library has not been built.

:class:`Simulation` is a convenience owner of one context: it allocates the device buffer
with PyTorch (device memory and streams are the only things PyTorch does here) and turns
diagnostics into numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblpic.so")

LPIC_OK = 0
STATUS = {0: "LPIC_OK", 1: "LPIC_EINVAL", 2: "LPIC_ECFL", 3: "LPIC_ENOMEM_BUDGET", 4: "LPIC_EBUFSIZE",
          5: "LPIC_ECUDA", 6: "LPIC_ETIMEOUT", 7: "LPIC_ENONFINITE", 8: "LPIC_ESTATE"}
LPIC_FP64, LPIC_FP32_MIXED = 0, 1
PRECISION = {"fp64": LPIC_FP64, "fp32": LPIC_FP32_MIXED, "fp32_mixed": LPIC_FP32_MIXED}
DIAG = {"ex_axis": 0, "a_abs_max": 1, "waist": 2, "cont_residual": 3, "accel_energy": 4,
        "counters": 5, "beam": 6, "ex": 10, "er": 11, "bt": 12, "a": 13, "am": 14, "chi": 15, "jx": 16,
        "jr": 17, "dq": 18, "particles": 20, "particle_ids": 21, "particles_native": 22}
PART_COMPONENTS = ("x", "y", "z", "px", "py", "pz", "w")
NATIVE_COMPONENTS = ("ox", "y", "z", "px", "py", "pz", "w")   # in-cell x offset, then as above


def split_native(raw: np.ndarray, itemsize: int) -> dict:
    """Views of the blocks of a LPIC_DIAG_PARTICLES_NATIVE buffer: id (uint64), the seven
    working-precision components (float32 for itemsize 4, float64 for 8) and the lab cell
    index (int32)."""
    b = np.ascontiguousarray(raw).view(np.uint8)
    per = 12 + 7 * itemsize
    if b.size % per:
        raise ValueError(f"native particle buffer: {b.size} bytes is not a multiple of {per}")
    n = b.size // per
    ft = np.float32 if itemsize == 4 else np.float64
    out = {"id": b[: 8 * n].view(np.uint64)}
    at = 8 * n
    for k in NATIVE_COMPONENTS:
        out[k] = b[at: at + itemsize * n].view(ft)
        at += itemsize * n
    out["cell"] = b[at: at + 4 * n].view(np.int32)
    return out


class LpicError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class lpic_grid_params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("nr", C.c_int32), ("dx", C.c_double), ("dr", C.c_double),
                ("dt", C.c_double), ("moving_window", C.c_int32), ("sort_every", C.c_int32),
                ("particle_capacity", C.c_int64), ("track_continuity", C.c_int32),
                ("accel_px_min", C.c_double), ("filter_passes", C.c_int32), ("slab_x0", C.c_int32),
                ("slab_front_interior", C.c_int32)]


class lpic_laser_params(C.Structure):
    _fields_ = [("a0", C.c_double), ("w0", C.c_double), ("L", C.c_double),
                ("x_center", C.c_double), ("x_focus", C.c_double)]


class lpic_plasma_params(C.Structure):
    _fields_ = [("n0", C.c_double), ("x_start", C.c_double), ("ramp_len", C.c_double),
                ("ppc_x", C.c_int32), ("ppc_r", C.c_int32), ("ppc_theta", C.c_int32),
                ("seed", C.c_uint64)]


_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes), in header order
_SIGS = {
    "lpic_check_params": (C.c_int, [C.POINTER(lpic_grid_params), C.POINTER(lpic_plasma_params), C.c_char_p, C.c_size_t]),
    "lpic_particle_capacity": (C.c_int64, [C.POINTER(lpic_grid_params), C.POINTER(lpic_plasma_params)]),
    "lpic_required_bytes": (C.c_size_t, [C.POINTER(lpic_grid_params), C.c_int]),
    "lpic_init_grid": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(lpic_grid_params), C.c_int, C.c_void_p, C.c_size_t, C.c_void_p]),
    "lpic_init_envelope": (C.c_int, [C.c_void_p, C.POINTER(lpic_laser_params)]),
    "lpic_load_plasma": (C.c_int, [C.c_void_p, C.POINTER(lpic_plasma_params)]),
    "lpic_step": (C.c_int, [C.c_void_p, C.c_int]),
    "lpic_diagnose": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "lpic_diagnose_async": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t]),
    "lpic_upload": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t]),
    "lpic_set_kernel_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "lpic_kernel_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_int)]),
    "lpic_kernel_name": (C.c_char_p, [C.c_int]),
    "lpic_envelope_stats_noalloc": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_double, C.c_void_p, C.c_void_p]),
    "lpic_slab_exchange": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "lpic_probe_fp64_fma": (C.c_int, [C.c_int32, C.c_void_p, C.POINTER(C.c_int64), C.c_void_p]),
    "lpic_bunch_scratch_bytes": (C.c_size_t, [C.c_void_p]),
    "lpic_inject_bunch": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int64, C.c_double, C.c_void_p, C.c_size_t]),
    "lpic_destroy": (C.c_int, [C.c_void_p]),
    "lpic_last_error": (C.c_char_p, [C.c_void_p]),
    "lpic_batch_required_bytes": (C.c_size_t, [C.POINTER(C.c_void_p), C.c_int]),
    "lpic_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int, C.c_void_p, C.c_size_t, C.c_void_p]),
    "lpic_batch_step": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "lpic_batch_set_tuning": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "lpic_batch_launches": (C.c_int64, [C.c_void_p]),
    "lpic_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "lpic_batch_destroy": (C.c_int, [C.c_void_p]),
}


def lib():
    """Load the CUDA library (raises if it has not been built: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"lpic CUDA library not built: {LIB_PATH} is missing; run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype, f.argtypes = res, args
            _lib = L
    return _lib


def _check(status: int, ctx=None):
    if status != LPIC_OK:
        msg = lib().lpic_last_error(ctx)
        raise LpicError(status, msg.decode() if msg else "")


# ---- one wrapper per C entry point ----------------------------------------------------------
def lpic_check_params(grid: lpic_grid_params, plasma: lpic_plasma_params | None = None) -> str:
    buf = C.create_string_buffer(512)
    st = lib().lpic_check_params(C.byref(grid), C.byref(plasma) if plasma else None, buf, 512)
    if st != LPIC_OK:
        raise LpicError(st, buf.value.decode())
    return ""


def lpic_particle_capacity(grid, plasma) -> int:
    return int(lib().lpic_particle_capacity(C.byref(grid), C.byref(plasma) if plasma else None))


def lpic_required_bytes(grid, precision: int) -> int:
    return int(lib().lpic_required_bytes(C.byref(grid), int(precision)))


def lpic_init_grid(grid, precision, device_ptr: int, nbytes: int, stream_ptr: int):
    out = C.c_void_p()
    _check(lib().lpic_init_grid(C.byref(out), C.byref(grid), int(precision), C.c_void_p(device_ptr),
                                nbytes, C.c_void_p(stream_ptr)))
    return out


def lpic_init_envelope(ctx, laser):
    _check(lib().lpic_init_envelope(ctx, C.byref(laser)), ctx)


def lpic_load_plasma(ctx, plasma):
    _check(lib().lpic_load_plasma(ctx, C.byref(plasma)), ctx)


def lpic_step(ctx, nsteps: int):
    _check(lib().lpic_step(ctx, int(nsteps)), ctx)


def lpic_diagnose(ctx, kind: int, host_ptr, cap: int) -> int:
    written = C.c_size_t(0)
    _check(lib().lpic_diagnose(ctx, int(kind), host_ptr, cap, C.byref(written)), ctx)
    return int(written.value)


def lpic_diagnose_async(ctx, kind: int, host_ptr, cap: int):
    _check(lib().lpic_diagnose_async(ctx, int(kind), host_ptr, cap), ctx)


def lpic_diagnose_size(ctx, kind: int) -> int:
    """Bytes a diagnostic needs (the library reports it with LPIC_EBUFSIZE for cap 0)."""
    written = C.c_size_t(0)
    st = lib().lpic_diagnose(ctx, int(kind), None, 0, C.byref(written))
    if st not in (LPIC_OK, 4):
        _check(st, ctx)
    return int(written.value)


def lpic_upload(ctx, kind: int, host_ptr, nbytes: int):
    _check(lib().lpic_upload(ctx, int(kind), host_ptr, nbytes), ctx)


def lpic_set_kernel_timing(ctx, enable: bool):
    _check(lib().lpic_set_kernel_timing(ctx, int(bool(enable))), ctx)


def lpic_kernel_stats(ctx) -> dict:
    """{family: (launches, device ms since the last call)}; synchronises the stream."""
    n = C.c_int(0)
    la = (C.c_int64 * 32)()
    ms = (C.c_double * 32)()
    _check(lib().lpic_kernel_stats(ctx, la, ms, 32, C.byref(n)), ctx)
    return {lpic_kernel_name(k): (int(la[k]), float(ms[k])) for k in range(n.value)}


def lpic_kernel_name(k: int) -> str | None:
    v = lib().lpic_kernel_name(int(k))
    return v.decode() if v else None


def lpic_envelope_stats_noalloc(a_dev_ptr: int, nx: int, nr: int, dr: float, out_dev_ptr: int,
                                stream_ptr: int):
    """Peak |A| and waist from a caller-owned device envelope, without any allocation."""
    st = lib().lpic_envelope_stats_noalloc(C.c_void_p(a_dev_ptr), int(nx), int(nr), float(dr),
                                           C.c_void_p(out_dev_ptr), C.c_void_p(stream_ptr))
    if st != LPIC_OK:
        raise LpicError(st, "lpic_envelope_stats_noalloc failed")


def lpic_slab_exchange(left, right, halo: int):
    _check(lib().lpic_slab_exchange(left, right, int(halo)), left)


def lpic_probe_fp64_fma(iters: int, out_dev_ptr: int, stream_ptr: int) -> int:
    """Enqueue the FP64 FMA probe launch; returns its FP64 operation count."""
    flops = C.c_int64(0)
    st = lib().lpic_probe_fp64_fma(int(iters), C.c_void_p(out_dev_ptr), C.byref(flops), C.c_void_p(stream_ptr))
    if st != LPIC_OK:
        raise LpicError(st, "lpic_probe_fp64_fma failed")
    return int(flops.value)


def lpic_bunch_scratch_bytes(ctx) -> int:
    return int(lib().lpic_bunch_scratch_bytes(ctx))


def lpic_inject_bunch(ctx, parts7n: np.ndarray, gamma: float, scratch_ptr: int, scratch_bytes: int):
    a = np.ascontiguousarray(parts7n, dtype=np.float64)
    n = a.size // 7
    _check(lib().lpic_inject_bunch(ctx, a.ctypes.data_as(C.POINTER(C.c_double)), n, float(gamma),
                                   C.c_void_p(scratch_ptr), int(scratch_bytes)), ctx)


def lpic_destroy(ctx):
    _check(lib().lpic_destroy(ctx))


def lpic_last_error(ctx=None) -> str:
    m = lib().lpic_last_error(ctx)
    return m.decode() if m else ""


def _ctx_array(ctxs):
    return (C.c_void_p * len(ctxs))(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])


def lpic_batch_required_bytes(ctxs) -> int:
    return int(lib().lpic_batch_required_bytes(_ctx_array(ctxs), len(ctxs)))


def lpic_batch_create(ctxs, device_ptr: int, nbytes: int, stream_ptr: int):
    out = C.c_void_p()
    _check(lib().lpic_batch_create(C.byref(out), _ctx_array(ctxs), len(ctxs), C.c_void_p(device_ptr),
                                   nbytes, C.c_void_p(stream_ptr)))
    return out


def lpic_batch_step(batch, steps):
    arr = (C.c_int * len(steps))(*[int(s) for s in steps])
    st = lib().lpic_batch_step(batch, arr)
    if st != LPIC_OK:
        raise LpicError(st, lpic_batch_last_error(batch))


def lpic_batch_set_tuning(batch, particles_per_item: int, packs: int = 0):
    st = lib().lpic_batch_set_tuning(batch, int(particles_per_item), int(packs))
    if st != LPIC_OK:
        raise LpicError(st, lpic_batch_last_error(batch))


def lpic_batch_launches(batch) -> int:
    return int(lib().lpic_batch_launches(batch))


def lpic_batch_last_error(batch) -> str:
    m = lib().lpic_batch_last_error(batch)
    return m.decode() if m else ""


def lpic_batch_destroy(batch):
    _check(lib().lpic_batch_destroy(batch))


class Batch:
    """Owner of one lpic_batch over Simulation objects, with its device buffer from PyTorch."""

    def __init__(self, sims, stream=None):
        import torch

        self.sims = list(sims)
        ctxs = [s.ctx for s in self.sims]
        self.nbytes = lpic_batch_required_bytes(ctxs)
        if self.nbytes == 0:
            raise LpicError(1, "batch: contexts must be valid and share one precision")
        dev = self.sims[0].device
        self.stream = stream if stream is not None else torch.cuda.Stream(dev)
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=dev)
        ptr = (self.buf.data_ptr() + 255) // 256 * 256
        with torch.cuda.device(dev):
            self.b = lpic_batch_create(ctxs, ptr, self.nbytes, self.stream.cuda_stream)

    def step(self, steps):
        lpic_batch_step(self.b, steps)

    def set_tuning(self, particles_per_item: int, packs: int = 0):
        """Work-item size of the fused particle passes and pack count (0: as few packs as the
        launch parameter space allows; -1: no fused launches, each simulation's own step
        graph in turn), effective at the next step."""
        lpic_batch_set_tuning(self.b, particles_per_item, packs)

    def launches(self) -> int:
        return lpic_batch_launches(self.b)

    def close(self):
        if getattr(self, "b", None) is not None:
            lpic_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- convenience owner ------------------------------------------------------------------------
@dataclass
class Grid:
    nx: int
    nr: int
    dx: float
    dr: float
    dt: float
    moving_window: bool = True
    sort_every: int = 20
    track_continuity: bool = False
    accel_px_min: float = 0.0
    filter_passes: int = 0
    slab_x0: int = 0                  # x-slab: global window column of column 0
    slab_front_interior: bool = False  # x-slab whose front column is inside the window


@dataclass
class Laser:
    a0: float
    w0: float
    L: float
    x_center: float
    x_focus: float


@dataclass
class Plasma:
    n0: float
    x_start: float = 0.0
    ramp_len: float = 0.0
    ppc: tuple = (2, 2, 4)
    seed: int = 0


def grid_struct(g: Grid, plasma: Plasma | None = None, capacity: int | None = None) -> lpic_grid_params:
    s = lpic_grid_params(g.nx, g.nr, g.dx, g.dr, g.dt, int(g.moving_window), int(g.sort_every), 0,
                         int(g.track_continuity), float(g.accel_px_min), int(g.filter_passes),
                         int(g.slab_x0), int(bool(g.slab_front_interior)))
    if capacity is not None:
        s.particle_capacity = int(capacity)
    elif plasma is not None:
        s.particle_capacity = lpic_particle_capacity(s, plasma_struct(plasma))
    return s


def laser_struct(l: Laser) -> lpic_laser_params:
    return lpic_laser_params(l.a0, l.w0, l.L, l.x_center, l.x_focus)


def plasma_struct(p: Plasma) -> lpic_plasma_params:
    return lpic_plasma_params(p.n0, p.x_start, p.ramp_len, int(p.ppc[0]), int(p.ppc[1]),
                              int(p.ppc[2]), int(p.seed))


class Simulation:
    """One simulation context with a PyTorch-allocated device buffer."""

    def __init__(self, grid: Grid, laser: Laser | None = None, plasma: Plasma | None = None,
                 precision: str = "fp64", device: int = 0, stream=None, capacity: int | None = None):
        import torch

        self.grid = grid
        self.precision = PRECISION[precision]
        self.gs = grid_struct(grid, plasma, capacity)
        lpic_check_params(self.gs, plasma_struct(plasma) if plasma else None)
        self.nbytes = lpic_required_bytes(self.gs, self.precision)
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.buf.data_ptr()
        self.ptr = (base + 255) // 256 * 256
        with torch.cuda.device(self.device):
            self.ctx = lpic_init_grid(self.gs, self.precision, self.ptr, self.nbytes,
                                      self.stream.cuda_stream)
        if laser is not None:
            lpic_init_envelope(self.ctx, laser_struct(laser))
        if plasma is not None:
            lpic_load_plasma(self.ctx, plasma_struct(plasma))

    def close(self):
        if getattr(self, "ctx", None) is not None:
            lpic_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        lpic_step(self.ctx, n)

    def set_timing(self, enable: bool = True):
        lpic_set_kernel_timing(self.ctx, enable)

    def kernel_stats(self) -> dict:
        return lpic_kernel_stats(self.ctx)

    # -- diagnostics ---------------------------------------------------------------------
    def _diag(self, kind: str, dtype, count: int | None = None) -> np.ndarray:
        k = DIAG[kind]
        n = lpic_diagnose_size(self.ctx, k) if count is None else count * np.dtype(dtype).itemsize
        out = np.empty(max(n, 1) // np.dtype(dtype).itemsize, dtype=dtype)
        w = lpic_diagnose(self.ctx, k, out.ctypes.data_as(C.c_void_p), out.nbytes)
        return out[: w // np.dtype(dtype).itemsize]

    def ex_axis(self) -> np.ndarray:
        return self._diag("ex_axis", np.float64, self.grid.nx)

    def ex_axis_async(self, out: np.ndarray):
        """Enqueue the on-axis wake read into `out` (Nx float64, page-locked, e.g. from a
        pinned torch tensor) on this simulation's stream; `out` holds it once the stream has
        passed this point (record an event on self.stream after the call)."""
        if out.dtype != np.float64 or out.size < self.grid.nx or not out.flags.c_contiguous:
            raise LpicError(1, "ex_axis_async: out must be a contiguous float64 array of Nx values")
        lpic_diagnose_async(self.ctx, DIAG["ex_axis"], out.ctypes.data_as(C.c_void_p), out.nbytes)

    def a_abs_max(self) -> float:
        return float(self._diag("a_abs_max", np.float64, 1)[0])

    def waist(self) -> float:
        return float(self._diag("waist", np.float64, 1)[0])

    def cont_residual(self) -> float:
        return float(self._diag("cont_residual", np.float64, 1)[0])

    def accel_energy(self) -> np.ndarray:
        return self._diag("accel_energy", np.float64, 4)

    BEAM_FIELDS = ("n_accel", "n_beam", "charge", "e_peak", "fwhm", "de_over_e", "eps_y", "eps_z",
                   "eps_mean", "e_mean", "e_max", "nbins")

    def beam_parameters(self) -> dict:
        """Injected-beam parameters of Table BeamParams (see LPIC_DIAG_BEAM)."""
        v = self._diag("beam", np.float64, 12)
        return {k: float(x) for k, x in zip(self.BEAM_FIELDS, v)}

    def counters(self) -> dict:
        v = self._diag("counters", np.int64, 4)
        return {"step": int(v[0]), "shift": int(v[1]), "slots": int(v[2]), "alive": int(v[3])}

    def field(self, name: str) -> np.ndarray:
        nx, nr = self.grid.nx, self.grid.nr
        shape = {"ex": (nx, nr + 1), "jx": (nx, nr + 1), "er": (nx + 1, nr), "jr": (nx + 1, nr),
                 "bt": (nx, nr)}.get(name, (nx + 1, nr + 1))
        if name in ("a", "am"):
            raw = self._diag(name, np.float64, 2 * shape[0] * shape[1])
            return raw.view(np.complex128).reshape(shape)
        return self._diag(name, np.float64, shape[0] * shape[1]).reshape(shape)

    def particles(self) -> dict:
        raw = self._diag("particles", np.float64)
        n = raw.size // 7
        out = {k: raw[i * n:(i + 1) * n].copy() for i, k in enumerate(PART_COMPONENTS)}
        out["id"] = self._diag("particle_ids", np.uint64)
        return out

    @property
    def native_itemsize(self) -> int:
        """Bytes of one working-precision value (4 for FP32_MIXED, 8 for FP64)."""
        return 8 if self.precision == LPIC_FP64 else 4

    def particles_native(self) -> np.ndarray:
        """The particle store as the context holds it (LPIC_DIAG_PARTICLES_NATIVE), as bytes;
        split_native(raw, self.native_itemsize) gives its blocks.  Bit-exact checkpoint form."""
        return self._diag("particles_native", np.uint8)

    # -- uploads -----------------------------------------------------------------------------
    def upload_field(self, name: str, arr: np.ndarray):
        a = np.ascontiguousarray(arr)       # no copy of a contiguous array of the right type
        if name in ("a", "am"):
            a = np.ascontiguousarray(a.astype(np.complex128, copy=False)).view(np.float64)
        else:
            a = a.astype(np.float64, copy=False)
        lpic_upload(self.ctx, DIAG[name], a.ctypes.data_as(C.c_void_p), a.nbytes)

    def upload_particles(self, parts: dict):
        n = len(parts["x"])
        raw = np.concatenate([np.asarray(parts[k], dtype=np.float64) for k in PART_COMPONENTS]) if n else np.zeros(0)
        self.upload_particles_raw(raw, parts.get("id") if n else None)

    def upload_particles_raw(self, raw: np.ndarray, ids: np.ndarray | None = None):
        """Replace the particle set from one contiguous float64 array of 7n values in the
        dump layout (x, y, z, px, py, pz, w blocks), and optionally its n ids; no host copy
        is made, so a page-locked `raw` is copied to the device at full link speed."""
        if raw.dtype != np.float64 or not raw.flags.c_contiguous or raw.size % 7:
            raise LpicError(1, "upload_particles_raw: contiguous float64 array of 7n values expected")
        lpic_upload(self.ctx, DIAG["particles"], raw.ctypes.data_as(C.c_void_p), raw.nbytes)
        if ids is not None and raw.size:
            ids = np.ascontiguousarray(ids, dtype=np.uint64)
            lpic_upload(self.ctx, DIAG["particle_ids"], ids.ctypes.data_as(C.c_void_p), ids.nbytes)

    def upload_particles_native(self, raw: np.ndarray):
        """Replace the particle store by a LPIC_DIAG_PARTICLES_NATIVE buffer of the same
        precision (ids included), bit for bit; no host copy is made of a contiguous buffer."""
        b = np.ascontiguousarray(raw)
        lpic_upload(self.ctx, DIAG["particles_native"], b.ctypes.data_as(C.c_void_p), b.nbytes)

    def inject_bunch(self, parts: dict, gamma: float):
        """Append a relativistic electron bunch (x lab, y, z, px, py, pz, w) and add its
        self-consistent fields (lpic_inject_bunch); the solver scratch comes from PyTorch."""
        import torch

        n = len(parts["x"])
        raw = np.concatenate([np.asarray(parts[k], dtype=np.float64) for k in PART_COMPONENTS]) if n else np.zeros(0)
        nbytes = lpic_bunch_scratch_bytes(self.ctx)
        buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        ptr = (buf.data_ptr() + 255) // 256 * 256
        with torch.cuda.device(self.device):
            lpic_inject_bunch(self.ctx, raw, gamma, ptr, nbytes)
        del buf

    def upload_counters(self, step: int, shift: int):
        v = np.array([step, shift, 0, 0], dtype=np.int64)
        lpic_upload(self.ctx, DIAG["counters"], v.ctypes.data_as(C.c_void_p), v.nbytes)
