"""Python handle on the FP64 CPU oracle (``lpic_oracle.c``).

Test infrastructure only: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only users.  The product library never
imports this module and this module never imports the product library.

The oracle keeps its own arrays (C ``malloc``); this wrapper exposes them as
numpy views that are re-created after every call, since particle arrays may be
reallocated.  Field layout is ``[i][j]``, radial index fastest (see the C
header comment for the staggering).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lpic_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liblpic_oracle.so")
_lock = threading.Lock()
_lib = None

FIELDS = {"ex": 0, "er": 1, "bt": 2, "btn": 3, "a": 4, "am": 5, "chi": 6, "jx": 7,
          "jr": 8, "dq": 9, "phi": 10, "dphix": 11, "dphir": 12, "phih": 13}
PARTS = {"x": 0, "y": 1, "z": 2, "px": 3, "py": 4, "pz": 5, "w": 6, "id": 7}


def build(force: bool = False) -> str:
    """Compile the oracle with plain IEEE FP64 semantics (no contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp, d, i, l, u64 = C.c_void_p, C.c_double, C.c_int, C.c_long, C.c_uint64
            L.osim_create.restype = vp
            L.osim_create.argtypes = [i, i, d, d, d, i]
            L.osim_free.argtypes = [vp]
            L.osim_init_envelope.argtypes = [vp, d, d, d, d, d]
            L.osim_load_plasma.argtypes = [vp, d, d, d, i, i, i, u64]
            L.osim_set_filter.argtypes = [vp, i]
            for f in ("osim_step", "osim_faraday", "osim_pass_a", "osim_envelope",
                      "osim_pass_b", "osim_ampere", "osim_window", "osim_filter"):
                getattr(L, f).argtypes = [vp]
            L.osim_run.argtypes = [vp, l]
            L.osim_field.restype = vp
            L.osim_field.argtypes = [vp, i]
            L.osim_particles.restype = vp
            L.osim_particles.argtypes = [vp, i]
            L.osim_np.restype = l
            L.osim_np.argtypes = [vp]
            L.osim_step_index.restype = l
            L.osim_step_index.argtypes = [vp]
            L.osim_shift.restype = l
            L.osim_shift.argtypes = [vp]
            L.osim_set_np.argtypes = [vp, l]
            L.osim_set_counters.argtypes = [vp, l, l]
            L.osim_get_x.argtypes = [vp, C.POINTER(d)]
            L.osim_set_x.argtypes = [vp, C.POINTER(d)]
            L.osim_splitmix64.restype = u64
            L.osim_splitmix64.argtypes = [u64, u64]
            _lib = L
    return _lib


class OSim:
    """One oracle simulation (normalised units, electrons q=-1, m=1)."""

    def __init__(self, nx, nr, dx, dr, dt, moving_window=True):
        self.L = lib()
        self.nx, self.nr, self.dx, self.dr, self.dt = int(nx), int(nr), float(dx), float(dr), float(dt)
        self.h = self.L.osim_create(self.nx, self.nr, self.dx, self.dr, self.dt, int(bool(moving_window)))

    def __del__(self):
        h, self.h = getattr(self, "h", None), None
        if h:
            self.L.osim_free(h)

    # -- set-up --------------------------------------------------------------
    def init_envelope(self, a0, w0, L, x_center, x_focus):
        self.L.osim_init_envelope(self.h, a0, w0, L, x_center, x_focus)

    def load_plasma(self, n0, x_start=0.0, ramp_len=0.0, ppc=(2, 2, 4), seed=0):
        self.L.osim_load_plasma(self.h, n0, x_start, ramp_len, int(ppc[0]), int(ppc[1]),
                                int(ppc[2]), int(seed))

    # -- stepping ------------------------------------------------------------
    def step(self, n=1):
        self.L.osim_run(self.h, int(n))

    def faraday(self): self.L.osim_faraday(self.h)
    def pass_a(self): self.L.osim_pass_a(self.h)
    def envelope(self): self.L.osim_envelope(self.h)
    def pass_b(self): self.L.osim_pass_b(self.h)
    def ampere(self): self.L.osim_ampere(self.h)
    def window(self): self.L.osim_window(self.h)
    def filter(self): self.L.osim_filter(self.h)

    def set_filter(self, passes: int):
        """Binomial current filter of `passes` passes along x after each deposit (0: off)."""
        self.L.osim_set_filter(self.h, int(passes))

    # -- state views -----------------------------------------------------------
    def _shape(self, name):
        nx, nr = self.nx, self.nr
        return {"ex": (nx, nr + 1), "jx": (nx, nr + 1), "er": (nx + 1, nr), "jr": (nx + 1, nr),
                "bt": (nx, nr), "btn": (nx, nr)}.get(name, (nx + 1, nr + 1))

    def field(self, name) -> np.ndarray:
        """Writable numpy view of an oracle grid array."""
        ptr = self.L.osim_field(self.h, FIELDS[name])
        shape = self._shape(name)
        n = shape[0] * shape[1]
        if name in ("a", "am"):
            buf = (C.c_double * (2 * n)).from_address(ptr)
            return np.frombuffer(buf, dtype=np.complex128).reshape(shape)
        buf = (C.c_double * n).from_address(ptr)
        return np.frombuffer(buf, dtype=np.float64).reshape(shape)

    @property
    def np(self) -> int:
        return int(self.L.osim_np(self.h))

    @property
    def step_index(self) -> int:
        return int(self.L.osim_step_index(self.h))

    @property
    def shift(self) -> int:
        return int(self.L.osim_shift(self.h))

    def set_counters(self, step, shift):
        self.L.osim_set_counters(self.h, int(step), int(shift))

    def part(self, name) -> np.ndarray:
        """View of a particle component; "x" (lab frame) is a computed copy."""
        n = self.np
        if name == "x":
            out = np.empty(n)
            if n:
                self.L.osim_get_x(self.h, out.ctypes.data_as(C.POINTER(C.c_double)))
            return out
        ptr = self.L.osim_particles(self.h, PARTS[name])
        if n == 0 or not ptr:
            return np.zeros(0, dtype=np.uint64 if name == "id" else np.float64)
        ct = C.c_uint64 if name == "id" else C.c_double
        buf = (ct * n).from_address(ptr)
        return np.frombuffer(buf, dtype=np.uint64 if name == "id" else np.float64)

    def set_particles(self, **arrs):
        """Replace the particle set; missing momenta default to 0, ids to 0..n-1."""
        n = len(arrs["x"])
        self.L.osim_set_np(self.h, n)
        for k in PARTS:
            v = arrs.get(k)
            if v is None:
                v = np.arange(n, dtype=np.uint64) if k == "id" else np.zeros(n)
            if not n:
                continue
            if k == "x":
                xv = np.ascontiguousarray(v, dtype=np.float64)
                self.L.osim_set_x(self.h, xv.ctypes.data_as(C.POINTER(C.c_double)))
            else:
                self.part(k)[:] = v

    def particles(self) -> dict:
        return {k: self.part(k).copy() for k in PARTS}

    def fields(self) -> dict:
        return {k: self.field(k).copy() for k in ("ex", "er", "bt", "a", "am", "chi", "jx", "jr")}


def splitmix64(seed: int, k: int) -> int:
    return int(lib().osim_splitmix64(seed, k))
