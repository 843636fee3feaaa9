"""Host-side checks of the C ABI (no GPU needed): the library loads and exports every entry
point declared in include/lpic.h, the structs agree with the C layout, parameter checks accept
every configuration the paper ran (Sec. 4) and reject unstable ones, memory planning is sane."""
import ctypes as C
import json
import os
import re
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lpic.h")


@pytest.fixture(scope="module")
def L():
    from paper_1912_04674_gb300 import build as b
    b.build()
    from paper_1912_04674_gb300 import lpic
    return lpic


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lpic_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(L):
    lib = L.lib()
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(L._SIGS), "binding and header disagree"


def test_struct_layout_matches_c(L, tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include "lpic.h"\n#include <stdio.h>\n#include <stddef.h>\nint main(void){'
                   'printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(lpic_grid_params), sizeof(lpic_laser_params),'
                   'sizeof(lpic_plasma_params), offsetof(lpic_grid_params, particle_capacity),'
                   'offsetof(lpic_plasma_params, seed), offsetof(lpic_grid_params, slab_front_interior));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert got == [C.sizeof(L.lpic_grid_params), C.sizeof(L.lpic_laser_params),
                   C.sizeof(L.lpic_plasma_params), L.lpic_grid_params.particle_capacity.offset,
                   L.lpic_plasma_params.seed.offset, L.lpic_grid_params.slab_front_interior.offset]


def paper_cases():
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_parameters.json")))
    return [(k, v) for k, v in g.items() if isinstance(v, dict) and "dx" in v]


@pytest.mark.parametrize("name,case", paper_cases())
def test_paper_benchmark_parameters_are_stable(L, name, case):
    dx, dr = case["dx"], case["dr"]
    gs = L.grid_struct(L.Grid(512, 64, dx, dr, case["dt_over_dx"] * dx))
    L.lpic_check_params(gs)  # raises if rejected


def test_speedup_arithmetic_of_the_paper():
    s = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_parameters.json")))["speedup_estimate"]
    est = s["N_perp"] ** 2 * s["N_par"] * s["ppc_3d"] / (s["N_perp"] / 2 * s["N_par"] * s["ppc_cyl"])
    assert abs(est / s["printed"] - 1) < 0.01


def test_unstable_steps_are_rejected(L):
    cases = [L.Grid(64, 32, 0.69, 1.0, 0.60),    # Yee
             L.Grid(64, 32, 0.69, 1.0, 0.552),   # envelope (radial term, see oracle probe)
             L.Grid(64, 32, 0.5, 3.0, 0.5)]      # dt = dx
    for g in cases:
        with pytest.raises(L.LpicError) as e:
            L.lpic_check_params(L.grid_struct(g))
        assert e.value.status == 2


def test_invalid_arguments_are_rejected(L):
    for g in (L.Grid(1, 32, 0.7, 1.5, 0.5), L.Grid(64, 32, -0.7, 1.5, 0.5),
              L.Grid(64, 32, 0.7, float("nan"), 0.5),
              L.Grid(64, 32, 0.69, 1.5, 0.552, filter_passes=-1),
              L.Grid(64, 32, 0.69, 1.5, 0.552, filter_passes=17)):
        with pytest.raises(L.LpicError) as e:
            L.lpic_check_params(L.grid_struct(g))
        assert e.value.status == 1
    gs = L.grid_struct(L.Grid(64, 32, 0.69, 1.5, 0.552))
    bad = L.plasma_struct(L.Plasma(0.001, ppc=(0, 2, 4)))
    with pytest.raises(L.LpicError):
        L.lpic_check_params(gs, bad)
    assert L.lpic_required_bytes(L.grid_struct(L.Grid(1, 32, 0.7, 1.5, 0.5)), 0) == 0


def test_memory_plan_and_capacity(L):
    from workloads import C1, C2
    for w in (C1, C2):
        p = L.Plasma(w.n0, 0.0, w.ramp_len, w.ppc, w.seed)
        gs = L.grid_struct(L.Grid(w.nx, w.nr, w.dx, w.dr, w.dt, True, w.sort_every), p)
        assert gs.particle_capacity >= 1.1 * w.particles + (w.sort_every + 2) * w.nr * 16
        b64 = L.lpic_required_bytes(gs, L.LPIC_FP64)
        b32 = L.lpic_required_bytes(gs, L.LPIC_FP32_MIXED)
        # two particle buffers dominate: 68 B (FP64) / 40 B (FP32) per slot
        assert b64 > 2 * 68 * gs.particle_capacity and b32 > 2 * 40 * gs.particle_capacity
        assert b32 < b64 < 2 * 68 * gs.particle_capacity + 400e6


def test_diagnostic_kinds_match_the_header(L):
    """The binding's kind numbers are the header's lpic_diag_kind values (compiled by gcc)."""
    import tempfile
    names = {k: "LPIC_DIAG_" + k.upper() for k in L.DIAG}
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "k.c")
        with open(src, "w") as f:
            f.write('#include "lpic.h"\n#include <stdio.h>\nint main(void){\n')
            for c_name in names.values():
                f.write(f'printf("%d\\n", (int){c_name});\n')
            f.write("return 0;}\n")
        exe = os.path.join(d, "k")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        got = [int(v) for v in subprocess.check_output([exe]).split()]
    assert got == list(L.DIAG.values())


@pytest.mark.parametrize("itemsize", [4, 8])
def test_native_particle_layout_split(L, itemsize):
    """LPIC_DIAG_PARTICLES_NATIVE: ids, seven working-precision blocks, then int32 cells, each
    block aligned to its element size."""
    n = 5
    ft = np.float32 if itemsize == 4 else np.float64
    ids = np.arange(100, 100 + n, dtype=np.uint64)
    comps = {k: (np.arange(n) + 10 * q).astype(ft) for q, k in enumerate(L.NATIVE_COMPONENTS)}
    cells = np.arange(-2, n - 2, dtype=np.int32)
    blob = np.concatenate([ids.view(np.uint8)] + [comps[k].view(np.uint8) for k in L.NATIVE_COMPONENTS]
                          + [cells.view(np.uint8)])
    assert blob.nbytes == (12 + 7 * itemsize) * n
    p = L.split_native(blob, itemsize)
    np.testing.assert_array_equal(p["id"], ids)
    for k in L.NATIVE_COMPONENTS:
        np.testing.assert_array_equal(p[k], comps[k])
        assert p[k].dtype == ft
    np.testing.assert_array_equal(p["cell"], cells)
    with pytest.raises(ValueError):
        L.split_native(blob[:-1], itemsize)
