"""Checkpoint form of the particle store (LPIC_DIAG_PARTICLES_NATIVE) through the C ABI.

The particle dump of the canonical kind gives lab x = (cell + offset) dx in FP64, which does
not always give back the stored offset; the native kind copies the stored bits.  Bars: a
restored context holds the same bytes as the one it was dumped from (native dump, canonical
particles and ids, fields), whether the buffer is pageable (staged), page-locked (read in
place) or page-locked at an address that is not 8-byte aligned (staged: the in-place path
reads 8-byte values); and the two contexts then step alike, to the rounding of the FP64
atomic order (1e-12 relative after 5 steps).
"""
import dataclasses

import numpy as np
import pytest

from helpers import gpu_from, rel_err
from workloads import C1

pytestmark = pytest.mark.gpu

W = dataclasses.replace(C1, name="checkpoint", nx=64, nr=32, a0=1.0, w0=10.0, L=6.0, n0=0.01)
FIELDS = ("ex", "er", "bt", "a", "am")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1912_04674_gb300 import build
    build.build()


def _restore(dst, c, fields, blob):
    dst.upload_counters(c["step"], c["shift"])
    for k, v in fields.items():
        dst.upload_field(k, v)
    dst.upload_particles_native(blob)


def _pinned_copy(blob, offset):
    """A page-locked byte buffer holding blob at `offset` bytes from an aligned base."""
    import torch

    t = torch.empty(blob.nbytes + 16, dtype=torch.uint8).pin_memory()
    view = t.numpy()[offset: offset + blob.nbytes]
    view[:] = blob
    return t, view


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_native_particle_dump_restores_bit_for_bit(precision):
    from paper_1912_04674_gb300 import lpic as L

    src = gpu_from(W, precision=precision)
    src.step(9)
    c = src.counters()
    blob = src.particles_native()
    fields = {k: src.field(k) for k in FIELDS}
    canon = src.particles()
    es = src.native_itemsize
    assert blob.nbytes == (12 + 7 * es) * c["alive"]
    parts = L.split_native(blob, es)
    np.testing.assert_array_equal(parts["id"], canon["id"])
    # the canonical x is (cell + offset) dx, evaluated in FP64
    np.testing.assert_array_equal((parts["cell"].astype(np.float64) + parts["ox"].astype(np.float64)) * W.dx,
                                  canon["x"])
    assert np.all((parts["ox"] >= 0) & (parts["ox"] < 1))

    keep, restored = [], []
    for offset in (0, 8, 4):       # pageable; page-locked aligned; page-locked misaligned
        dst = gpu_from(W, precision=precision)
        if offset == 0:
            _restore(dst, c, fields, blob)
        else:
            buf, view = _pinned_copy(blob, offset)
            keep.append(buf)
            _restore(dst, c, fields, view)
        np.testing.assert_array_equal(dst.particles_native(), blob)
        got = dst.particles()
        for k in canon:
            np.testing.assert_array_equal(got[k], canon[k])
        for k in FIELDS:
            np.testing.assert_array_equal(dst.field(k), fields[k])
        d = dst.counters()
        assert (d["step"], d["shift"], d["alive"]) == (c["step"], c["shift"], c["alive"])
        restored.append(dst)
    src.step(5)
    for offset, dst in zip((0, 8, 4), restored):
        dst.step(5)
        for k in ("ex", "er", "bt", "a", "chi", "jx", "jr"):
            assert rel_err(dst.field(k), src.field(k)) <= 1e-12, (offset, k)


def test_native_upload_rejects_a_wrong_size():
    from paper_1912_04674_gb300 import lpic as L

    sim = gpu_from(W, precision="fp32")
    blob = sim.particles_native()
    with pytest.raises(L.LpicError) as e:
        sim.upload_particles_native(blob[:-3])
    assert e.value.status == 1
