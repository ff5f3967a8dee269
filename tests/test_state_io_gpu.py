"""State transfers with FP32 host arrays (dgh_set_state_f32 / dgh_get_state_f32)
against the FP64 transfers (dgh_set_state / dgh_get_state), through the C ABI.

The device state is FP32, so both directions are exact relations, checked bit
for bit: an FP32 read equals the FP64 read rounded to float (the FP64 read
widens a float, which is exact), an FP32 write leaves on the device the
floats that an FP64 write of the same values rounds to (round to nearest on
both sides), and a run continued from either write is identical.
"""
import numpy as np
import pytest

import paper_1610_05023_b300 as dgh
from paper_1610_05023_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _solver(prec=dgh.PREC_FP32):
    VX, EToV = W.kuhn_mesh(3, 1.0, 0.02, seed=11)
    g = dgh.Solver(VX, EToV, 3, 2, cfl=0.5, precision=prec)
    g.init_gaussian([0.1, -0.2, 0.15], 0.35)
    g.step(4)
    return g


@pytest.mark.parametrize("prec", [dgh.PREC_FP32, dgh.PREC_SPLIT_TF32])
def test_fp32_reads_equal_fp64_reads(prec):
    g = _solver(prec)
    for lv in (3, 2, 1):
        a64 = g.get_state(lv)
        a32 = g.get_state(lv, dtype=np.float32)
        assert a32.dtype == np.float32 and a32.shape == a64.shape
        assert np.array_equal(a32, a64.astype(np.float32)), lv
        assert np.array_equal(a32.astype(np.float64), a64), lv   # the FP64 read is an exact widening
        assert np.abs(a64).max() > 0, lv
    g.close()


def test_fp32_writes_match_fp64_writes_and_runs_continue_identically():
    rng = np.random.default_rng(5)
    g1, g2 = _solver(), _solver()
    x = {lv: rng.standard_normal(g1.shape(lv)) * 1e-2 for lv in (3, 2, 1)}
    for lv in (3, 2, 1):
        g1.set_state(lv, x[lv])                       # FP64, rounded on the device
        g2.set_state(lv, x[lv].astype(np.float32))    # FP32, unchanged
    for lv in (3, 2, 1):
        b1 = g1.get_state(lv, dtype=np.float32)
        b2 = g2.get_state(lv, dtype=np.float32)
        assert np.array_equal(b2, x[lv].astype(np.float32)), lv
        assert np.array_equal(b1, b2), lv
    g1.step(3)
    g2.step(3)
    for lv in (3, 2, 1):
        assert np.array_equal(g1.get_state(lv), g2.get_state(lv)), lv
    assert g1.energy() == g2.energy()
    g1.close()
    g2.close()


def test_fp32_transfers_into_pinned_buffers_and_size_errors():
    import torch

    g = _solver()
    for lv in (3, 2, 1):
        shp = g.shape(lv)
        pin = torch.empty(shp, dtype=torch.float32, pin_memory=True).numpy()
        g.get_state(lv, out=pin)
        assert np.array_equal(pin, g.get_state(lv, dtype=np.float32)), lv
        g.set_state(lv, pin)
        assert np.array_equal(g.get_state(lv, dtype=np.float32), pin), lv
    lib = dgh.load_library()
    bad = np.zeros(7, np.float32)
    ptr = bad.ctypes.data_as(dgh.ctypes.POINTER(dgh.ctypes.c_float))
    assert lib.dgh_set_state_f32(g._h, 3, ptr, bad.size) == dgh.DGH_EINVAL
    assert lib.dgh_get_state_f32(g._h, 3, ptr, bad.size) == dgh.DGH_EINVAL
    assert lib.dgh_set_state_f32(g._h, 3, None, 5) == dgh.DGH_EINVAL
    g.close()
