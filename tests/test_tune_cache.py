"""Autotuner cache: launch shapes stored in a JSON file keyed by the orders,
the precision and the level sizes.  The file logic runs on the CPU; the GPU
test checks that a second tuning call applies the stored shape (no search)
and that the shape leaves the results unchanged."""
import os

import numpy as np
import pytest

import paper_1610_05023_b300 as dgh
from paper_1610_05023_b300 import workloads as W


def _info(**kw):
    i = dict(order=4, habc_order=6, n_cells=663552, n_tris=27648, n_lines=576, n_corners=8)
    i.update(kw)
    return i


def test_key_separates_orders_precisions_and_sizes():
    keys = {dgh.tune_cache_key(_info(), 0), dgh.tune_cache_key(_info(order=3), 0),
            dgh.tune_cache_key(_info(habc_order=2), 0), dgh.tune_cache_key(_info(), dgh.PREC_SPLIT_BF16),
            dgh.tune_cache_key(_info(n_cells=384), 0), dgh.tune_cache_key(_info(n_tris=0), 0)}
    assert len(keys) == 6
    assert dgh.tune_cache_key(_info(), 0) == dgh.tune_cache_key(_info(), 0)


def test_store_and_load_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    assert dgh.tune_cache_load(path) == {}
    a = dict(tile2=21, tile1=1, cta3_per_sm=0, thr2=128, thr1=256, ms_before=4.2, ms_after=4.1)
    b = dict(a, tile2=10, thr2=64)
    dgh.tune_cache_store(path, "k1", a)
    dgh.tune_cache_store(path, "k2", b)
    dgh.tune_cache_store(path, "k1", dict(a, tile1=2))    # replaces
    data = dgh.tune_cache_load(path)
    assert data["k2"] == b and data["k1"]["tile1"] == 2 and len(data) == 2
    assert not os.path.exists(path + ".tmp")


@pytest.mark.gpu
def test_tune_cache_applies_the_stored_shape(tmp_path):
    path = str(tmp_path / "tune.json")
    VX, EToV = W.kuhn_mesh(3, 1.0, 0.02, seed=80)
    a = dgh.Solver(VX, EToV, 3, 2)
    a.init_gaussian([0.1, 0.0, 0.2], 0.3)
    first = a.tune(steps=2, cache=path)
    entry = dgh.tune_cache_load(path)[dgh.tune_cache_key(a.info, dgh.PREC_FP32)]
    b = dgh.Solver(VX, EToV, 3, 2)
    b.init_gaussian([0.1, 0.0, 0.2], 0.3)
    b.set_launch(tile2=1, thr2=32, tile1=1, thr1=32)        # something else first
    assert b.tune(steps=2, cache=path) == first            # served from the cache
    assert all(b.launch[k] == entry[k] for k in dgh.TUNABLE)
    assert b.info["step_count"] == 0
    a.step(10)
    b.step(10)
    for lv in (3, 2, 1):
        assert np.array_equal(a.get_state(lv), b.get_state(lv))
