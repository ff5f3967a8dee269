"""Material changes and field initialisation through the C ABI
(dgh_set_material, dgh_set_material_layers, dgh_init_fields).  A material
change rebuilds the set-up and carries the state over: the run must continue
exactly as a solver created with that material from the same state would.
The layered material itself is checked against the oracle by
test_parity_gpu.py::test_parity_layered_material."""
import numpy as np
import pytest

import paper_1610_05023_b300 as dgh
from paper_1610_05023_b300 import workloads as W

Z_TOPS, C_L, RHO_L = [-1 / 3, 1 / 3], [1.0, 1.5, 2.0], [1.0, 1.2, 1.5]


def _mesh():
    return W.kuhn_mesh(3, 1.0, 0.02, seed=90)


def _levels(g):
    return [g.get_state(lv) for lv in (3, 2, 1)]


@pytest.mark.gpu
def test_set_material_continues_like_a_solver_created_with_it():
    VX, EToV = _mesh()
    c, rho = W.layered_material(VX, EToV, Z_TOPS, C_L, RHO_L, hex_centroid=False)
    xs = [0.1, -0.2, 0.05]
    a = dgh.Solver(VX, EToV, 3, 2)
    a.add_point_source(xs, 2.5, 0.3)
    a.init_gaussian([0.2, 0.1, -0.1], 0.3)
    a.step(6)
    snap, t = _levels(a), a.info["time"]
    a.set_material(c, rho)
    assert a.info["step_count"] == 6 and a.info["time"] == t
    b = dgh.Solver(VX, EToV, 3, 2, c=c, rho=rho)
    assert a.info["dt"] == b.info["dt"]           # the time-step rule follows the new c
    b.add_point_source(xs, 2.5, 0.3)
    for lv, q in zip((3, 2, 1), snap):
        b.set_state(lv, q)
    b.set_time(t)
    a.step(12)
    b.step(12)
    for qa, qb in zip(_levels(a), _levels(b)):
        assert np.array_equal(qa, qb)
    assert a.info["step_count"] == 18


@pytest.mark.gpu
def test_set_material_layers_equals_the_per_cell_call():
    VX, EToV = _mesh()
    c, rho = W.layered_material(VX, EToV, Z_TOPS, C_L, RHO_L, hex_centroid=False)
    a, b = dgh.Solver(VX, EToV, 3, 2), dgh.Solver(VX, EToV, 3, 2)
    a.set_material_layers(Z_TOPS, C_L, RHO_L)
    b.set_material(c, rho)
    for g in (a, b):
        g.init_gaussian([0.0, 0.1, 0.3], 0.3)
        g.step(10)
    for qa, qb in zip(_levels(a), _levels(b)):
        assert np.array_equal(qa, qb)


@pytest.mark.gpu
def test_set_material_rejects_bad_values_and_keeps_the_context():
    VX, EToV = _mesh()
    g = dgh.Solver(VX, EToV, 3, 2)
    g.init_gaussian([0.0, 0.0, 0.0], 0.3)
    g.step(3)
    before = _levels(g)
    K = g.info["n_cells"]
    bad = np.ones(K)
    bad[7] = -1.0
    with pytest.raises(dgh.DghError):
        g.set_material(bad, np.ones(K))
    with pytest.raises(dgh.DghError):
        g.set_material_layers([0.5, 0.0], [1, 2, 3], [1, 1, 1])   # z_top not increasing
    for qa, qb in zip(_levels(g), before):
        assert np.array_equal(qa, qb)
    g.step(2)
    assert np.isfinite(g.energy())


@pytest.mark.gpu
def test_init_fields_sets_the_3d_state_and_zeroes_the_rest():
    VX, EToV = _mesh()
    g = dgh.Solver(VX, EToV, 3, 2)
    g.init_gaussian([0.2, 0.0, 0.1], 0.3)
    g.step(5)                                       # auxiliary fields and clock now nonzero
    q = W.random_state(91, g.get_state(3).shape)
    g.init_fields(q)
    assert np.array_equal(g.get_state(3), q.astype(np.float32).astype(np.float64))
    assert not g.get_state(2).any() and not g.get_state(1).any()
    assert g.info["time"] == 0.0 and g.info["step_count"] == 0
