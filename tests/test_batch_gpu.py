"""Batching form on the GPU: independent problems of different N, P, mesh,
material, time step and source stepped together in one graph per step.

Each problem of the batch is compared with its own FP64 oracle run (same
seeded inputs, per-field relative L2 <= 2e-5), with the same problem run
alone through libdgh (the batch folds each problem's dt into its
coefficients, so the two differ by rounding order only: <= 5e-6, a few
times the rounding of the split-TF32 products, whose operands carry 2^-22
relative error), and the autotuner and the launch-shape setter are checked
to leave every result bit-identical.
"""
import numpy as np
import pytest

import paper_1610_05023_b300 as dgh
from oracle.mesh import BC_DIRICHLET, BC_HABC, CuboidMesh
from oracle.solver import Solver
from paper_1610_05023_b300 import workloads as W

pytestmark = pytest.mark.gpu

SINGLE_TOL = 5e-6   # batch against the same problem run alone: rounding order only
MIXED = (BC_DIRICHLET, BC_HABC, BC_HABC, BC_HABC, BC_HABC, BC_DIRICHLET)

# (n, N, P, bc, layered, init): init = ("gauss", x0, width) or ("ricker", xs, f_peak, t_s)
PROBLEMS = [
    (2, 3, 2, (BC_HABC,) * 6, False, ("gauss", (0.1, 0.0, -0.1), 0.3)),
    (2, 4, 1, (BC_HABC,) * 6, False, ("ricker", (0.11, -0.07, 0.05), 2.5, 0.2)),
    (3, 3, 2, (BC_HABC,) * 6, True, ("gauss", (0.0, 0.2, 0.3), 0.35)),
    (2, 2, 0, MIXED, False, ("gauss", (-0.2, 0.1, 0.0), 0.3)),
    (2, 3, 2, MIXED, False, ("ricker", (-0.1, 0.1, 0.2), 2.0, 0.25)),
]


def _problem(i, spec):
    n, N, P, bc, layered, init = spec
    VX, EToV = W.kuhn_mesh(n, 1.0, 0.03, seed=300 + i)
    if layered:
        c, rho = W.layered_material(VX, EToV, [-1 / 3, 1 / 3], [1.0, 1.5, 2.0], [1.0, 1.2, 1.5])
    else:
        c, rho = np.full(EToV.shape[0], 1.0 + 0.25 * i), np.ones(EToV.shape[0])
    m = CuboidMesh(VX, EToV, N, P, bc, rho, c)
    dt = m.dt_rule()
    o = Solver(m)
    g = dgh.Solver(VX, EToV, N, P, bc=bc, c=c, rho=rho, dt=dt)
    if init[0] == "gauss":
        Y = o.gaussian_state(list(init[1]), init[2])
        g.init_gaussian(list(init[1]), init[2])
    else:
        o.add_point_source(list(init[1]), init[2], init[3])
        g.add_point_source(list(init[1]), init[2], init[3])
        Y = o.zero_state()
    return o, g, Y, dt


def _levels(get, P):
    return {lv: get(lv) for lv in (3, 2, 1) if lv == 3 or P > 0}


def _rel(a, b, floor):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), floor)


def _compare(got, ref, tol):
    p3 = np.linalg.norm(ref[3][:, 0])
    for lv in got:
        for f in range(got[lv].shape[-2]):
            floor = 1e-3 * p3 if lv < 3 else 1e-30
            e = _rel(got[lv][..., f, :], ref[lv][..., f, :], floor)
            assert e <= tol, "level %d field %d: %.3g" % (lv, f, e)


@pytest.fixture(scope="module")
def batch_setup():
    made = [_problem(i, s) for i, s in enumerate(PROBLEMS)]
    b = dgh.Batch([g for _, g, _, _ in made])
    return made, b


def test_batch_grouping(batch_setup):
    made, b = batch_setup
    n, ng = b.counts
    assert n == len(PROBLEMS)
    assert ng == len({(s[1], s[2]) for s in PROBLEMS})
    for i, (o, g, _, dt) in enumerate(made):
        bi, gi = b.info(i), g.info
        for k in ("order", "habc_order", "n_cells", "n_tris", "n_lines", "n_corners", "ndof"):
            assert bi[k] == gi[k], k
        assert bi["dt"] == dt


def test_batch_matches_oracle_and_single_runs(batch_setup):
    made, b = batch_setup
    nst = 30
    b.step(nst)
    b.sync()
    for i, (o, g, Y, dt) in enumerate(made):
        P = PROBLEMS[i][2]
        Yr, _, t = o.run(Y, 0.0, dt, nst)
        ref = {3: Yr["q3"], 2: Yr["q2"], 1: Yr["q1"]}
        got = _levels(lambda lv: b.get_state(i, lv), P)
        _compare(got, ref, 2e-5)
        g.step(nst)
        alone = _levels(g.get_state, P)
        _compare(got, alone, SINGLE_TOL)
        info = b.info(i)
        assert info["step_count"] == nst
        assert abs(info["time"] - t) < 1e-12
        assert abs(b.energy(i) - g.energy()) <= 1e-6 * g.energy()


def test_batch_tune_changes_no_result():
    made = [_problem(i, s) for i, s in enumerate(PROBLEMS[:3])]
    a = dgh.Batch([g for _, g, _, _ in made])
    c = dgh.Batch([g for _, g, _, _ in made])
    before, after = c.tune(steps=2)
    assert after <= before
    assert all(c.info(i)["step_count"] == 0 for i in range(3))
    a.step(12)
    c.step(12)
    for i in range(3):
        for lv in (3, 2, 1):
            assert np.array_equal(a.get_state(i, lv), c.get_state(i, lv))


def test_solver_launch_shape_and_tune_change_no_result():
    VX, EToV = W.kuhn_mesh(3, 1.0, 0.02, seed=17)
    runs = []
    for mode in ("default", "shape", "tuned"):
        g = dgh.Solver(VX, EToV, 3, 3)
        g.init_gaussian([0.1, -0.1, 0.2], 0.3)
        if mode == "shape":
            g.set_launch(tile2=1, tile1=3, cta3_per_sm=1, thr2=32, thr1=64, sm3_div=4, split3=0)
            L = g.launch
            assert ((L["tile2"], L["tile1"], L["cta3_per_sm"], L["thr2"], L["thr1"], L["sm3_div"], L["split3"])
                    == (1, 3, 1, 32, 64, 4, 0))
        if mode == "tuned":
            g.tune(steps=2)
            assert g.info["step_count"] == 0
        g.step(15)
        runs.append({lv: g.get_state(lv) for lv in (3, 2, 1)})
        g.close()
    for r in runs[1:]:
        for lv in (3, 2, 1):
            assert np.array_equal(r[lv], runs[0][lv])


def test_set_launch_rejects_bad_shapes():
    VX, EToV = W.kuhn_mesh(2, 1.0, 0.02, seed=18)
    g = dgh.Solver(VX, EToV, 3, 2)
    before = g.launch
    with pytest.raises(dgh.DghError):
        g.set_launch(tile2=0)
    with pytest.raises(dgh.DghError):
        g.set_launch(tile2=100000)   # shared memory of the 2D tile does not fit
    with pytest.raises(dgh.DghError):
        g.set_launch(thr2=48)
    with pytest.raises(dgh.DghError):
        g.set_launch(sm3_div=0)
    with pytest.raises(dgh.DghError):
        g.set_launch(split3=2)
    with pytest.raises(dgh.DghError):
        g.set_launch(tile2=17, thr2=32)   # one thread per (triangle, set): 17 * 2 > 32
    assert g.launch == before


def test_batch_fullsize_48_problems():
    """The batching form's workload at full size: the 48 seeded problems the
    benchmark times (n ~ U{8..24}, N ~ U{3,4,5}, P ~ U{2,4,6}, Ricker point
    source, each at its own time step; 1.58 M tets), batched with the shapes
    the autotuner picks.  Each problem also starts from a Gaussian pulse of
    width 0.3 at its source point, so that every level carries data from the
    first step.  After 20 steps every problem equals the same problem run
    alone (<= 5e-6 per field), and two 8^3-hex problems, the one with the
    highest HABC order and the one with the highest degree, equal their FP64
    oracle runs (<= 2e-5)."""
    import torch
    probs = W.batch_problems(4000)
    seq = torch.cuda.Stream()
    solvers, meshes = [], []
    for p in probs:
        VX, EToV = W.kuhn_mesh(p["n"], 1.0, 0.02, seed=p["mesh_seed"])
        s = dgh.Solver(VX, EToV, p["N"], p["P"], stream=seq)
        s.add_point_source(p["xs"], p["f0"], p["t_s"])
        s.init_gaussian(p["xs"], 0.3)
        solvers.append(s)
        meshes.append((VX, EToV))
    b = dgh.Batch(solvers)
    b.tune(steps=3)
    nst = 20
    b.step(nst)
    b.sync()
    n_min = min(p["n"] for p in probs)
    smallest = [i for i, p in enumerate(probs) if p["n"] == n_min]
    checked = {max(smallest, key=lambda i: (probs[i]["P"], -probs[i]["N"])),
               max(smallest, key=lambda i: (probs[i]["N"], -probs[i]["P"]))}
    assert len(checked) == 2
    for i, (p, s) in enumerate(zip(probs, solvers)):
        s.step(nst)
        got = _levels(lambda lv: b.get_state(i, lv), p["P"])
        _compare(got, _levels(s.get_state, p["P"]), SINGLE_TOL)
        assert b.info(i)["step_count"] == nst
        if i in checked:
            VX, EToV = meshes[i]
            o = Solver(CuboidMesh(VX, EToV, p["N"], p["P"], [BC_HABC] * 6, 1.0, 1.0))
            o.add_point_source(p["xs"], p["f0"], p["t_s"])
            Yr, _, _ = o.run(o.gaussian_state(p["xs"], 0.3), 0.0, s.info["dt"], nst)
            _compare(got, {3: Yr["q3"], 2: Yr["q2"], 1: Yr["q1"]}, 2e-5)
    b.close()
    for s in solvers:
        s.close()
