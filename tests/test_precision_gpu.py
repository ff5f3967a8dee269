"""Precision form on the GPU: the 3D volume and lift products on the tcgen05
tensor cores (BF16, FP16, split BF16 with FP32 accumulation in tensor
memory) against the FP64 oracle.

Tolerances (per-field relative L2 after 10 steps from a random state, the
worst case for rounding since every node carries independent values): the
products round each operand to 8 (BF16), 11 (FP16) or ~16 (split BF16)
significant bits, so the field errors sit near 2^-9, 2^-12 and 2^-17 times
the number of accumulated steps; the bounds below are about three times the
values measured on a B300.  The acceptance rule of the precision form (its
error against the oracle at most 10% of the discretisation error against the
exact solution) is checked on a Gaussian pulse in free space.
"""
import math

import numpy as np
import pytest

import paper_1610_05023_b300 as dgh
from oracle.mesh import BC_DIRICHLET, BC_HABC, CuboidMesh
from oracle.solver import Solver
from paper_1610_05023_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {dgh.PREC_BF16_TC: 1e-2, dgh.PREC_FP16_TC: 1.5e-3, dgh.PREC_SPLIT_BF16: 2e-5}


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("prec", [dgh.PREC_BF16_TC, dgh.PREC_FP16_TC, dgh.PREC_SPLIT_BF16])
@pytest.mark.parametrize("N,P", [(1, 1), (2, 2), (3, 2), (4, 3), (5, 1), (6, 2)])
def test_tensor_core_parity_random_state(N, P, prec):
    VX, EToV = W.kuhn_mesh(2, 1.0, 0.04, seed=7 + N)
    m = CuboidMesh(VX, EToV, N, P, [BC_HABC] * 6, 1.0, 1.0)
    dt = m.dt_rule()
    o = Solver(m)
    Y = o.zero_state()
    for i, k in enumerate(("q3", "q2", "q1")):
        Y[k] = W.random_state(100 + i, Y[k].shape)
    g = dgh.Solver(VX, EToV, N, P, dt=dt, precision=prec)
    g.set_state(3, Y["q3"])
    g.set_state(2, Y["q2"])
    g.set_state(1, Y["q1"])
    Y, _, _ = o.run(Y, 0.0, dt, 10)
    g.step(10)
    q3 = g.get_state(3)
    for f in range(4):
        assert _rel(q3[:, f], Y["q3"][:, f]) <= TOL[prec], f
    assert _rel(g.get_state(2), Y["q2"]) <= TOL[prec]
    assert _rel(g.get_state(1), Y["q1"]) <= TOL[prec]


def test_tensor_core_multitile_mixed_boundaries_layers_source():
    """5^3 x 6 = 750 tets (24 blocks of 32 cells, interior and boundary
    launches with ragged 128-cell tiles), three layers, p = 0 on two faces,
    HABC P = 2 elsewhere, Ricker source, N = 5: split BF16 vs the oracle."""
    VX, EToV = W.kuhn_mesh(5, 1.0, 0.02, seed=31)
    c, rho = W.layered_material(VX, EToV, [-1 / 3, 1 / 3], [1.0, 1.5, 2.0], [1.0, 1.2, 1.5])
    bc = (BC_DIRICHLET, BC_HABC, BC_HABC, BC_HABC, BC_HABC, BC_DIRICHLET)
    m = CuboidMesh(VX, EToV, 5, 2, bc, rho, c)
    dt = m.dt_rule()
    o = Solver(m)
    xs = [0.13, -0.21, 0.08]
    o.add_point_source(xs, 3.0, 0.15)
    Y = o.gaussian_state([-0.2, 0.1, 0.3], 0.3)
    g = dgh.Solver(VX, EToV, 5, 2, bc=bc, c=c, rho=rho, dt=dt, precision=dgh.PREC_SPLIT_BF16)
    g.add_point_source(xs, 3.0, 0.15)
    g.init_gaussian([-0.2, 0.1, 0.3], 0.3)
    Y, _, _ = o.run(Y, 0.0, dt, 30)
    g.step(30)
    q3 = g.get_state(3)
    tol = 5e-5   # 30 steps: three times the 10-step bound's error growth, measured ~2e-5
    for f in range(4):
        assert _rel(q3[:, f], Y["q3"][:, f]) <= tol, f
    # auxiliary fields: relative to max(own norm, 1e-3 ||p_3D||) (they are ~0
    # where the wave has only just reached the boundary)
    floor = 1e-3 * np.linalg.norm(Y["q3"][:, 0])
    q2 = g.get_state(2)
    assert np.linalg.norm(q2 - Y["q2"]) / max(np.linalg.norm(Y["q2"]), floor) <= tol
    assert abs(g.energy() - o.energy(Y)) <= 1e-5 * o.energy(Y)


def _gaussian_exact(m, t, sigma):
    r = np.linalg.norm(m.x, axis=2)
    F = lambda s: s * np.exp(-s ** 2 / sigma ** 2)
    A = lambda s: -0.5 * sigma ** 2 * np.exp(-s ** 2 / sigma ** 2)
    rs = np.maximum(r, 1e-12)
    p = (F(rs - t) + F(rs + t)) / (2 * rs)
    ur = -((F(rs + t) - F(rs - t)) / (2 * rs) - (A(rs + t) - A(rs - t)) / (2 * rs ** 2))
    q = np.zeros((m.K, 4, m.ref3.Np))
    q[:, 0] = p
    for i in range(3):
        q[:, 1 + i] = ur * m.x[..., i] / rs
    return q


def test_precision_acceptance_rule():
    """N = 6, 4^3 x 6 tets, Gaussian pulse of width 0.25 in free space until
    t = 0.35: energy-norm error of each variant against the oracle, relative
    to the oracle's own error against the exact solution.  Split BF16 must
    stay below 10% of it; the variants must order by precision."""
    sigma, T = 0.25, 0.35
    VX, EToV = W.kuhn_mesh(4, 1.0, 0.02, seed=3)
    m = CuboidMesh(VX, EToV, 6, 0, [BC_HABC] * 6, 1.0, 1.0)
    o = Solver(m)
    Y0 = o.gaussian_state([0, 0, 0], sigma)
    E0 = o.energy(Y0)
    nst = int(math.ceil(T / m.dt_rule()))
    dt = T / nst
    Y, _, _ = o.run(Y0, 0.0, dt, nst)
    zero2, zero1 = np.zeros_like(Y["q2"]), np.zeros_like(Y["q1"])
    enorm = lambda q: math.sqrt(o.energy({"q3": q, "q2": zero2, "q1": zero1}) / E0)
    disc = enorm(Y["q3"] - _gaussian_exact(m, T, sigma))
    ratio = {}
    for prec in (dgh.PREC_FP32, dgh.PREC_BF16_TC, dgh.PREC_FP16_TC, dgh.PREC_SPLIT_BF16):
        g = dgh.Solver(VX, EToV, 6, 0, dt=dt, precision=prec)
        g.init_gaussian([0, 0, 0], sigma)
        g.step(nst)
        ratio[prec] = enorm(g.get_state(3) - Y["q3"]) / disc
        g.close()
    print("discretisation error %.3e, precision error / discretisation error: %s" % (disc, ratio))
    assert ratio[dgh.PREC_SPLIT_BF16] <= 0.1
    assert ratio[dgh.PREC_FP32] <= 1e-3
    assert ratio[dgh.PREC_FP32] < ratio[dgh.PREC_SPLIT_BF16] < ratio[dgh.PREC_FP16_TC] < ratio[dgh.PREC_BF16_TC]


def test_batch_groups_by_precision():
    VX, EToV = W.kuhn_mesh(2, 1.0, 0.02, seed=44)
    a = dgh.Solver(VX, EToV, 3, 2, precision=dgh.PREC_FP32)
    b = dgh.Solver(VX, EToV, 3, 2, precision=dgh.PREC_SPLIT_BF16)
    for s in (a, b):
        s.init_gaussian([0.1, 0.0, 0.0], 0.3)
    batch = dgh.Batch([a, b])
    assert batch.counts == (2, 2)
    batch.step(10)
    a.step(10)
    b.step(10)
    assert _rel(batch.get_state(0, 3), a.get_state(3)) <= 2e-6
    assert _rel(batch.get_state(1, 3), b.get_state(3)) <= 2e-5


# one step from a smooth state at full size, per precision: bounds on the
# state and on the one-step increment (relative L2 per field), about three
# times the largest values measured on a B300 (state / increment: FP32 6.1e-8 /
# 1.9e-5, split BF16 1.1e-6 / 2.6e-4, FP16 5.9e-5 / 1.5e-2, BF16 7.3e-4 / 0.17)
FULL_TOL = {dgh.PREC_FP32: (2e-7, 6e-5), dgh.PREC_SPLIT_BF16: (3e-6, 8e-4),
            dgh.PREC_FP16_TC: (2e-4, 5e-2), dgh.PREC_BF16_TC: (2e-3, 0.5)}


def test_precision_fullsize_one_step_on_sampled_cells():
    """The precision form's workload at full size: 32^3 x 6 = 196,608 tets,
    N = 6, three layers (c, rho) = (1, 1), (1.5, 1.2), (2, 1.5), HABC P = 4,
    each precision on its own stream as in the benchmark.  From one smooth
    state (two Gaussian pulses with a velocity field), one step of every
    precision against the FP64 oracle's step of 12^3-hex blocks cut out
    around two sampled 2^3-hex groups: one inside the top layer, one across
    the interface z = 1/3 (heterogeneous upwind flux, Sec. 2.3)."""
    import torch
    from patch_sampling import patch_and_centre, patch_mesh
    n, N = 32, 6
    h = 2.0 / n
    VX, EToV = W.kuhn_mesh(n, 1.0, 0.02, seed=3000)
    c, rho = W.layered_material(VX, EToV, [-1 / 3, 1 / 3], [1.0, 1.5, 2.0], [1.0, 1.2, 1.5])
    centres = [np.array([20, 12, 25]), np.array([8, 18, 20])]   # hexes 20 | 21 straddle z = 1/3
    g = dgh.Solver(VX, EToV, N, 4, c=c, rho=rho)
    x = g.nodes(3)
    dt = g.info["dt"]
    g.close()
    Y0 = np.zeros((x.shape[0], 4, x.shape[1]))
    for cc in centres:
        Y0[:, 0] += np.exp(-np.sum((x - (-1.0 + (cc + 1) * h)) ** 2, axis=2) / 0.1 ** 2)
    Y0[:, 1], Y0[:, 2], Y0[:, 3] = 0.3 * Y0[:, 0], -0.2 * Y0[:, 0], 0.25 * Y0[:, 0]
    Y0 = Y0.astype(np.float32).astype(np.float64)        # the values the GPU holds
    ref = []
    for cc in centres:
        tets, cen, pos = patch_and_centre(n, cc)
        o = Solver(patch_mesh(VX, EToV, tets, N, BC_HABC, c, rho))
        Y = o.zero_state()
        Y["q3"][:] = Y0[tets]
        res = {k: np.zeros_like(v) for k, v in Y.items()}
        o.step(Y, res, 0.0, dt)
        ref.append((cen, Y["q3"][pos]))
    assert np.unique(c[ref[1][0]]).size == 2            # the second group spans two layers
    for prec in (dgh.PREC_FP32, dgh.PREC_SPLIT_BF16, dgh.PREC_FP16_TC, dgh.PREC_BF16_TC):
        st = torch.cuda.Stream()
        g = dgh.Solver(VX, EToV, N, 4, c=c, rho=rho, stream=st, precision=prec)
        assert g.info["dt"] == dt
        g.set_state(3, Y0)
        g.step(1)
        g.sync()
        q3 = g.get_state(3)
        g.close()
        tol_s, tol_i = FULL_TOL[prec]
        for (cen, r), cc in zip(ref, centres):
            for f in range(4):
                e_s = _rel(q3[cen, f], r[:, f])
                e_i = _rel(q3[cen, f] - Y0[cen, f], r[:, f] - Y0[cen, f])
                where = tuple(int(v) for v in cc)
                print("precision %d block at hex %s field %d: state %.2e, one-step increment %.2e" % (prec, where, f, e_s, e_i))
                assert e_s <= tol_s, (prec, where, f, e_s)
                assert e_i <= tol_i, (prec, where, f, e_i)
