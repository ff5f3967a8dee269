"""The heterogeneous SEAM stand-in (Sec. 4.2) at full size, every boundary
ingredient at once: three layers, a fast inclusion touching the +x face, a
free surface (p = 0) on top, the HABC of order P = 3 on the other five faces
with its face, edge and corner levels, and a Ricker point source
(516,096 tets, N = 3).

The GPU advances the whole stand-in; one more step is then taken on the GPU
and by the FP64 oracle on two blocks cut out of it (the sampling argument of
tests/patch_sampling.py: the compared cells lie MARGIN hexes inside every cut,
domain faces are kept as they are):
- at the +x face around the inclusion's upper edge: the inclusion's y and z
  boundaries, the layer interface z = 0.25, the HABC face level, the source;
- at the top corner (+x, +y, +z): the layer interface z = 0.25, the free
  surface, two HABC faces, their HABC edge and its end at the free surface;
- at the bottom corner (-x, -y, -z): the layer interface z = -0.25, three
  HABC faces, their three edges and the corner system that joins them.
"""
import numpy as np
import pytest

import paper_1610_05023_b300 as dgh
from oracle.mesh import BC_DIRICHLET, BC_HABC
from oracle.solver import Solver
from paper_1610_05023_b300 import workloads as W
from patch_sampling import box_block, line_nodes, match_rows, patch_mesh, sampled_aux, tri_nodes

pytestmark = pytest.mark.gpu

N, P = 3, 3
BC = (BC_HABC,) * 5 + (BC_DIRICHLET,)                   # free surface on +z
SRC = ([1.68, 0.47, 0.20], 3.0)                          # in the sampled hexes of the face block
H = np.asarray(W.SEAM_HALF) * 2 / np.asarray(W.SEAM_DIMS)
TOL_STATE, TOL_INCR = 1e-6, 5e-5


def _hex(x):
    return np.floor((np.asarray(x) + np.asarray(W.SEAM_HALF)) / H).astype(int)


# (sampled hexes: first index and count per axis; the six codes of the block's sides)
BLOCKS = {
    # +x face, y across the inclusion's edge y = 0.5 (hex 40), z from the
    # inclusion's top z = 0.1 (hex 13) across the interface z = 0.25 (hex 16)
    "face": (([54, 38, 13], [2, 4, 4]), (BC_DIRICHLET, BC_HABC, BC_DIRICHLET, BC_DIRICHLET,
                                         BC_DIRICHLET, BC_DIRICHLET)),
    # the (+x, +y, +z) corner, z from below the interface z = 0.25 to the top
    "corner": (([54, 62, 14], [2, 2, 10]), (BC_DIRICHLET, BC_HABC, BC_DIRICHLET, BC_HABC,
                                            BC_DIRICHLET, BC_DIRICHLET)),
    # the (-x, -y, -z) corner, z from the bottom across the interface z = -0.25 (hex 8)
    "bottom": (([0, 0, 0], [2, 2, 10]), (BC_HABC, BC_DIRICHLET, BC_HABC, BC_DIRICHLET,
                                         BC_HABC, BC_DIRICHLET)),
}


def _bumps(x):
    """Initial pressure: three Gaussians of width 0.15 touching the boundary
    at the three blocks, so that the face, edge and corner levels are active."""
    r1 = np.sum((x - np.array([1.65, 0.45, 0.15])) ** 2, axis=-1)
    r2 = np.sum((x - np.array([1.65, 1.90, 0.60])) ** 2, axis=-1)
    r3 = np.sum((x - np.array([-1.65, -1.90, -0.60])) ** 2, axis=-1)
    return np.exp(-r1 / 0.15 ** 2) + 0.8 * np.exp(-r2 / 0.15 ** 2) + 0.6 * np.exp(-r3 / 0.15 ** 2)


def test_seam_standin_blocks_one_step_match_oracle():
    """After 30 GPU steps from the three bumps (source delay chosen so that the
    Ricker wavelet peaks at the compared step), one step on the GPU and by the
    oracle on each block, started from the GPU's state on every level: per
    field and level, the state within 1e-6 relative and the one-step increment
    within 5e-5 of its own norm (the bounds of the full-size corner check);
    measured on a B300 at most 1.2e-7 and 1.8e-5."""
    import torch
    VX, EToV, c, rho = W.seam_standin(seed=7000)
    cen = VX[EToV].mean(axis=1)
    s = torch.cuda.Stream()
    g = dgh.Solver(VX, EToV, N, P, bc=BC, c=c, rho=rho, stream=s)
    dt = g.info["dt"]
    nst = 30
    t_s = (nst + 0.5) * dt
    g.add_point_source(SRC[0], SRC[1], t_s)
    q3 = np.zeros(g.shape(3))
    q3[:, 0] = _bumps(g.nodes(3))
    q3[:, 1] = 0.3 * q3[:, 0]
    g.set_state(3, q3)
    g.tune(steps=2)
    g.step(nst)
    g.sync()
    Yk = {lv: g.get_state(lv) for lv in (3, 2, 1)}
    t = g.info["time"]
    x2, x1 = g.nodes(2), g.nodes(1)
    g.step(1)
    g.sync()
    Yk1 = {lv: g.get_state(lv) for lv in (3, 2, 1)}
    g.close()
    assert np.all(_hex(SRC[0]) == [54, 39, 15])

    for name, ((ilo, isz), bc) in BLOCKS.items():
        tets, cs, pos = box_block(W.SEAM_DIMS, ilo, isz)
        # the block holds what it is meant to test
        cc = c[cs]
        assert len(np.unique(c[tets])) >= 2
        if name == "face":
            assert np.any(cc == 4.5) and np.any(cc == 2.5) and np.any(cc == 1.5)   # inclusion, two layers
            assert np.isin(W.SEAM_DIMS[0] - 1, ilo[0] + np.arange(isz[0]))
        elif name == "corner":
            assert np.any(cc == 2.5) and np.any(cc == 1.5)                          # interface z = 0.25
            assert np.max(cen[cs, 2]) > 0.7                                        # free surface
        else:
            assert np.any(cc == 3.5) and np.any(cc == 2.5)                          # interface z = -0.25
        m = patch_mesh(VX, EToV, tets, N, bc, c=c, rho=rho, P=P)
        o = Solver(m)
        if name == "face":
            o.add_point_source(SRC[0], SRC[1], t_s)
        Y = o.zero_state()
        tmap, lmap = match_rows(tri_nodes(m), x2), match_rows(line_nodes(m), x1) if m.Klin else None
        Y["q3"][:] = Yk[3][tets]
        Y["q2"][:] = Yk[2][tmap]
        if m.Klin:
            Y["q1"][:] = Yk[1][lmap]
        o.step(Y, {k: np.zeros_like(v) for k, v in Y.items()}, t, dt)
        tri, lin = sampled_aux(m, tets, cs)
        assert len(tri) > 0
        if name == "face":
            assert m.Klin == 0           # the face block's only HABC face meets no other
        else:
            assert len(lin) > 0          # HABC edges: one at the top corner, three at the bottom
        cases = [(3, Y["q3"][pos], Yk1[3][cs], Yk[3][cs]),
                 (2, Y["q2"][tri], Yk1[2][tmap[tri]], Yk[2][tmap[tri]])]
        if len(lin):
            cases.append((1, Y["q1"][lin], Yk1[1][lmap[lin]], Yk[1][lmap[lin]]))
        for lv, ref, gpu, start in cases:
            for f in range(ref.shape[-2]):
                r, gg, st = ref[..., f, :], gpu[..., f, :], start[..., f, :]
                e_state = np.linalg.norm(gg - r) / np.linalg.norm(r)
                e_incr = np.linalg.norm((gg - st) - (r - st)) / np.linalg.norm(r - st)
                print("%s block level %d field %d: state %.2e, one-step increment %.2e (|incr|/|state| %.1e)"
                      % (name, lv, f, e_state, e_incr, np.linalg.norm(r - st) / np.linalg.norm(r)))
                assert e_state <= TOL_STATE, (name, lv, f, e_state)
                assert e_incr <= TOL_INCR, (name, lv, f, e_incr)
