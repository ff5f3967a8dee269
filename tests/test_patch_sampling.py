"""The sampling argument of the full-size GPU check, on the oracle alone: one
LSERK4 step of a block of hexes cut out of the 48^3 benchmark mesh leaves the
cells MARGIN = 5 hexes inside the block independent of what happens at the cut
(the cut condition, the block size).  MARGIN is the plain bound: one step
carries a change at most four face hops (five stages), and each hop moves at
most one hex.  Kuhn tetrahedra are slower: a tet has one face on a low side and
one on a high side of its hex, on different axes, so moving one hex along an
axis takes three hops and a margin of 2 is already enough, while a margin of 1
is not (the negative control)."""
import numpy as np

from oracle.mesh import BC_DIRICHLET, BC_HABC
from oracle.solver import Solver
from paper_1610_05023_b300 import workloads as W
from patch_sampling import MARGIN, box_block, corner_block, hex_tets, hex_tets_box, patch_and_centre, patch_mesh

N48 = 48


def _one_step(VX, EToV, tets, bc, x0, dt=5e-4):
    m = patch_mesh(VX, EToV, tets, 4, bc)
    o = Solver(m)
    Y = o.gaussian_state(x0, 0.1)
    Y["q3"][:, 1] = 0.3 * Y["q3"][:, 0]          # a velocity field as well
    Y["q3"][:, 3] = -0.2 * Y["q3"][:, 0]
    res = {k: np.zeros_like(v) for k, v in Y.items()}
    o.step(Y, res, 0.0, dt)
    return Y["q3"]


def test_sampled_cells_do_not_see_the_cut_within_one_step():
    VX, EToV = W.kuhn_mesh(N48, 1.0, 0.02, seed=2000)
    x0 = W.seeded_point(2000, [0.70, 0.65, 0.60], 0.05)
    c = np.floor((np.asarray(x0) + 1.0) / (2.0 / N48)).astype(int)
    tets, cen, pos = patch_and_centre(N48, c)
    abc = _one_step(VX, EToV, tets, BC_HABC, x0)[pos]
    dirichlet = _one_step(VX, EToV, tets, BC_DIRICHLET, x0)[pos]
    # a larger block: the same compared cells, now MARGIN + 2 hexes from the cut
    big = hex_tets(N48, c - MARGIN - 2, 2 + 2 * (MARGIN + 2))
    larger = _one_step(VX, EToV, big, BC_HABC, x0)[np.searchsorted(big, cen)]
    scale = np.abs(abc).max()
    assert scale > 0.5
    # the per-cell arithmetic is the same in all three runs: equal up to the
    # summation order of the library matrix products (bitwise in practice)
    assert np.abs(abc - dirichlet).max() <= 1e-14 * scale
    assert np.abs(abc - larger).max() <= 1e-14 * scale
    # one hex from the cut the cut condition does reach them; two are enough
    for margin, seen in ((1, True), (2, False)):
        near = hex_tets(N48, c - margin, 2 + 2 * margin)
        p2 = np.searchsorted(near, cen)
        d = np.abs(_one_step(VX, EToV, near, BC_HABC, x0)[p2] - _one_step(VX, EToV, near, BC_DIRICHLET, x0)[p2])
        assert (d.max() > 1e-6 * scale) == seen, (margin, d.max())


def _corner_step(VX, EToV, size, bc, x0):
    from patch_sampling import corner_block, line_nodes, patch_mesh, sampled_aux, tri_nodes
    tets, cen, pos = corner_block(N48, size=size)
    m = patch_mesh(VX, EToV, tets, 4, bc, P=6)
    o = Solver(m)
    Y = o.zero_state()
    w = lambda x: np.exp(-np.sum((x - x0) ** 2, axis=-1) / 0.15 ** 2)
    Y["q3"][:, 0] = w(m.x)
    Y["q3"][:, 1], Y["q3"][:, 2], Y["q3"][:, 3] = 0.3 * Y["q3"][:, 0], -0.2 * Y["q3"][:, 0], 0.25 * Y["q3"][:, 0]
    x2, x1 = tri_nodes(m), line_nodes(m)
    for i in range(m.P):
        for f, a in enumerate((1.0, 0.3, -0.2)):
            Y["q2"][:, i, f] = (1 + 0.1 * i) * a * w(x2)
    for s in range(m.P ** 2):
        for f, a in enumerate((1.0, 0.4)):
            Y["q1"][:, s, f] = (1 + 0.05 * s) * a * w(x1)
    res = {k: np.zeros_like(v) for k, v in Y.items()}
    o.step(Y, res, 0.0, 5e-4)
    tri, lin = sampled_aux(m, tets, cen)
    return {"q3": Y["q3"][pos], "q2": Y["q2"][tri], "q1": Y["q1"][lin], "x2": x2[tri], "x1": x1[lin]}


def test_corner_block_levels_do_not_see_the_cut_within_one_step():
    """The same at a domain corner with the HABC (P = 6) on the three domain
    faces: the sampled corner hexes' cells, face triangles and edge line cells
    after one step do not depend on the cut (p = 0 there, or the HABC with its
    own auxiliary fields, which renumbers every level) or on the block size.
    The triangles and line cells are matched across the block meshes by node
    coordinates (patch_sampling.match_rows), as the GPU check matches them to
    the full mesh."""
    from patch_sampling import CORNER_BC, match_rows
    VX, EToV = W.kuhn_mesh(N48, 1.0, 0.02, seed=2000)
    x0 = np.array([0.9, 0.9, 0.9])
    a = _corner_step(VX, EToV, 12, CORNER_BC, x0)
    runs = [_corner_step(VX, EToV, 12, BC_HABC, x0), _corner_step(VX, EToV, 14, CORNER_BC, x0)]
    assert len(a["q2"]) == 3 * 4 * 2 and len(a["q1"]) == 3 * 2    # 3 faces x 2x2 hex faces x 2 tris; 3 edges x 2 lines
    for key in ("q3", "q2", "q1"):
        assert np.abs(a[key]).max() > 0.1, key
    for b in runs:
        j2, j1 = match_rows(a["x2"], b["x2"]), match_rows(a["x1"], b["x1"])
        for key, got in (("q3", b["q3"]), ("q2", b["q2"][j2]), ("q1", b["q1"][j1])):
            scale = np.abs(a[key]).max()
            assert np.abs(got - a[key]).max() <= 1e-14 * scale, key


def test_box_block_indexing():
    """The general block of an (nx, ny, nz) mesh agrees with the cubic
    helpers, and its tets are those whose centroids lie in the block's and
    the sampled hexes' boxes (mesh without jitter: hexes of size h)."""
    t1, c1, p1 = box_block(N48, [20, 21, 22], 2)
    t2, c2, p2 = patch_and_centre(N48, [20, 21, 22])
    assert np.array_equal(t1, t2) and np.array_equal(c1, c2) and np.array_equal(p1, p2)
    t1, c1, p1 = box_block(N48, [N48 - 2] * 3, 2)
    t2, c2, p2 = corner_block(N48, size=2 + MARGIN)
    assert np.array_equal(t1, t2) and np.array_equal(c1, c2) and np.array_equal(p1, p2)
    n3 = (7, 9, 16)
    VX, EToV = W.kuhn_mesh(n3, (0.5 * 7, 0.5 * 9, 0.5 * 16), 0.0)   # unit hexes, corner at -n/2
    cen = VX[EToV].mean(axis=1) + 0.5 * np.asarray(n3)
    tets, cs, pos = box_block(n3, [5, 1, 8], [2, 3, 4])
    inside = lambda lo, hi: np.nonzero(np.all((cen > lo) & (cen < hi), axis=1))[0]
    assert np.array_equal(tets, inside([0, 0, 3], [7, 9, 16]))          # clipped at +x, -y, +z
    assert np.array_equal(cs, inside([5, 1, 8], [7, 4, 12]))
    assert np.array_equal(tets[pos], cs)
    assert np.array_equal(hex_tets_box(N48, [3, 4, 5], 2), hex_tets(N48, [3, 4, 5], 2))
