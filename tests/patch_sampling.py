"""Sampled cells of a full-size Kuhn mesh that the FP64 oracle can advance on
its own: a block of hexes cut out of the mesh, with the compared cells at
least 5 hexes inside it.

One LSERK4 step (Appendix A) evaluates the right-hand side five times, and a
cell's right-hand side reads only its own nodes and the traces of its face
neighbours (Sec. 3.2, upwind flux).  A step therefore carries information at
most five face hops, and a face hop between Kuhn tetrahedra changes one hex
index by at most one.  The cut faces of the block lie in hexes that are at
least 5 hexes away from the compared cells, so whatever boundary condition the
block gets there cannot reach them within one step.  A CPU test checks this by
swapping the cut condition and the block size.
"""
import numpy as np
from scipy.spatial import cKDTree

from oracle.mesh import BC_DIRICHLET, BC_HABC, TET_FACE_VERTS, CuboidMesh

MARGIN = 5     # hexes between the compared cells and the cut (one step = 5 stages)


class PatchMesh(CuboidMesh):
    """A block of hexes cut out of a larger mesh.  Its boundary vertices are
    interior vertices of the larger mesh, jittered in 3D, so the boundary
    faces are not on the planes of a box: each is assigned to the nearest
    plane of the block's bounding box.  With P = 0 that only selects the
    condition applied on the cut (basic ABC, or p = 0)."""

    def _build_boundary(self):
        bf = self.bfaces
        k, f = bf // 4, bf % 4
        cen = self.VX[self.EToV[k[:, None], TET_FACE_VERTS[f]]].mean(axis=1)
        a = np.argmin(np.concatenate([cen - self.lo, self.hi - cen], axis=1), axis=1)
        self.bface_dom = np.where(a < 3, 2 * a, 2 * (a - 3) + 1)
        self.bface_k, self.bface_f = k, f
        self.bface_index = np.full((self.K, 4), -1, np.int64)
        self.bface_index[k, f] = np.arange(len(bf))
        # the later plane tests (edges and corners of the domain faces) meet
        # the jittered cut too: a tenth of a hex (h^3 = 6 tets x 4/3 |J|)
        self.tol = 0.1 * float(np.cbrt(8.0 * np.mean(np.abs(self.J))))


def hex_tets(n, lo, size):
    """Tet ids of the hexes [lo, lo + size)^3 of an n^3 Kuhn mesh from
    workloads.kuhn_mesh (hex (i, j, k) = i + n (j + n k), x fastest; its 6
    tets are consecutive)."""
    r = [np.arange(lo[a], lo[a] + size) for a in range(3)]
    I, J, K = np.meshgrid(*r, indexing="ij")
    hexes = (I + n * (J + n * K)).ravel(order="F")
    return (6 * hexes[:, None] + np.arange(6)).ravel()


def patch_and_centre(n, centre_hex, inner=2):
    """(block tet ids, compared tet ids, positions of the compared tets in
    the block) for a block of inner + 2 MARGIN hexes per axis whose inner^3
    central hexes start at centre_hex."""
    c = np.asarray(centre_hex, int)
    lo = c - MARGIN
    size = inner + 2 * MARGIN
    if np.any(lo < 0) or np.any(lo + size > n):
        raise ValueError("block outside the mesh")
    tets = hex_tets(n, lo, size)          # ascending (x fastest, as the hex ids)
    cen = hex_tets(n, c, inner)
    pos = np.searchsorted(tets, cen)
    assert np.array_equal(tets[pos], cen)
    return tets, cen, pos


def patch_mesh(VX, EToV, tets, N, bc_code, c=1.0, rho=1.0, P=0):
    """The oracle mesh of a block; bc_code is one code for all six sides or
    six codes (-x, +x, -y, +y, -z, +z); c and rho are scalars or per-tet
    arrays of the whole mesh."""
    E = EToV[tets]
    v = VX[E].reshape(-1, 3)
    pick = lambda a: np.asarray(a, float)[tets] if np.ndim(a) else float(a)
    bc = list(bc_code) if np.ndim(bc_code) else [bc_code] * 6
    return PatchMesh(VX, E, N, P, bc, pick(rho), pick(c), lo=v.min(0), hi=v.max(0))


# ------------------------------------------------------------ corner blocks
# A block at the (+, +, +) corner of the domain keeps three real domain faces
# (the HABC, with its face, edge and corner levels) and three cut faces (p = 0
# there: no auxiliary fields on the cut and on its edges).  The sampled cells
# are the inner^3 hexes at the corner, size - inner hexes from the cut; the
# auxiliary levels couple only co-located nodes across levels and face or line
# neighbours within a level, so the cut reaches them no faster than the cells.
CORNER_BC = (BC_DIRICHLET, BC_HABC) * 3


def corner_block(n, size=12, inner=2):
    """(block tet ids, sampled tet ids, their positions in the block)."""
    tets = hex_tets(n, np.full(3, n - size), size)
    cen = hex_tets(n, np.full(3, n - inner), inner)
    pos = np.searchsorted(tets, cen)
    assert np.array_equal(tets[pos], cen)
    return tets, cen, pos


def hex_tets_box(n3, lo, size):
    """Tet ids of the hexes lo + [0, size) (per axis) of an (nx, ny, nz) Kuhn
    mesh from workloads.kuhn_mesh (hex (i, j, k) = i + nx (j + ny k))."""
    n3, lo, size = (np.broadcast_to(np.asarray(a, int), (3,)) for a in (n3, lo, size))
    r = [np.arange(lo[a], lo[a] + size[a]) for a in range(3)]
    I, J, K = np.meshgrid(*r, indexing="ij")
    hexes = (I + n3[0] * (J + n3[1] * K)).ravel(order="F")
    return (6 * hexes[:, None] + np.arange(6)).ravel()


def box_block(n3, inner_lo, inner_size):
    """(block tet ids, sampled tet ids, their positions in the block) for the
    sampled hexes inner_lo + [0, inner_size) and a block reaching MARGIN hexes
    beyond them on every side, clipped at the mesh's own faces (which stay
    real domain faces of the block)."""
    n3, ilo, isz = (np.broadcast_to(np.asarray(a, int), (3,)) for a in (n3, inner_lo, inner_size))
    lo = np.maximum(ilo - MARGIN, 0)
    hi = np.minimum(ilo + isz + MARGIN, n3)
    tets = hex_tets_box(n3, lo, hi - lo)
    cen = hex_tets_box(n3, ilo, isz)
    pos = np.searchsorted(tets, cen)
    assert np.array_equal(tets[pos], cen)
    return tets, cen, pos


def tri_nodes(m):
    """[K^tri, Np2, 3] node coordinates of a mesh's triangles in the order of
    its face-level state (the owning tet face's nodes)."""
    return m.x[m.tri_k[:, None], m.ref3.Fmask[m.tri_f]]


def line_nodes(m):
    """[K^lin, Np1, 3] node coordinates of a mesh's line cells in the order
    of its edge-level state (ascending along the edge)."""
    X = np.empty((m.Klin, m.ref1.Np, 3))
    for l in range(m.Klin):
        X[l, :, m.lin_axis[l]] = m.x1[l]
        for d in (m.lin_A[l], m.lin_B[l]):
            X[l, :, d // 2] = m.hi[d // 2] if d % 2 else m.lo[d // 2]
    return X


def match_rows(sub, full, tol=1e-12):
    """For each cell of sub ([M, n, 3] node coordinates) the index of the cell
    of full with the same nodes in the same order."""
    d, j = cKDTree(full.mean(axis=1)).query(sub.mean(axis=1))
    assert np.all(d < 1e-9), d.max()
    assert np.abs(full[j] - sub).max() < tol
    return j


def sampled_aux(m, tets, cen):
    """Triangles and line cells of a block mesh that belong to the sampled
    tets (a line cell through its face-A triangle)."""
    on = np.isin(tets[m.tri_k], cen)
    tri = np.nonzero(on)[0]
    lin = np.nonzero(on[m.lin_triA])[0] if m.Klin else np.zeros(0, np.int64)
    return tri, lin


def block_step(VX, EToV, tets, N, P, bc_code, Yk, x2, x1, t, dt, c=1.0, rho=1.0, sources=()):
    """One oracle step of a block from a full-mesh state Yk = {3: q3, 2: q2,
    1: q1} (canonical layouts; x2, x1: the full mesh's triangle and line node
    coordinates, to match the block's).  sources: (x_s, f_peak, t_s) Ricker
    point sources.  Returns (block mesh, stepped state, triangle map, line
    map, the block's oracle solver)."""
    from oracle.solver import Solver
    m = patch_mesh(VX, EToV, tets, N, bc_code, c=c, rho=rho, P=P)
    o = Solver(m)
    for xs, f, ts in sources:
        o.add_point_source(xs, f, ts)
    Y = o.zero_state()
    Y["q3"][:] = Yk[3][tets]
    tmap = match_rows(tri_nodes(m), x2) if m.Ktri else np.zeros(0, np.int64)
    lmap = match_rows(line_nodes(m), x1) if m.Klin else np.zeros(0, np.int64)
    if m.Ktri:
        Y["q2"][:] = Yk[2][tmap]
    if m.Klin:
        Y["q1"][:] = Yk[1][lmap]
    o.step(Y, {k: np.zeros_like(v) for k, v in Y.items()}, t, dt)
    return m, Y, tmap, lmap, o
