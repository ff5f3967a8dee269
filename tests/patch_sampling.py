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

from oracle.mesh import TET_FACE_VERTS, CuboidMesh

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


def patch_mesh(VX, EToV, tets, N, bc_code, c=1.0, rho=1.0):
    """The oracle mesh of a block (P = 0, the same code on all six sides);
    c and rho are scalars or per-tet arrays of the whole mesh."""
    E = EToV[tets]
    v = VX[E].reshape(-1, 3)
    pick = lambda a: np.asarray(a, float)[tets] if np.ndim(a) else float(a)
    return PatchMesh(VX, E, N, 0, [bc_code] * 6, pick(rho), pick(c), lo=v.min(0), hi=v.max(0))
