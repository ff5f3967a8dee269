"""Volume, surface and line meshes of a cuboid (oracle, FP64).

Sec. 3.2: the volume mesh is made of K^tet tetrahedra; the surface mesh is the
set of cell faces lying on the domain faces where the HABC is prescribed, and
the line mesh the set of cell edges lying on the domain edges where two HABCs
meet (K^tri triangles, K^lin line cells, K^pnt corners).  Triangle and line
nodes coincide with the tetrahedron face / edge nodes (they are matched here by
physical coordinates).

Boundary conditions per domain face d = 0..5 (-x,+x,-y,+y,-z,+z):
  BC_HABC       the Pade HABC of the common order P (P = 0 is the basic ABC);
  BC_DIRICHLET  p = 0 (Sec. 2.4; no auxiliary fields on its edges / corners).

Geometry (affine simplices):
  drdx[k, j, i] = d r_j / d x_i         (j: reference direction, i: physical)
  n[k, f, :]    outward unit normal,  Fscale[k, f] = |grad zeta_f| = sJ / J
  where zeta_f = t, s, r+s+t, r for the four tet faces (s, r+s, r for the
  three triangle edges), so that Fscale is the ratio of the face to the volume
  Jacobian whatever the vertex orientation.
"""
import numpy as np

from .refelem import RefLine, RefTet, RefTri

BC_HABC = 0
BC_DIRICHLET = 1

TET_FACE_VERTS = np.array([[0, 1, 2], [0, 1, 3], [1, 2, 3], [0, 2, 3]])
TRI_EDGE_VERTS = np.array([[0, 1], [1, 2], [0, 2]])


def _match_nodes(xa, xb, tol):
    """For point sets xa[..., m, :] and xb[..., m', :] (same shape) return the
    index map perm[..., m] such that xb[..., perm[m]] == xa[..., m]."""
    d = np.linalg.norm(xa[..., :, None, :] - xb[..., None, :, :], axis=-1)
    perm = np.argmin(d, axis=-1)
    dmin = np.take_along_axis(d, perm[..., None], axis=-1)[..., 0]
    if np.any(dmin > tol):
        raise ValueError("node matching failed (max distance %g)" % dmin.max())
    return perm


def _pair_keys(keys):
    """Given integer keys (one per item), return (i, j) index pairs of equal
    keys and the indices of unmatched items.  Raise if a key repeats > 2."""
    order = np.argsort(keys, kind="stable")
    ks = keys[order]
    same = ks[1:] == ks[:-1]
    if np.any(same[1:] & same[:-1]):
        raise ValueError("non-manifold mesh: a face is shared by more than two cells")
    i = order[:-1][same]
    j = order[1:][same]
    matched = np.zeros(len(keys), bool)
    matched[i] = True
    matched[j] = True
    return i, j, np.nonzero(~matched)[0]


class CuboidMesh:
    """All meshes and maps of the multidimensional solver."""

    def __init__(self, VX, EToV, N, P, bc, rho, c, lo=None, hi=None):
        VX = np.asarray(VX, dtype=np.float64)
        EToV = np.asarray(EToV, dtype=np.int64)
        self.N, self.P = int(N), int(P)
        self.bc = np.asarray(bc, dtype=np.int64)
        self.VX, self.EToV = VX, EToV
        self.K = K = EToV.shape[0]
        self.rho = np.asarray(rho, float) * np.ones(K)
        self.c = np.asarray(c, float) * np.ones(K)
        self.lo = VX.min(axis=0) if lo is None else np.asarray(lo, float)
        self.hi = VX.max(axis=0) if hi is None else np.asarray(hi, float)
        self.h = float(np.min(self.hi - self.lo))
        self.tol = 1e-9 * max(1.0, float(np.max(self.hi - self.lo)))
        self.ref3 = RefTet(N)
        self.ref2 = RefTri(N)
        self.ref1 = RefLine(N)
        self._build_volume()
        self._build_boundary()
        self._build_surface()
        self._build_lines()
        self._build_corners()

    # ------------------------------------------------------------------ 3D
    def _build_volume(self):
        ref, K = self.ref3, self.K
        v = self.VX[self.EToV]                        # [K,4,3]
        r, s, t = ref.r, ref.s, ref.t
        self.x = (np.einsum("n,kd->knd", -(1 + r + s + t) / 2, v[:, 0])
                  + np.einsum("n,kd->knd", (1 + r) / 2, v[:, 1])
                  + np.einsum("n,kd->knd", (1 + s) / 2, v[:, 2])
                  + np.einsum("n,kd->knd", (1 + t) / 2, v[:, 3]))
        Jm = np.stack([(v[:, 1] - v[:, 0]) / 2, (v[:, 2] - v[:, 0]) / 2, (v[:, 3] - v[:, 0]) / 2], axis=2)
        self.J = np.linalg.det(Jm)                    # signed
        if np.any(np.abs(self.J) < 1e-14):
            raise ValueError("degenerate tetrahedron")
        self.drdx = np.linalg.inv(Jm)                 # [K, j, i] = d r_j / d x_i
        g = self.drdx
        zeta = np.stack([-g[:, 2], -g[:, 1], g[:, 0] + g[:, 1] + g[:, 2], -g[:, 0]], axis=1)  # [K,4,3]
        self.Fscale = np.linalg.norm(zeta, axis=2)
        self.n = zeta / self.Fscale[..., None]
        # connectivity by sorted vertex triples
        fv = np.sort(self.EToV[:, TET_FACE_VERTS], axis=2).reshape(K * 4, 3)
        nv = self.VX.shape[0]
        keys = (fv[:, 0] * nv + fv[:, 1]) * nv + fv[:, 2]
        i, j, unmatched = _pair_keys(keys)
        self.EToE = np.full((K, 4), -1, np.int64)
        self.EToF = np.full((K, 4), -1, np.int64)
        self.EToE.flat[i], self.EToF.flat[i] = j // 4, j % 4
        self.EToE.flat[j], self.EToF.flat[j] = i // 4, i % 4
        self.bfaces = unmatched                       # global face ids k*4+f
        # node maps of interior faces: neighbour face node index for own face node m
        Fm = ref.Fmask
        self.nbr_perm = np.zeros((K, 4, ref.Nfp), np.int64)
        ii = np.concatenate([i, j])
        jj = np.concatenate([j, i])
        for chunk in np.array_split(np.arange(len(ii)), max(1, len(ii) // 200000)):
            a, b = ii[chunk], jj[chunk]
            xa = self.x[a // 4][np.arange(len(a))[:, None], Fm[a % 4]]
            xb = self.x[b // 4][np.arange(len(b))[:, None], Fm[b % 4]]
            self.nbr_perm.reshape(K * 4, -1)[a] = _match_nodes(xa, xb, self.tol * 10 + 1e-9)

    # ---------------------------------------------------------- boundary
    def _build_boundary(self):
        """Classify every boundary cell face by the domain face it lies on."""
        bf = self.bfaces
        k, f = bf // 4, bf % 4
        pts = self.VX[self.EToV[k[:, None], TET_FACE_VERTS[f]]]   # [Nb,3,3]
        dom = np.full(len(bf), -1, np.int64)
        for a in range(3):
            on_lo = np.all(np.abs(pts[:, :, a] - self.lo[a]) < self.tol, axis=1)
            on_hi = np.all(np.abs(pts[:, :, a] - self.hi[a]) < self.tol, axis=1)
            dom[on_lo] = 2 * a
            dom[on_hi] = 2 * a + 1
        if np.any(dom < 0):
            raise ValueError("a boundary face is not on the cuboid boundary")
        self.bface_dom = dom
        self.bface_k, self.bface_f = k, f
        self.bface_index = np.full((self.K, 4), -1, np.int64)
        self.bface_index[k, f] = np.arange(len(bf))

    def face_is_habc(self, d):
        return self.bc[d] == BC_HABC and self.P >= 1

    # ------------------------------------------------------------- 2D
    def _build_surface(self):
        ref2 = self.ref2
        sel = np.array([self.face_is_habc(d) for d in self.bface_dom], bool)
        self.tri_bface = np.nonzero(sel)[0]           # boundary face index of each triangle
        T = len(self.tri_bface)
        self.Ktri = T
        self.bface_tri = np.full(len(self.bfaces), -1, np.int64)
        self.bface_tri[self.tri_bface] = np.arange(T)
        k = self.bface_k[self.tri_bface]
        f = self.bface_f[self.tri_bface]
        d = self.bface_dom[self.tri_bface]
        self.tri_k, self.tri_f, self.tri_d = k, f, d
        self.tri_vid = self.EToV[k[:, None], TET_FACE_VERTS[f]]  # [T,3] vertex ids in face order
        axes = np.array([[1, 2], [0, 2], [0, 1]])
        self.tri_axes = axes[d // 2]                  # in-plane axes of the triangle
        w = self.VX[self.tri_vid]                     # [T,3,3]
        w2 = np.take_along_axis(w, self.tri_axes[:, None, :], axis=2)  # [T,3,2]
        r, s = ref2.r, ref2.s
        self.x2 = (np.einsum("n,td->tnd", -(r + s) / 2, w2[:, 0])
                   + np.einsum("n,td->tnd", (1 + r) / 2, w2[:, 1])
                   + np.einsum("n,td->tnd", (1 + s) / 2, w2[:, 2]))
        # triangle nodes must coincide with the tet face nodes, in Fmask order
        if T:
            x3 = self.x[k[:, None], self.ref3.Fmask[f]]  # [T,Nfp,3]
            x3p = np.take_along_axis(x3, self.tri_axes[:, None, :], axis=2)
            if np.max(np.abs(x3p - self.x2)) > 1e-9 * max(1.0, self.h):
                raise ValueError("triangle nodes do not coincide with tet face nodes")
        Jm = np.stack([(w2[:, 1] - w2[:, 0]) / 2, (w2[:, 2] - w2[:, 0]) / 2], axis=2)
        self.J2 = np.linalg.det(Jm) if T else np.zeros(0)
        self.drdx2 = np.linalg.inv(Jm) if T else np.zeros((0, 2, 2))
        g = self.drdx2
        zeta = np.stack([-g[:, 1], g[:, 0] + g[:, 1], -g[:, 0]], axis=1) if T else np.zeros((0, 3, 2))
        self.Fscale2 = np.linalg.norm(zeta, axis=2)
        self.n2 = zeta / np.where(self.Fscale2 > 0, self.Fscale2, 1.0)[..., None]
        self.rho2 = self.rho[k]
        self.c2 = self.c[k]
        # connectivity inside each domain face (edges by vertex pairs)
        ev = np.sort(self.tri_vid[:, TRI_EDGE_VERTS], axis=2).reshape(T * 3, 2)
        nv = self.VX.shape[0]
        keys = (ev[:, 0] * nv + ev[:, 1]) * 6 + np.repeat(self.tri_d, 3)
        i, j, unmatched = _pair_keys(keys)
        self.EToE2 = np.full((T, 3), -1, np.int64)
        self.EToF2 = np.full((T, 3), -1, np.int64)
        self.EToE2.flat[i], self.EToF2.flat[i] = j // 3, j % 3
        self.EToE2.flat[j], self.EToF2.flat[j] = i // 3, i % 3
        if len(i) and np.any(self.tri_d[i // 3] != self.tri_d[j // 3]):
            raise ValueError("triangles of different domain faces share an edge")
        Fm = ref2.Fmask
        self.nbr_perm2 = np.zeros((T, 3, ref2.Nfp), np.int64)
        if len(i):
            a = np.concatenate([i, j])
            b = np.concatenate([j, i])
            xa = self.x2[a // 3][np.arange(len(a))[:, None], Fm[a % 3]]
            xb = self.x2[b // 3][np.arange(len(b))[:, None], Fm[b % 3]]
            self.nbr_perm2.reshape(T * 3, -1)[a] = _match_nodes(xa, xb, 1e-8 * max(1.0, self.h))
        # triangle edges on domain edges: the adjacent domain face
        self.tri_edge_dom = np.full((T, 3), -1, np.int64)
        for ge in unmatched:
            t, e = ge // 3, ge % 3
            pts = self.VX[self.tri_vid[t, TRI_EDGE_VERTS[e]]]
            a_own = self.tri_d[t] // 2
            found = -1
            for b in range(3):
                if b == a_own:
                    continue
                if np.all(np.abs(pts[:, b] - self.lo[b]) < self.tol):
                    found = 2 * b
                elif np.all(np.abs(pts[:, b] - self.hi[b]) < self.tol):
                    found = 2 * b + 1
            if found < 0:
                raise ValueError("open triangle edge inside a domain face")
            self.tri_edge_dom[t, e] = found

    # ------------------------------------------------------------- 1D
    def _build_lines(self):
        ref1, ref2 = self.ref1, self.ref2
        lines = []
        for t in range(self.Ktri):
            A = self.tri_d[t]
            for e in range(3):
                B = self.tri_edge_dom[t, e]
                if B < 0 or B < A or not self.face_is_habc(B):
                    continue
                lines.append((t, e, A, B))
        L = len(lines)
        self.Klin = L
        self.lin_triA = np.array([x[0] for x in lines], np.int64)
        self.lin_edgeA = np.array([x[1] for x in lines], np.int64)
        self.lin_A = np.array([x[2] for x in lines], np.int64)
        self.lin_B = np.array([x[3] for x in lines], np.int64)
        self.lin_axis = np.array([3 - self.lin_A[l] // 2 - self.lin_B[l] // 2 for l in range(L)], np.int64)
        # face-B triangle edge with the same vertex pair
        ekey = {}
        for t in range(self.Ktri):
            for e in range(3):
                if self.tri_edge_dom[t, e] >= 0:
                    ekey[(tuple(sorted(self.tri_vid[t, TRI_EDGE_VERTS[e]])), self.tri_d[t])] = (t, e)
        self.lin_triB = np.zeros(L, np.int64)
        self.lin_edgeB = np.zeros(L, np.int64)
        self.lin_vid = np.zeros((L, 2), np.int64)
        self.x1 = np.zeros((L, ref1.Np))
        self.J1 = np.zeros(L)
        self.lin_mapA = np.zeros((L, ref1.Np), np.int64)   # line node -> index in tri edge node list
        self.lin_mapB = np.zeros((L, ref1.Np), np.int64)
        for l, (t, e, A, B) in enumerate(lines):
            vids = self.tri_vid[t, TRI_EDGE_VERTS[e]]
            tB, eB = ekey[(tuple(sorted(vids)), B)]
            if self.tri_d[tB] != B:
                raise ValueError("edge partner is not on face B")
            self.lin_triB[l], self.lin_edgeB[l] = tB, eB
            g = self.lin_axis[l]
            xs = self.VX[vids, g]
            if xs[0] > xs[1]:
                vids = vids[::-1]
                xs = xs[::-1]
            self.lin_vid[l] = vids
            self.x1[l] = xs[0] + (1 + ref1.r) / 2 * (xs[1] - xs[0])
            self.J1[l] = (xs[1] - xs[0]) / 2
            # match with the triangle edge nodes along the axis g
            for side, (tt, ee) in enumerate(((t, e), (tB, eB))):
                ax = self.tri_axes[tt]
                pos = int(np.nonzero(ax == g)[0][0])
                xe = self.x2[tt, ref2.Fmask[ee], pos]
                dist = np.abs(self.x1[l][:, None] - xe[None, :])
                m = np.argmin(dist, axis=1)
                if np.max(dist[np.arange(ref1.Np), m]) > 1e-8 * max(1.0, self.h):
                    raise ValueError("line nodes do not match triangle edge nodes")
                (self.lin_mapA if side == 0 else self.lin_mapB)[l] = m
        self.rho1 = self.rho2[self.lin_triA] if L else np.zeros(0)
        self.c1 = self.c2[self.lin_triA] if L else np.zeros(0)
        # neighbours along the same domain edge: share a vertex
        self.EToE1 = np.full((L, 2), -1, np.int64)
        self.EToF1 = np.full((L, 2), -1, np.int64)
        vend = {}
        for l in range(L):
            for end in range(2):
                vend.setdefault((self.lin_A[l], self.lin_B[l], self.lin_vid[l, end]), []).append((l, end))
        for key, lst in vend.items():
            if len(lst) == 2:
                (l1, e1), (l2, e2) = lst
                self.EToE1[l1, e1], self.EToF1[l1, e1] = l2, e2
                self.EToE1[l2, e2], self.EToF1[l2, e2] = l1, e1
            elif len(lst) > 2:
                raise ValueError("line mesh is not a chain")

    # ------------------------------------------------------------- 0D
    def _build_corners(self):
        """Ends of line cells at domain corners; a corner gets the 0D system
        only when its three faces are all HABC (K^pnt corners)."""
        L = self.Klin
        self.lin_end_dom = np.full((L, 2), -1, np.int64)   # third face at a corner end
        corners = {}
        for l in range(L):
            g = self.lin_axis[l]
            for end in range(2):
                if self.EToE1[l, end] >= 0:
                    continue
                xg = self.VX[self.lin_vid[l, end], g]
                if abs(xg - self.lo[g]) < self.tol:
                    X = 2 * g
                elif abs(xg - self.hi[g]) < self.tol:
                    X = 2 * g + 1
                else:
                    raise ValueError("line chain ends inside the domain edge")
                self.lin_end_dom[l, end] = X
                faces = tuple(sorted((self.lin_A[l], self.lin_B[l], X)))
                corners.setdefault(faces, []).append((l, end))
        self.corners = []
        for faces, lst in sorted(corners.items()):
            if all(self.face_is_habc(d) for d in faces):
                if len(lst) != 3:
                    raise ValueError("corner must join three line cells")
                self.corners.append((faces, lst))
        self.Kpnt = len(self.corners)

    # ------------------------------------------------------------- misc
    def ndof(self):
        """Unknowns of all levels (Table 1 / Table 3 convention)."""
        return (4 * self.ref3.Np * self.K + 3 * self.P * self.ref2.Np * self.Ktri
                + 2 * self.P ** 2 * self.ref1.Np * self.Klin)

    def dt_rule(self, cfl=1.0):
        """Time step of eq. (validBench:timeStep), read with min over cells:
        dt = cfl * min_k 1 / (c_k (N+1)^2 Fscale_k), Fscale_k = max_f sJ/J."""
        return cfl * float(np.min(1.0 / (self.c * (self.N + 1) ** 2 * self.Fscale.max(axis=1))))


def dof_count(Ktet, Ktri, Klin, N, P):
    """Unknowns of the multidimensional solver (Table 1 sizes of q summed over
    the 3D, 2D and 1D solvers): 4 Np K^tet + 3 P Np2 K^tri + 2 P^2 Np1 K^lin."""
    Np3 = (N + 1) * (N + 2) * (N + 3) // 6
    Np2 = (N + 1) * (N + 2) // 2
    Np1 = N + 1
    return 4 * Np3 * Ktet + 3 * P * Np2 * Ktri + 2 * P * P * Np1 * Klin
