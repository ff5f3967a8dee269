"""Nodal reference elements of the 1D, 2D and 3D solvers (oracle, FP64).

Sec. 3.2: the fields are nodal polynomials of degree N on lines, triangles and
tetrahedra; the tetrahedron nodes are Warp & Blend nodes (Warburton 2006) and
the triangle / line nodes are chosen to coincide with the face / edge nodes of
the tetrahedron.  The elemental matrices D_j (differentiation) and L_f
(lifting) of eq. (dgLocalRhs) are the standard nodal ones (Hesthaven &
Warburton 2008, cited by the paper): V the modal Vandermonde matrix,
D_r = V_r V^{-1}, M = (V V^T)^{-1}, LIFT = V V^T E with the face mass blocks E.

Reference simplices
  line   [-1, 1]
  tri    (-1,-1), (1,-1), (-1,1)
  tet    (-1,-1,-1), (1,-1,-1), (-1,1,-1), (-1,-1,1)
Node order (the canonical order of every read-back): the lattice order of the
equispaced points before warping -- line: r ascending; triangle: s outer, r
inner; tetrahedron: t outer, s middle, r inner.
Face numbering: tet faces t=-1, s=-1, r+s+t=-1, r=-1 (face-local coordinates
(r,s), (r,t), (s,t), (s,t)); triangle edges s=-1, r+s=0, r=-1 (edge
coordinates r, r, s); line ends r=-1, r=1.
"""
import math

import numpy as np

from .jacobi import gauss_jacobi, gll_points, grad_jacobi_p, jacobi_p

# Optimised blending exponents alpha(N) of the 3D Warp & Blend construction
# (Warburton 2006, table for the tetrahedron); alpha = 1 beyond N = 15.
_ALPHA_TET = [0.0, 0.0, 0.0, 0.1002, 1.1332, 1.5608, 1.3413, 1.2577, 1.1603,
              1.10153, 0.6080, 0.4523, 0.8856, 0.8717, 0.9655]

NODE_TOL = 1e-10


def alpha_tet(n):
    return _ALPHA_TET[n - 1] if n <= len(_ALPHA_TET) else 1.0


# ----------------------------------------------------------------------------
# Warp & Blend nodes
# ----------------------------------------------------------------------------
def _divided_warp(n, x):
    """1D warp w(x) = sum_i (x_i^GLL - x_i^equi) l_i^equi(x), divided by the
    edge blend (1 - x^2); zero at the end points."""
    x = np.asarray(x, dtype=np.float64)
    xg = gll_points(n)
    xe = np.linspace(-1.0, 1.0, n + 1)
    warp = np.zeros_like(x)
    for i in range(n + 1):
        li = np.ones_like(x)
        for j in range(n + 1):
            if j != i:
                li = li * (x - xe[j]) / (xe[i] - xe[j])
        warp = warp + (xg[i] - xe[i]) * li
    inside = np.abs(x) < 1.0 - 1e-10
    out = np.zeros_like(x)
    out[inside] = warp[inside] / (1.0 - x[inside] ** 2)
    return out


def _triangle_shift(n, alpha, l1, l2, l3):
    """Warp & Blend displacement inside an equilateral triangle whose vertex
    with barycentric l1 is at the top, l2 bottom-left and l3 bottom-right.
    Returns (dx, dy) in the frame (bottom edge direction, upward)."""
    w1 = 4.0 * l2 * l3 * _divided_warp(n, l3 - l2) * (1.0 + (alpha * l1) ** 2)
    w2 = 4.0 * l1 * l3 * _divided_warp(n, l1 - l3) * (1.0 + (alpha * l2) ** 2)
    w3 = 4.0 * l1 * l2 * _divided_warp(n, l2 - l1) * (1.0 + (alpha * l3) ** 2)
    c2, s2 = math.cos(2 * math.pi / 3), math.sin(2 * math.pi / 3)
    c3, s3 = math.cos(4 * math.pi / 3), math.sin(4 * math.pi / 3)
    dx = w1 + c2 * w2 + c3 * w3
    dy = s2 * w2 + s3 * w3
    return dx, dy


def nodes_line(n):
    return gll_points(n)


def _equi_tri(n):
    """Lattice of the triangle, s outer / r inner, as barycentrics."""
    pts = []
    for j in range(n + 1):          # s index
        for i in range(n + 1 - j):  # r index
            pts.append((i / n, j / n))
    a = np.array(pts)
    # (r, s) of the equispaced lattice
    r = -1.0 + 2.0 * a[:, 0]
    s = -1.0 + 2.0 * a[:, 1]
    return r, s


def nodes_tri(n, alpha):
    """Warp & Blend nodes on the reference triangle (lattice order s outer,
    r inner).  alpha is the blending exponent; the 2D solver uses the 3D value
    so that triangle nodes coincide with tetrahedron face nodes."""
    if n == 0:
        return np.array([-1.0 / 3]), np.array([-1.0 / 3])
    r0, s0 = _equi_tri(n)
    # barycentrics: top vertex (-1,1) <-> l1, (-1,-1) <-> l2, (1,-1) <-> l3
    l1 = (1.0 + s0) / 2.0
    l3 = (1.0 + r0) / 2.0
    l2 = 1.0 - l1 - l3
    # equilateral triangle: l2 -> (-1,-1/sqrt3), l3 -> (1,-1/sqrt3), l1 -> (0,2/sqrt3)
    X = -l2 + l3
    Y = (-l2 - l3 + 2.0 * l1) / math.sqrt(3.0)
    dx, dy = _triangle_shift(n, alpha, l1, l2, l3)
    X = X + dx
    Y = Y + dy
    # back to (r, s): invert the affine map of the equilateral triangle
    L1 = (math.sqrt(3.0) * Y + 1.0) / 3.0
    L3 = (3.0 * X - math.sqrt(3.0) * Y + 2.0) / 6.0
    return 2.0 * L3 - 1.0, 2.0 * L1 - 1.0


def _equi_tet(n):
    pts = []
    for k in range(n + 1):              # t index
        for j in range(n + 1 - k):      # s index
            for i in range(n + 1 - k - j):  # r index
                pts.append((i / n, j / n, k / n))
    a = np.array(pts)
    return -1.0 + 2.0 * a[:, 0], -1.0 + 2.0 * a[:, 1], -1.0 + 2.0 * a[:, 2]


def nodes_tet(n):
    """Warp & Blend nodes on the reference tetrahedron (t outer, s, r inner)."""
    alpha = alpha_tet(n)
    r0, s0, t0 = _equi_tet(n)
    # barycentrics of the four vertices
    bary = {
        1: (1.0 + t0) / 2.0,            # vertex (-1,-1, 1)
        2: (1.0 + s0) / 2.0,            # vertex (-1, 1,-1)
        3: -(1.0 + r0 + s0 + t0) / 2.0,  # vertex (-1,-1,-1)
        4: (1.0 + r0) / 2.0,            # vertex ( 1,-1,-1)
    }
    # equilateral tetrahedron, vertex of barycentric 3,4,2,1 respectively
    q3 = math.sqrt(3.0)
    q6 = math.sqrt(6.0)
    P = {3: np.array([-1.0, -1.0 / q3, -1.0 / q6]),
         4: np.array([1.0, -1.0 / q3, -1.0 / q6]),
         2: np.array([0.0, 2.0 / q3, -1.0 / q6]),
         1: np.array([0.0, 0.0, 3.0 / q6])}
    XYZ = sum(np.outer(bary[v], P[v]) for v in (1, 2, 3, 4))
    # Each face is the zero set of one barycentric la; its triangle has a top
    # vertex (lb), bottom-left (lc) and bottom-right (ld).
    faces = [(1, 2, 3, 4), (2, 1, 3, 4), (3, 1, 4, 2), (4, 1, 3, 2)]
    tol = NODE_TOL
    shift = np.zeros_like(XYZ)
    for la, lb, lc, ld in faces:
        La, Lb, Lc, Ld = bary[la], bary[lb], bary[lc], bary[ld]
        e1 = P[ld] - P[lc]
        e1 = e1 / np.linalg.norm(e1)
        e2 = P[lb] - 0.5 * (P[lc] + P[ld])
        e2 = e2 / np.linalg.norm(e2)
        dx, dy = _triangle_shift(n, alpha, Lb, Lc, Ld)
        blend = Lb * Lc * Ld
        denom = (Lb + 0.5 * La) * (Lc + 0.5 * La) * (Ld + 0.5 * La)
        ok = denom > tol
        blend = np.where(ok, (1.0 + (alpha * La) ** 2) * blend / np.where(ok, denom, 1.0), blend)
        shift = shift + np.outer(blend * dx, e1) + np.outer(blend * dy, e2)
        # nodes on the edges of this face take the face warp alone
        on_edge = (La < tol) & ((Lb > tol).astype(int) + (Lc > tol) + (Ld > tol) < 3)
        shift[on_edge] = np.outer(dx[on_edge], e1) + np.outer(dy[on_edge], e2)
    XYZ = XYZ + shift
    # invert x = c0 + (r/2)(P4-P3) + (s/2)(P2-P3) + (t/2)(P1-P3)
    c0 = 0.5 * (P[4] + P[2] + P[1] - P[3])
    A = 0.5 * np.column_stack((P[4] - P[3], P[2] - P[3], P[1] - P[3]))
    rst = np.linalg.solve(A, (XYZ - c0).T).T
    return rst[:, 0], rst[:, 1], rst[:, 2]


# ----------------------------------------------------------------------------
# Orthonormal modal bases on the simplices
# ----------------------------------------------------------------------------
def _collapsed_tri(r, s):
    a = np.where(np.abs(1.0 - s) > 1e-12, 2.0 * (1.0 + r) / np.where(np.abs(1.0 - s) > 1e-12, 1.0 - s, 1.0) - 1.0, -1.0)
    return a, s


def _pw(x, e):
    """x**e for e >= 0, and 0 for e < 0 (those terms carry a zero factor)."""
    if e < 0:
        return np.zeros_like(x)
    return x ** e


def modes_tri(n):
    return [(i, j) for i in range(n + 1) for j in range(n + 1 - i)]


def basis_tri(r, s, i, j):
    a, b = _collapsed_tri(np.asarray(r, float), np.asarray(s, float))
    return math.sqrt(2.0) * jacobi_p(a, 0, 0, i) * jacobi_p(b, 2 * i + 1, 0, j) * (1.0 - b) ** i


def grad_basis_tri(r, s, i, j):
    a, b = _collapsed_tri(np.asarray(r, float), np.asarray(s, float))
    f, df = jacobi_p(a, 0, 0, i), grad_jacobi_p(a, 0, 0, i)
    g, dg = jacobi_p(b, 2 * i + 1, 0, j), grad_jacobi_p(b, 2 * i + 1, 0, j)
    q = 1.0 - b
    dr = 2.0 * df * g * _pw(q, i - 1)
    ds = df * (1.0 + a) * g * _pw(q, i - 1) + f * dg * _pw(q, i) - i * f * g * _pw(q, i - 1)
    return math.sqrt(2.0) * dr, math.sqrt(2.0) * ds


def _collapsed_tet(r, s, t):
    st = -s - t
    a = np.where(np.abs(st) > 1e-12, 2.0 * (1.0 + r) / np.where(np.abs(st) > 1e-12, st, 1.0) - 1.0, -1.0)
    b = np.where(np.abs(1.0 - t) > 1e-12, 2.0 * (1.0 + s) / np.where(np.abs(1.0 - t) > 1e-12, 1.0 - t, 1.0) - 1.0, -1.0)
    return a, b, t


def modes_tet(n):
    return [(i, j, k) for i in range(n + 1) for j in range(n + 1 - i) for k in range(n + 1 - i - j)]


def basis_tet(r, s, t, i, j, k):
    a, b, c = _collapsed_tet(*(np.asarray(v, float) for v in (r, s, t)))
    return (2.0 * math.sqrt(2.0) * jacobi_p(a, 0, 0, i) * jacobi_p(b, 2 * i + 1, 0, j) * (1.0 - b) ** i
            * jacobi_p(c, 2 * i + 2 * j + 2, 0, k) * (1.0 - c) ** (i + j))


def grad_basis_tet(r, s, t, i, j, k):
    a, b, c = _collapsed_tet(*(np.asarray(v, float) for v in (r, s, t)))
    A, dA = jacobi_p(a, 0, 0, i), grad_jacobi_p(a, 0, 0, i)
    B, dB = jacobi_p(b, 2 * i + 1, 0, j), grad_jacobi_p(b, 2 * i + 1, 0, j)
    C, dC = jacobi_p(c, 2 * i + 2 * j + 2, 0, k), grad_jacobi_p(c, 2 * i + 2 * j + 2, 0, k)
    qb, qc = 1.0 - b, 1.0 - c
    # d/db [B (1-b)^i]
    Bb = dB * _pw(qb, i) - i * B * _pw(qb, i - 1)
    dr = 4.0 * dA * B * C * _pw(qb, i - 1) * _pw(qc, i + j - 1)
    ds = (2.0 * (1.0 + a) * dA * B * C * _pw(qb, i - 1) * _pw(qc, i + j - 1)
          + 2.0 * A * Bb * C * _pw(qc, i + j - 1))
    dt = (2.0 * (1.0 + a) * dA * B * C * _pw(qb, i - 1) * _pw(qc, i + j - 1)
          + (1.0 + b) * A * Bb * C * _pw(qc, i + j - 1)
          + A * B * _pw(qb, i) * (dC * _pw(qc, i + j) - (i + j) * C * _pw(qc, i + j - 1)))
    f = 2.0 * math.sqrt(2.0)
    return f * dr, f * ds, f * dt


def vandermonde_line(n, r):
    return np.column_stack([jacobi_p(r, 0, 0, j) for j in range(n + 1)])


def grad_vandermonde_line(n, r):
    return np.column_stack([grad_jacobi_p(r, 0, 0, j) for j in range(n + 1)])


def vandermonde_tri(n, r, s):
    return np.column_stack([basis_tri(r, s, i, j) for i, j in modes_tri(n)])


def grad_vandermonde_tri(n, r, s):
    g = [grad_basis_tri(r, s, i, j) for i, j in modes_tri(n)]
    return np.column_stack([x[0] for x in g]), np.column_stack([x[1] for x in g])


def vandermonde_tet(n, r, s, t):
    return np.column_stack([basis_tet(r, s, t, i, j, k) for i, j, k in modes_tet(n)])


def grad_vandermonde_tet(n, r, s, t):
    g = [grad_basis_tet(r, s, t, i, j, k) for i, j, k in modes_tet(n)]
    return tuple(np.column_stack([x[d] for x in g]) for d in range(3))


# ----------------------------------------------------------------------------
# Reference elements with D, M, LIFT
# ----------------------------------------------------------------------------
class RefLine:
    """Reference line: N+1 GLL nodes; ends r=-1 (face 0) and r=+1 (face 1)."""

    def __init__(self, n):
        self.N = n
        self.Np = n + 1
        self.r = nodes_line(n)
        self.V = vandermonde_line(n, self.r)
        Vi = np.linalg.inv(self.V)
        self.Dr = grad_vandermonde_line(n, self.r) @ Vi
        self.M = np.linalg.inv(self.V @ self.V.T)
        self.Fmask = np.array([[0], [n]])
        E = np.zeros((self.Np, 2))
        E[0, 0] = 1.0
        E[n, 1] = 1.0
        self.LIFT = self.V @ (self.V.T @ E)


class RefTri:
    """Reference triangle; Warp & Blend nodes with the tetrahedron's alpha."""

    def __init__(self, n, alpha=None):
        self.N = n
        self.Np = (n + 1) * (n + 2) // 2
        self.Nfp = n + 1
        self.alpha = alpha_tet(n) if alpha is None else alpha
        self.r, self.s = nodes_tri(n, self.alpha)
        self.V = vandermonde_tri(n, self.r, self.s)
        Vi = np.linalg.inv(self.V)
        Vr, Vs = grad_vandermonde_tri(n, self.r, self.s)
        self.Dr = Vr @ Vi
        self.Ds = Vs @ Vi
        self.M = np.linalg.inv(self.V @ self.V.T)
        tol = NODE_TOL
        self.Fmask = np.array([
            np.nonzero(np.abs(self.s + 1.0) < tol)[0],
            np.nonzero(np.abs(self.r + self.s) < tol)[0],
            np.nonzero(np.abs(self.r + 1.0) < tol)[0],
        ])
        fcoord = [self.r, self.r, self.s]
        E = np.zeros((self.Np, 3 * self.Nfp))
        for f in range(3):
            x = fcoord[f][self.Fmask[f]]
            V1 = vandermonde_line(n, x)
            E[np.ix_(self.Fmask[f], np.arange(f * self.Nfp, (f + 1) * self.Nfp))] = np.linalg.inv(V1 @ V1.T)
        self.LIFT = self.V @ (self.V.T @ E)


class RefTet:
    """Reference tetrahedron with Warp & Blend nodes."""

    def __init__(self, n):
        self.N = n
        self.Np = (n + 1) * (n + 2) * (n + 3) // 6
        self.Nfp = (n + 1) * (n + 2) // 2
        self.r, self.s, self.t = nodes_tet(n)
        self.V = vandermonde_tet(n, self.r, self.s, self.t)
        Vi = np.linalg.inv(self.V)
        Vr, Vs, Vt = grad_vandermonde_tet(n, self.r, self.s, self.t)
        self.Dr, self.Ds, self.Dt = Vr @ Vi, Vs @ Vi, Vt @ Vi
        self.M = np.linalg.inv(self.V @ self.V.T)
        tol = NODE_TOL
        r, s, t = self.r, self.s, self.t
        self.Fmask = np.array([
            np.nonzero(np.abs(1.0 + t) < tol)[0],
            np.nonzero(np.abs(1.0 + s) < tol)[0],
            np.nonzero(np.abs(1.0 + r + s + t) < tol)[0],
            np.nonzero(np.abs(1.0 + r) < tol)[0],
        ])
        fcoords = [(r, s), (r, t), (s, t), (s, t)]
        E = np.zeros((self.Np, 4 * self.Nfp))
        for f in range(4):
            a, b = (c[self.Fmask[f]] for c in fcoords[f])
            V2 = vandermonde_tri(n, a, b)
            E[np.ix_(self.Fmask[f], np.arange(f * self.Nfp, (f + 1) * self.Nfp))] = np.linalg.inv(V2 @ V2.T)
        self.LIFT = self.V @ (self.V.T @ E)

    def interp_row(self, r, s, t):
        """Values l_n(r,s,t) of the nodal (Lagrange) basis at one point."""
        v = vandermonde_tet(self.N, np.array([r]), np.array([s]), np.array([t]))
        return (v @ np.linalg.inv(self.V))[0]


def gauss_tet_rule(q):
    """Collapsed (Stroud conical product) Gauss rule on the reference tet,
    q points per direction, exact for polynomials of degree 2q-1."""
    xa, wa = gauss_jacobi(0.0, 0.0, q)
    xb, wb = gauss_jacobi(1.0, 0.0, q)
    xc, wc = gauss_jacobi(2.0, 0.0, q)
    A, B, C = np.meshgrid(xa, xb, xc, indexing="ij")
    W = np.einsum("i,j,k->ijk", wa, wb, wc) * 0.125
    A, B, C, W = (x.ravel() for x in (A, B, C, W))
    r = (1.0 + A) * (1.0 - B) * (1.0 - C) / 4.0 - 1.0
    s = (1.0 + B) * (1.0 - C) / 2.0 - 1.0
    t = C
    return r, s, t, W


def gauss_tri_rule(q):
    """Collapsed Gauss rule on the reference triangle (degree 2q-1)."""
    xa, wa = gauss_jacobi(0.0, 0.0, q)
    xb, wb = gauss_jacobi(1.0, 0.0, q)
    A, B = np.meshgrid(xa, xb, indexing="ij")
    W = np.einsum("i,j->ij", wa, wb) * 0.5
    A, B, W = A.ravel(), B.ravel(), W.ravel()
    r = (1.0 + A) * (1.0 - B) / 2.0 - 1.0
    s = B
    return r, s, W
