"""Pins of the oracle's reference elements against closed forms computed with
a monomial basis (independent of the Jacobi-polynomial route the oracle uses).
"""
import itertools
import math

import numpy as np
import pytest

from oracle.jacobi import gauss_jacobi, gll_points, jacobi_p
from oracle.refelem import RefLine, RefTet, RefTri, gauss_tri_rule, nodes_tet


# ---------------------------------------------------------------- closed forms
def simplex_monomial_integral(exps):
    """Integral over the reference simplex of prod (1 + x_i)^{e_i}.

    The reference simplex is the image of the unit simplex under x = 2y - 1,
    so the integral is 2^d * 2^{sum e} * Dirichlet integral
    prod e_i! / (sum e + d)!.
    """
    d = len(exps)
    s = sum(exps)
    return 2.0 ** (d + s) * math.prod(math.factorial(e) for e in exps) / math.factorial(s + d)


def monomials(deg, d):
    return [e for e in itertools.product(range(deg + 1), repeat=d) if sum(e) <= deg]


def mono_eval(pts, exps):
    """prod (1 + x_i)^{e_i} at the points pts [n, d]."""
    return np.prod([(1.0 + pts[:, i]) ** e for i, e in enumerate(exps)], axis=0)


def mono_deriv(pts, exps, axis):
    e = list(exps)
    if e[axis] == 0:
        return np.zeros(len(pts))
    c = e[axis]
    e[axis] -= 1
    return c * mono_eval(pts, e)


# ---------------------------------------------------------------- Jacobi / GLL
def test_gauss_jacobi_exactness():
    for a, b in ((0, 0), (1, 0), (2, 0), (1, 1)):
        for q in (1, 2, 4, 6):
            x, w = gauss_jacobi(float(a), float(b), q)
            for k in range(2 * q):
                # int (1-x)^a (1+x)^b (1+x)^k = 2^{a+b+k+1} B(a+1, b+k+1)
                exact = 2.0 ** (a + b + k + 1) * math.gamma(a + 1) * math.gamma(b + k + 1) / math.gamma(a + b + k + 2)
                assert abs(np.sum(w * (1 + x) ** k) - exact) < 1e-12 * max(1, exact)


def test_gll_known_values():
    assert np.allclose(gll_points(1), [-1, 1])
    assert np.allclose(gll_points(2), [-1, 0, 1])
    assert np.allclose(gll_points(3), [-1, -1 / math.sqrt(5), 1 / math.sqrt(5), 1])
    assert np.allclose(gll_points(4), [-1, -math.sqrt(3 / 7), 0, math.sqrt(3 / 7), 1])


def test_jacobi_orthonormal():
    x, w = gauss_jacobi(0.0, 0.0, 12)
    for a, b in ((0, 0), (3, 0), (5, 0)):
        xq, wq = gauss_jacobi(float(a), float(b), 12)
        G = np.array([[np.sum(wq * jacobi_p(xq, a, b, i) * jacobi_p(xq, a, b, j)) for j in range(8)] for i in range(8)])
        assert np.allclose(G, np.eye(8), atol=1e-12)


# ---------------------------------------------------------------- nodes
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6])
def test_tet_nodes_structure(N):
    r, s, t = nodes_tet(N)
    Np = (N + 1) * (N + 2) * (N + 3) // 6
    assert len(r) == Np
    pts = np.stack([r, s, t], 1)
    assert len(np.unique(np.round(pts, 9), axis=0)) == Np
    bary = np.stack([(1 + t) / 2, (1 + s) / 2, -(1 + r + s + t) / 2, (1 + r) / 2], 1)
    assert bary.min() > -1e-12
    # invariance of the node set under all vertex permutations
    key = lambda B: set(map(tuple, np.round(B, 9)))
    base = key(bary)
    for perm in itertools.permutations(range(4)):
        assert key(bary[:, perm]) == base
    # edge nodes are the GLL points
    on_edge = (np.abs(bary) < 1e-10).sum(1) >= 2
    edge_r = np.sort(r[on_edge & (np.abs(s + 1) < 1e-10) & (np.abs(t + 1) < 1e-10)])
    assert np.allclose(edge_r, gll_points(N), atol=1e-12)
    if N <= 2:   # GLL = equispaced: Warp & Blend reduces to the lattice
        lat = [(-1 + 2 * i / N, -1 + 2 * j / N, -1 + 2 * k / N)
               for k in range(N + 1) for j in range(N + 1 - k) for i in range(N + 1 - k - j)]
        assert np.allclose(pts, lat, atol=1e-13)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 6])
def test_triangle_nodes_equal_tet_face_nodes(N):
    tet, tri = RefTet(N), RefTri(N)
    coords = [(tet.r, tet.s), (tet.r, tet.t), (tet.s, tet.t), (tet.s, tet.t)]
    for f in range(4):
        a, b = (c[tet.Fmask[f]] for c in coords[f])
        assert np.allclose(a, tri.r, atol=1e-13) and np.allclose(b, tri.s, atol=1e-13)
    line = RefLine(N)
    for e, coord in enumerate((tri.r, tri.r, tri.s)):
        x = coord[tri.Fmask[e]]
        assert np.allclose(np.sort(x), line.r, atol=1e-13)


# ---------------------------------------------------------------- operators
def _lagrange_from_monomials(nodes, deg, pts):
    """Values of the nodal basis at pts via a monomial Vandermonde matrix."""
    d = nodes.shape[1]
    ex = monomials(deg, d)
    Vn = np.column_stack([mono_eval(nodes, e) for e in ex])
    Vp = np.column_stack([mono_eval(pts, e) for e in ex])
    return Vp @ np.linalg.inv(Vn)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_derivatives_exact(N):
    for ref, d in ((RefLine(N), 1), (RefTri(N), 2), (RefTet(N), 3)):
        pts = np.stack([ref.r, ref.s, ref.t][:d] if d == 3 else ([ref.r, ref.s] if d == 2 else [ref.r]), 1)
        Ds = [ref.Dr] + ([ref.Ds] if d >= 2 else []) + ([ref.Dt] if d == 3 else [])
        for e in monomials(N, d):
            f = mono_eval(pts, e)
            for ax in range(d):
                assert np.allclose(Ds[ax] @ f, mono_deriv(pts, e, ax), atol=1e-10 * max(1, np.abs(f).max()))


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_mass_matrix_exact(N):
    for ref, d in ((RefLine(N), 1), (RefTri(N), 2), (RefTet(N), 3)):
        pts = np.stack([ref.r, ref.s, ref.t][:d] if d == 3 else ([ref.r, ref.s] if d == 2 else [ref.r]), 1)
        ex = monomials(N, d)
        for e1 in ex[:6]:
            for e2 in ex[-6:]:
                f, g = mono_eval(pts, e1), mono_eval(pts, e2)
                exact = simplex_monomial_integral([a + b for a, b in zip(e1, e2)])
                assert abs(f @ ref.M @ g - exact) < 1e-10 * max(1, exact)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_tet_lift_is_face_integral(N):
    """M LIFT g equals int_face g l_n dS (face-coordinate measure), computed by
    a collapsed Gauss rule with the nodal basis built from monomials."""
    tet = RefTet(N)
    nodes = np.stack([tet.r, tet.s, tet.t], 1)
    rq, sq, wq = gauss_tri_rule(N + 2)
    rng = np.random.default_rng(3)
    # face points in 3D and face-local coordinates (r,s), (r,t), (s,t), (s,t)
    maps = [lambda a, b: np.stack([a, b, -np.ones_like(a)], 1),
            lambda a, b: np.stack([a, -np.ones_like(a), b], 1),
            lambda a, b: np.stack([-1 - a - b, a, b], 1),
            lambda a, b: np.stack([-np.ones_like(a), a, b], 1)]
    fcoords = [(tet.r, tet.s), (tet.r, tet.t), (tet.s, tet.t), (tet.s, tet.t)]
    Nfp = tet.Nfp
    for f in range(4):
        g_nodes = rng.standard_normal(Nfp)
        fa, fb = (c[tet.Fmask[f]] for c in fcoords[f])
        g_q = _lagrange_from_monomials(np.stack([fa, fb], 1), N, np.stack([rq, sq], 1)) @ g_nodes
        l_q = _lagrange_from_monomials(nodes, N, maps[f](rq, sq))        # [nq, Np]
        exact = l_q.T @ (wq * g_q)
        got = tet.M @ tet.LIFT[:, f * Nfp:(f + 1) * Nfp] @ g_nodes
        assert np.allclose(got, exact, atol=1e-11)


def test_tri_lift_is_edge_integral():
    for N in (1, 2, 3, 4):
        tri = RefTri(N)
        nodes = np.stack([tri.r, tri.s], 1)
        xq, wq = gauss_jacobi(0.0, 0.0, N + 2)
        maps = [lambda a: np.stack([a, -np.ones_like(a)], 1),
                lambda a: np.stack([a, -a], 1),
                lambda a: np.stack([-np.ones_like(a), a], 1)]
        ecoord = [tri.r, tri.r, tri.s]
        rng = np.random.default_rng(4)
        for e in range(3):
            g_nodes = rng.standard_normal(tri.Nfp)
            xe = ecoord[e][tri.Fmask[e]]
            g_q = _lagrange_from_monomials(xe[:, None], N, xq[:, None]) @ g_nodes
            l_q = _lagrange_from_monomials(nodes, N, maps[e](xq))
            exact = l_q.T @ (wq * g_q)
            got = tri.M @ tri.LIFT[:, e * tri.Nfp:(e + 1) * tri.Nfp] @ g_nodes
            assert np.allclose(got, exact, atol=1e-11)
