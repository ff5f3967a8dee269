"""Pins of the oracle's meshes, DG operators, HABC chain and time stepping
against exact solutions, invariants and physics (Sec. 3.2, 4.1)."""
import math

import numpy as np
import pytest

from oracle.mesh import BC_DIRICHLET, BC_HABC, CuboidMesh, dof_count
from oracle.solver import Solver
from paper_1610_05023_b300 import workloads as W


def make(n, N, P, bc=None, jitter=0.0, seed=1, L=1.0, rho=1.0, c=1.0):
    VX, EToV = W.kuhn_mesh(n, L, jitter, seed)
    bc = [BC_HABC] * 6 if bc is None else bc
    return CuboidMesh(VX, EToV, N, P, bc, rho, c)


# ------------------------------------------------------------------ mesh
@pytest.mark.parametrize("n", [1, 2, 3])
def test_mesh_counts_and_geometry(n):
    m = make(n, 2, 2, jitter=0.02)
    assert m.K == 6 * n ** 3 and m.Ktri == 12 * n * n and m.Klin == 12 * n and m.Kpnt == 8
    assert m.ndof() == dof_count(m.K, m.Ktri, m.Klin, 2, 2)
    assert abs(np.sum(np.abs(m.J)) * 4.0 / 3.0 - 8.0) < 1e-12       # |J| = 3 vol / 4
    # every interior face matched both ways, normals opposite
    k, f = np.nonzero(m.EToE >= 0)
    k2, f2 = m.EToE[k, f], m.EToF[k, f]
    assert np.all(m.EToE[k2, f2] == k) and np.all(m.EToF[k2, f2] == f)
    assert np.allclose(m.n[k, f], -m.n[k2, f2], atol=1e-12)
    assert np.allclose(m.Fscale[k, f] * np.abs(m.J[k]), m.Fscale[k2, f2] * np.abs(m.J[k2]), rtol=1e-12)
    # outward normals
    from oracle.mesh import TET_FACE_VERTS
    cen = m.VX[m.EToV].mean(1)
    fc = m.VX[m.EToV[:, TET_FACE_VERTS]].mean(2)
    assert np.all(np.einsum("kfi,kfi->kf", m.n, fc - cen[:, None]) > 0)
    # boundary faces: normal = domain normal
    ax = m.bface_dom // 2
    sgn = np.where(m.bface_dom % 2 == 1, 1.0, -1.0)
    nb = m.n[m.bface_k, m.bface_f]
    assert np.allclose(nb[np.arange(len(ax)), ax], sgn, atol=1e-12)
    # triangle edges on domain edges: in-plane normal = the other face's normal
    t, e = np.nonzero(m.tri_edge_dom >= 0)
    B = m.tri_edge_dom[t, e]
    pos = (m.tri_axes[t] == (B // 2)[:, None]).argmax(1)
    assert np.allclose(m.n2[t, e, pos], np.where(B % 2 == 1, 1.0, -1.0), atol=1e-12)
    # corner ends: outward tangent is the third face's normal
    for faces, ends in m.corners:
        for l, end in ends:
            X = m.lin_end_dom[l, end]
            assert X // 2 == m.lin_axis[l]
            assert (end == 1) == (X % 2 == 1)


def test_fscale_closed_form_unjittered():
    """E19: on an unjittered Kuhn tet of hex side h, max_f sJ/J = 2 sqrt(2)/h
    (the face through the long diagonal... checked against the geometry)."""
    for n in (1, 2, 4):
        m = make(n, 1, 0)
        h = 2.0 / n
        assert abs(m.Fscale.max() - 2 * math.sqrt(2) / h) < 1e-12
        # dt rule of eq. validBench:timeStep with min over cells
        assert abs(m.dt_rule() - 1.0 / (4 * 2 * math.sqrt(2) / h)) < 1e-14


# ------------------------------------------------------------------ operators
def test_free_stream_interior_rhs_zero():
    m = make(3, 3, 0, jitter=0.05, seed=5)
    s = Solver(m)
    Y = s.zero_state()
    Y["q3"][:, 0] = 1.3
    Y["q3"][:, 1], Y["q3"][:, 2], Y["q3"][:, 3] = 0.3, -0.2, 0.5
    r = s.rhs(Y, 0.0)["q3"]
    interior = np.all(m.EToE >= 0, axis=1)
    assert interior.sum() > 0
    assert np.abs(r[interior]).max() < 1e-11


def _standing_mode(m, t):
    k = math.pi / 2
    w = math.sqrt(3) * k
    x = m.x
    S = [np.sin(k * (x[..., i] + 1)) for i in range(3)]
    C = [np.cos(k * (x[..., i] + 1)) for i in range(3)]
    q = np.zeros((m.K, 4, m.ref3.Np))
    q[:, 0] = math.cos(w * t) * S[0] * S[1] * S[2]
    q[:, 1] = -k * C[0] * S[1] * S[2] * math.sin(w * t) / w
    q[:, 2] = -k * S[0] * C[1] * S[2] * math.sin(w * t) / w
    q[:, 3] = -k * S[0] * S[1] * C[2] * math.sin(w * t) / w
    return q


def test_dirichlet_standing_mode_convergence():
    """p = cos(wt) prod sin(pi (x_i+1)/2) is exact with p = 0 on the cube:
    h-refinement converges at (at least about) rate N+1."""
    errs = []
    N = 2
    for n in (2, 4):
        m = make(n, N, 0, bc=[BC_DIRICHLET] * 6)
        s = Solver(m)
        Y = s.zero_state()
        Y["q3"][:] = _standing_mode(m, 0.0)
        T = 0.5
        nst = int(math.ceil(T / m.dt_rule(0.9)))
        dt = T / nst
        Y, _, t = s.run(Y, 0.0, dt, nst)
        diff = {"q3": Y["q3"] - _standing_mode(m, T), "q2": Y["q2"], "q1": Y["q1"]}
        errs.append(math.sqrt(s.energy(diff)))
    rate = math.log2(errs[0] / errs[1])
    assert rate > N + 0.5, (errs, rate)


def _gaussian_exact(m, t, sigma):
    r = np.linalg.norm(m.x, axis=2)
    F = lambda s: s * np.exp(-s ** 2 / sigma ** 2)
    A = lambda s: -0.5 * sigma ** 2 * np.exp(-s ** 2 / sigma ** 2)
    rs = np.maximum(r, 1e-12)
    p = (F(rs - t) + F(rs + t)) / (2 * rs)
    ur = -((F(rs + t) - F(rs - t)) / (2 * rs) - (A(rs + t) - A(rs - t)) / (2 * rs ** 2))
    small = r < 1e-9
    g = lambda s: np.exp(-s ** 2 / sigma ** 2)
    p[small] = g(t) - 2 * t ** 2 / sigma ** 2 * g(t)     # F'(t)
    ur[small] = 0.0
    q = np.zeros((m.K, 4, m.ref3.Np))
    q[:, 0] = p
    for i in range(3):
        q[:, 1 + i] = ur * m.x[..., i] / rs
    return q


def test_gaussian_pulse_exact_solution():
    """Spherical pulse p0 = exp(-r^2/s^2), u0 = 0, free space (c = rho = 1):
    r p = [F(r-t) + F(r+t)]/2 with F(s) = s exp(-s^2/s0^2).  Compared before
    the pulse reaches the boundary; the error falls with refinement."""
    sigma, T, N = 0.25, 0.35, 3
    errs = []
    for n in (4, 8):
        m = make(n, N, 0, jitter=0.02, seed=3)
        s = Solver(m)
        Y = s.gaussian_state([0, 0, 0], sigma)
        E0 = s.energy(Y)
        nst = int(math.ceil(T / m.dt_rule()))
        Y, _, t = s.run(Y, 0.0, T / nst, nst)
        diff = {"q3": Y["q3"] - _gaussian_exact(m, T, sigma), "q2": Y["q2"], "q1": Y["q1"]}
        errs.append(math.sqrt(s.energy(diff) / E0))
    assert errs[1] < 0.03 and errs[1] < errs[0] / 6, errs


def _gaussian_exact_at(m, t, sigma, x0):
    """The free-space spherical pulse of _gaussian_exact, centred at x0."""
    class Shifted:
        pass
    sm = Shifted()
    sm.x, sm.K, sm.ref3 = m.x - np.asarray(x0, dtype=float), m.K, m.ref3
    return _gaussian_exact(sm, t, sigma)


def test_free_surface_matches_the_method_of_images():
    """A p = 0 face (Sec. 2.4) acts as a mirror with a sign change: in the
    half-space the exact field of a pulse at x0 is the free-space field of x0
    minus that of its mirror image x0' (method of images).  Pulse 0.45 from
    the +z face, compared at t = 0.35, when a large part of it has reflected
    while the other faces are still out of reach.  The image solution must be
    matched far better than the free-space field alone."""
    sigma, T, N, n = 0.25, 0.35, 3, 8
    x0, xi = [0.0, 0.0, 0.55], [0.0, 0.0, 1.45]     # +z face at z = 1
    m = make(n, N, 0, bc=[BC_HABC] * 5 + [BC_DIRICHLET], jitter=0.02, seed=5)
    s = Solver(m)
    Y = s.zero_state()
    Y["q3"] = _gaussian_exact_at(m, 0.0, sigma, x0) - _gaussian_exact_at(m, 0.0, sigma, xi)
    E0 = s.energy(Y)
    nst = int(math.ceil(T / m.dt_rule()))
    Y, _, _ = s.run(Y, 0.0, T / nst, nst)
    img = _gaussian_exact_at(m, T, sigma, x0) - _gaussian_exact_at(m, T, sigma, xi)
    free = _gaussian_exact_at(m, T, sigma, x0)

    def err(ref):
        return math.sqrt(s.energy({"q3": Y["q3"] - ref, "q2": Y["q2"], "q1": Y["q1"]}) / E0)

    e_img, e_free = err(img), err(free)
    assert e_img < 0.03 and e_free > 8 * e_img, (e_img, e_free)


@pytest.mark.parametrize("bc", [BC_HABC, BC_DIRICHLET])
def test_energy_non_increasing(bc):
    """Upwind DG with the basic ABC (HABC of order 0) or p = 0: the discrete
    energy cannot increase (Sec. 4.1)."""
    m = make(2, 2, 0, bc=[bc] * 6, jitter=0.03, seed=9)
    s = Solver(m)
    Y = s.gaussian_state([0.2, -0.1, 0.1], 0.35)
    res = {k: np.zeros_like(v) for k, v in Y.items()}
    dt = m.dt_rule()
    E = [s.energy(Y)]
    t = 0.0
    for _ in range(40):
        t = s.step(Y, res, t, dt)
        E.append(s.energy(Y))
    E = np.array(E)
    assert np.all(np.diff(E) <= 1e-13 * E[0])
    assert E[-1] < 0.9 * E[0] or bc == BC_DIRICHLET


def _operator_matrix(s):
    Y = s.zero_state()
    keys = list(Y)
    sizes = [Y[k].size for k in keys]
    n = sum(sizes)
    A = np.zeros((n, n))
    for j in range(n):
        v = np.zeros(n)
        v[j] = 1.0
        off = 0
        for k, sz in zip(keys, sizes):
            Y[k] = v[off:off + sz].reshape(Y[k].shape)
            off += sz
        r = s.rhs(Y, 0.0)
        A[:, j] = np.concatenate([r[k].ravel() for k in keys])
    return A


@pytest.mark.parametrize("bc,P", [(BC_HABC, 0), (BC_DIRICHLET, 0), (BC_HABC, 1), (BC_HABC, 2)])
def test_semidiscrete_operator_stability(bc, P):
    """Brute-force operator of the full multidimensional system on one hex:
    no eigenvalue with a positive real part (beyond rounding)."""
    m = make(1, 1, P, bc=[bc] * 6)
    s = Solver(m)
    A = _operator_matrix(s)
    lam = np.linalg.eigvals(A)
    assert lam.real.max() < 1e-8 * np.abs(lam).max()
    # one LSERK step equals the degree-5 stability polynomial of dt A
    Y = s.zero_state()
    rng = np.random.default_rng(0)
    y0 = rng.standard_normal(A.shape[0])
    off = 0
    for k in Y:
        Y[k] = y0[off:off + Y[k].size].reshape(Y[k].shape).copy()
        off += Y[k].size
    dt = m.dt_rule()
    Y1, _, _ = s.run(Y, 0.0, dt, 1)
    y1 = np.concatenate([Y1[k].ravel() for k in Y1])
    B = dt * A
    ref = y0.copy()
    term = y0.copy()
    for coef in (1, 1 / 2, 1 / 6, 1 / 24, 1 / 200):
        term = B @ term
        ref = ref + coef * term
    assert np.allclose(y1, ref, atol=1e-12 * np.abs(y0).max())


# ------------------------------------------------------------------ HABC
def test_aux_fields_driven_only_by_boundary_traces():
    """Zero initial auxiliary fields stay exactly zero while the 3D field
    vanishes on the boundary cells (Sec. 2.2: the auxiliary fields start at 0
    for data supported inside the domain)."""
    m = make(3, 2, 2, jitter=0.02)
    s = Solver(m)
    Y = s.gaussian_state([0, 0, 0], 0.3)
    on_bnd = np.zeros(m.K, bool)
    on_bnd[m.bface_k] = True
    Y["q3"][on_bnd] = 0.0
    r = s.rhs(Y, 0.0)
    assert np.abs(r["q2"]).max() == 0.0 and np.abs(r["q1"]).max() == 0.0
    assert np.abs(r["q3"]).max() > 0.1


def _tet_image_map(m, A):
    """For the orthogonal map x -> A x of the mesh onto itself: image cell and
    image node index of every (cell, node)."""
    cen = m.VX[m.EToV].mean(1)
    key = {tuple(np.round(c, 8)): k for k, c in enumerate(cen)}
    kimg = np.array([key[tuple(np.round(A @ c, 8))] for c in cen])
    ximg = np.einsum("ij,knj->kni", A, m.x)
    d = np.linalg.norm(ximg[:, :, None, :] - m.x[kimg][:, None, :, :], axis=3)
    nimg = d.argmin(2)
    assert d.min(2).max() < 1e-10
    return kimg, nimg


def test_symmetry_all_faces_edges_corners():
    """Unjittered Kuhn mesh (invariant under axis permutations and x -> -x),
    centred pulse, HABC on all faces: the 3D solution is invariant under the
    12 symmetries; this exercises every face, edge and corner formula."""
    m = make(2, 2, 2)
    s = Solver(m)
    Y = s.gaussian_state([0, 0, 0], 0.3)
    Y, _, _ = s.run(Y, 0.0, m.dt_rule(), 32)
    assert np.abs(Y["q1"]).max() > 1e-4          # the corners have been reached
    import itertools
    q = Y["q3"]
    scale = np.abs(q).max()
    for perm in itertools.permutations(range(3)):
        for sign in (1.0, -1.0):
            A = sign * np.eye(3)[list(perm)]
            kimg, nimg = _tet_image_map(m, A)
            p_img = q[kimg[:, None], 0, nimg]
            assert np.abs(p_img - q[:, 0]).max() < 1e-10 * scale
            u = q[:, 1:4].transpose(0, 2, 1)                      # [K,Np,3]
            u_img = u[kimg[:, None], nimg]                        # [K,Np,3]
            assert np.abs(u_img - np.einsum("ij,knj->kni", A, u)).max() < 1e-10 * scale


def _inner_error(small, Ys, large, Yl):
    """Energy norm of the difference on the small domain, node for node."""
    cen_l = {tuple(np.round(c, 8)): k for k, c in enumerate(large.VX[large.EToV].mean(1))}
    kmap = np.array([cen_l[tuple(np.round(c, 8))] for c in small.VX[small.EToV].mean(1)])
    return Ys["q3"] - Yl["q3"][kmap]


def test_reflection_falls_with_habc_order():
    """Reflection error (Sec. 4.1, eq. validBench:error against a large-domain
    run with the same inner mesh) falls strictly for P = 0, 1, 2, 3."""
    N, sigma, T = 3, 0.3, 1.6
    big = make(8, N, 0, L=2.0)
    sb = Solver(big)
    dt = big.dt_rule()
    nst = int(math.ceil(T / dt))
    dt = T / nst
    Yb, _, _ = sb.run(sb.gaussian_state([0, 0, 0], sigma), 0.0, dt, nst)
    errs = []
    for P in (0, 1, 2, 3):
        m = make(4, N, P)
        s = Solver(m)
        Y0 = s.gaussian_state([0, 0, 0], sigma)
        E0 = s.energy(Y0)
        Y, _, _ = s.run(Y0, 0.0, dt, nst)
        d = {"q3": _inner_error(m, Y, big, Yb), "q2": Y["q2"] * 0, "q1": Y["q1"] * 0}
        errs.append(math.sqrt(s.energy(d) / E0))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[0] > 10 * errs[3], errs


def test_volume_energy_rate_is_the_upwind_dissipation_across_materials():
    """Sec. 3.2 upwind flux with cell-wise materials (reading E18): the
    semi-discrete 3D energy E = sum_k int p^2 / (2 rho c^2) + rho |u|^2 / 2
    changes at exactly -sum over interior faces of
    int ([p]^2 + Z- Z+ [u.n]^2) / (Z- + Z+), Z = rho c of each side (the
    exact Riemann flux; summation by parts of the nodal operators).  Three
    layers give faces with impedance jumps; the fields are random and
    discontinuous and zero on cells with a boundary face.  The same sum with
    an impedance of 1 everywhere must miss."""
    VX, EToV = W.kuhn_mesh(4, 1.0, 0.03, seed=83)
    c, rho = W.layered_material(VX, EToV, [-1 / 3, 1 / 3], [1.0, 1.5, 2.0], [1.0, 1.2, 1.5])
    m = CuboidMesh(VX, EToV, 3, 0, [BC_HABC] * 6, rho, c)
    o = Solver(m)
    ref, K, Nfp = m.ref3, m.K, m.ref3.Nfp
    inner = np.all(m.EToE >= 0, axis=1)
    q3 = np.random.default_rng(7).normal(size=(K, 4, ref.Np)) * inner[:, None, None]
    rhs = o._rhs3(q3, np.zeros((len(m.bfaces), Nfp)), 0.0)
    J = np.abs(m.J)
    Mr = np.einsum("nj,kfj->kfn", ref.M, rhs)
    dE = np.sum(J * (np.sum(q3[:, 0] * Mr[:, 0], -1) / (m.rho * m.c ** 2)
                     + m.rho * np.sum(q3[:, 1:] * Mr[:, 1:], axis=(-1, -2))))
    E = ref.M @ ref.LIFT                       # face mass blocks (Np x 4 Nfp)
    Z = m.rho * m.c
    diss, diss1, jumps = 0.0, 0.0, 0
    for k in range(K):
        for f in range(4):
            k2 = m.EToE[k, f]
            if k2 < 0:
                continue
            own = ref.Fmask[f]
            nb = ref.Fmask[m.EToF[k, f]][m.nbr_perm[k, f]]
            Ef = E[own][:, f * Nfp:(f + 1) * Nfp] * J[k] * m.Fscale[k, f]
            jp = q3[k, 0, own] - q3[k2, 0, nb]
            ju = m.n[k, f] @ (q3[k, 1:][:, own] - q3[k2, 1:][:, nb])
            pp, uu = jp @ Ef @ jp, ju @ Ef @ ju
            diss += 0.5 * (pp + Z[k] * Z[k2] * uu) / (Z[k] + Z[k2])   # each face seen from both sides
            diss1 += 0.5 * (pp + uu) / 2.0
            jumps += Z[k] != Z[k2]
    assert jumps > 0
    assert abs(dE + diss) <= 1e-12 * diss
    assert abs(dE + diss1) > 1e-2 * diss


def test_point_source_is_the_delta_functional_of_its_cell():
    """Reading E14: the point source enters the pressure equation as
    S(t) M_k^-1 l(x_s) in the cell k that contains x_s.  Pins: the cell
    contains x_s (barycentric coordinates, independent of the oracle's
    reference map), and for every monomial q of degree <= N the cell's exact
    mass matrix gives int_k q s dV = q(x_s)."""
    N = 3
    VX, EToV = W.kuhn_mesh(2, 1.0, 0.05, seed=91)
    m = CuboidMesh(VX, EToV, N, 0, [BC_HABC] * 6, 1.0, 1.0)
    o = Solver(m)
    rng = np.random.default_rng(3)
    for _ in range(6):
        xs = rng.uniform(-0.9, 0.9, 3)
        k = o.add_point_source(xs, 2.0, 0.5)
        vec = o.sources[-1][1]
        v = m.VX[m.EToV[k]]
        lam = np.linalg.solve(np.vstack([v.T, np.ones(4)]), np.append(xs, 1.0))
        assert lam.min() >= -1e-12
        Mk = abs(m.J[k]) * m.ref3.M
        x = m.x[k]
        for a in range(N + 1):
            for b in range(N + 1 - a):
                for c in range(N + 1 - a - b):
                    q = x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** c
                    assert abs(q @ Mk @ vec - xs[0] ** a * xs[1] ** b * xs[2] ** c) < 1e-10


def test_ricker_integral_is_the_antiderivative_of_the_wavelet():
    """Sec. 4.1 Ricker wavelet s(t) = (1 - 2 a) exp(-a), a = (pi f (t - t_s))^2,
    and the source time function S = its antiderivative that vanishes far
    from t_s: central differences of S give s, s(t_s) = 1, S(t_s) = 0, and
    the wavelet has zero mean (S vanishes on both sides)."""
    from oracle.solver import ricker, ricker_integral
    f, ts, h = 2.5, 0.5, 1e-5
    for t in np.linspace(0.0, 1.5, 31):
        fd = (ricker_integral(t + h, f, ts) - ricker_integral(t - h, f, ts)) / (2 * h)
        assert abs(fd - ricker(t, f, ts)) < 1e-8
    assert ricker(ts, f, ts) == 1.0 and ricker_integral(ts, f, ts) == 0.0
    tt = np.linspace(ts - 2.0, ts + 2.0, 400001)
    s = np.array([ricker(t, f, ts) for t in tt])
    assert abs(np.trapezoid(s, tt)) < 1e-9
    assert abs(ricker_integral(ts - 2.0, f, ts)) < 1e-12 and abs(ricker_integral(ts + 2.0, f, ts)) < 1e-12


def test_energy_closed_forms():
    """Sec. 4.1 energy E = sum_k int p^2 / (2 rho c^2) + rho |u|^2 / 2 with
    the exact cell mass matrices: a constant state on three layers gives
    sum_k vol_k (p0^2 / (2 rho_k c_k^2) + rho_k |u0|^2 / 2) with the volumes
    from the vertices, and p = x (u = 0, rho = c = 1) on the jittered cube
    [-1, 1]^3, which the cells still tile exactly, gives int x^2 / 2 = 4/3."""
    N = 2
    VX, EToV = W.kuhn_mesh(3, 1.0, 0.04, seed=92)
    c, rho = W.layered_material(VX, EToV, [-1 / 3, 1 / 3], [1.0, 1.5, 2.0], [1.0, 1.2, 1.5])
    m = CuboidMesh(VX, EToV, N, 0, [BC_HABC] * 6, rho, c)
    o = Solver(m)
    p0, u0 = 0.7, np.array([0.3, -0.4, 0.5])
    Y = o.zero_state()
    Y["q3"][:, 0] = p0
    Y["q3"][:, 1:] = u0[None, :, None]
    v = VX[EToV]
    vol = np.abs(np.linalg.det(np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]], axis=1))) / 6.0
    assert abs(vol.sum() - 8.0) < 1e-12
    E = np.sum(vol * (p0 ** 2 / (2 * rho * c ** 2) + rho * (u0 @ u0) / 2))
    assert abs(o.energy(Y) - E) < 1e-12 * E
    m1 = CuboidMesh(VX, EToV, N, 0, [BC_HABC] * 6, 1.0, 1.0)
    o1 = Solver(m1)
    Y = o1.zero_state()
    Y["q3"][:, 0] = m1.x[..., 0]
    assert abs(o1.energy(Y) - 4.0 / 3.0) < 1e-12


def test_volume_energy_rate_with_boundary_faces():
    """The 3D identity with fields on every cell, p = 0 on two domain faces
    and a random incoming characteristic r- (rm3) on the others: a boundary
    face adds - (p^2 / (2Z) + Z (u.n)^2 / 2) + r- (p - Z u.n) / Z (exterior
    state 2 r-, 0: Sec. 2.2, eq. proc:faceBC) or, on a p = 0 face, - p^2 / Z
    (mirror state, Sec. 2.4).  Pins how the 3D boundary fluxes use r-."""
    from oracle.mesh import BC_DIRICHLET
    VX, EToV = W.kuhn_mesh(3, 1.0, 0.03, seed=86)
    c, rho = W.layered_material(VX, EToV, [-1 / 3, 1 / 3], [1.0, 1.5, 2.0], [1.0, 1.2, 1.5])
    bc = (BC_DIRICHLET, BC_HABC, BC_HABC, BC_HABC, BC_HABC, BC_DIRICHLET)
    m = CuboidMesh(VX, EToV, 3, 0, bc, rho, c)
    o = Solver(m)
    ref, K, Nfp = m.ref3, m.K, m.ref3.Nfp
    rng = np.random.default_rng(10)
    q3 = rng.normal(size=(K, 4, ref.Np))
    rm3 = rng.normal(size=(len(m.bfaces), Nfp))
    rhs = o._rhs3(q3, rm3, 0.0)
    J, Z = np.abs(m.J), m.rho * m.c
    Mr = np.einsum("nj,kfj->kfn", ref.M, rhs)
    dE = np.sum(J * (np.sum(q3[:, 0] * Mr[:, 0], -1) / (m.rho * m.c ** 2)
                     + m.rho * np.sum(q3[:, 1:] * Mr[:, 1:], axis=(-1, -2))))
    E = ref.M @ ref.LIFT
    rate, kinds = 0.0, set()
    for k in range(K):
        for f in range(4):
            own = ref.Fmask[f]
            Ef = E[own][:, f * Nfp:(f + 1) * Nfp] * J[k] * m.Fscale[k, f]
            p, un = q3[k, 0, own], m.n[k, f] @ q3[k, 1:][:, own]
            k2 = m.EToE[k, f]
            if k2 >= 0:
                nb = ref.Fmask[m.EToF[k, f]][m.nbr_perm[k, f]]
                jp, ju = p - q3[k2, 0, nb], un - m.n[k, f] @ q3[k2, 1:][:, nb]
                rate -= 0.5 * (jp @ Ef @ jp + Z[k] * Z[k2] * (ju @ Ef @ ju)) / (Z[k] + Z[k2])
                kinds.add("interior")
            else:
                b = m.bface_index[k, f]
                if m.bc[m.bface_dom[b]] == BC_DIRICHLET:
                    rate -= (p @ Ef @ p) / Z[k]
                    kinds.add("p = 0")
                else:
                    r = rm3[b]
                    rate -= (p @ Ef @ p) / (2 * Z[k]) + Z[k] * (un @ Ef @ un) / 2
                    rate += (r @ Ef @ (p - Z[k] * un)) / Z[k]
                    kinds.add("HABC")
    assert kinds == {"interior", "p = 0", "HABC"}
    assert abs(dE - rate) <= 1e-10 * abs(rate)


def test_ricker_spectrum_peaks_at_the_peak_frequency():
    """Frequency convention of the Ricker wavelet (Sec. 4.1, eq.
    validBench:ricker): its Fourier amplitude |S(f)| = |int s(t) e^{-2 pi i f t} dt|
    has the closed form (2 / sqrt(pi)) (f^2 / f_p^3) exp(-f^2 / f_p^2), whose
    maximum is at f = f_p.  The integral is taken numerically here (trapezoid
    rule on a fine grid), independently of the oracle's formula, so a wrong
    scale inside the exponent (a missing or extra pi, f instead of 2 pi f)
    moves the peak and fails."""
    from oracle.solver import ricker
    for f_peak, ts in ((2.5, 0.5), (4.0, 0.3125)):
        tau = np.linspace(-4.0 / f_peak, 4.0 / f_peak, 40001)
        s = np.array([ricker(ts + x, f_peak, ts) for x in tau])
        freqs = np.linspace(0.05, 3.0, 300) * f_peak
        amp = np.array([abs(np.trapezoid(s * np.exp(-2j * np.pi * f * tau), tau)) for f in freqs])
        closed = 2.0 / np.sqrt(np.pi) * freqs ** 2 / f_peak ** 3 * np.exp(-(freqs / f_peak) ** 2)
        assert np.max(np.abs(amp - closed)) < 1e-8 * np.max(closed)
        assert abs(freqs[np.argmax(amp)] - f_peak) <= (freqs[1] - freqs[0])
