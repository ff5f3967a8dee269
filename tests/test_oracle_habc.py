"""Pins of the Pade coefficients, the edge / corner algebra and LSERK4."""
import math
import os

import numpy as np
import pytest

from oracle import habc
from oracle.mesh import dof_count
from oracle.solver import LSERK_A, LSERK_B, LSERK_C

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ Pade
@pytest.mark.parametrize("P", [1, 2, 3, 4, 6, 8])
def test_pade_two_representations_agree(P):
    X = np.linspace(-0.95, 5.0, 101)
    assert np.allclose(habc.pade_sqrt(X, P), habc.pade_sqrt_ab(X, P), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("P", [1, 2, 3])
def test_pade_matches_taylor_to_order_2P(P):
    # f_P(X) - sqrt(1+X) = O(X^(2P+1)): halving X divides the error by 2^(2P+1)
    e1 = abs(habc.pade_sqrt(0.1, P) - math.sqrt(1.1))
    e2 = abs(habc.pade_sqrt(0.05, P) - math.sqrt(1.05))
    order = math.log2(e1 / e2)
    assert order > 2 * P + 0.5


@pytest.mark.parametrize("P", [0, 1, 2, 3, 5])
def test_plane_wave_reflection_closed_form(P):
    """Continuous HABC reflection for a plane wave at incidence theta:
    R = |cos - f_P(-sin^2)| / (cos + f_P(-sin^2)) = tan(theta/2)^(2(2P+1))."""
    th = np.linspace(0.05, 1.5, 30)
    f = habc.pade_sqrt(-np.sin(th) ** 2, P) if P else np.ones_like(th)
    R = np.abs(np.cos(th) - f) / (np.cos(th) + f)
    assert np.allclose(R, np.tan(th / 2) ** (2 * (2 * P + 1)), rtol=1e-10, atol=1e-15)


# ------------------------------------------------------------------ edge system
@pytest.mark.parametrize("P", [1, 2, 3, 6])
def test_edge_matrix_block_structure(P):
    """The matrix has the form [[D, E], [E, D]] with D diagonal,
    D_a = M + sum_b c_a c_b / (1 + c_a + c_b), E_ab = -c_b (1+c_a)/(1+c_a+c_b)
    (derived by substituting r^- + r^+ = p_ab into eqs. proc:edgeBC1-2)."""
    c, M = habc.pade_coefficients(P)
    A = habc.edge_matrix(c, M) * M
    ca, cb = c[:, None], c[None, :]
    D = np.diag(M + (ca * cb / (1 + ca + cb)).sum(1))
    E = -cb * (1 + ca) / (1 + ca + cb)
    assert np.allclose(A, np.block([[D, E], [E, D]]), atol=1e-12)


@pytest.mark.parametrize("P", [1, 2, 4])
def test_edge_solution_satisfies_integrated_bcs(P):
    """Plug the solution into the first-order BCs of Sec. 2.3 written with
    p and rho c v (eqs. HABCsyst:BClev2a-b) and the time-integrated 1D relation
    (eq. HABCsyst:GovLev2):  (1+c_a+c_b) p_ab - (1+c_b) p_A,a - (1+c_a) p_B,b
    = (1+c_a+c_b) p*_ab,  p - rho c v = 2 r^-."""
    c, M = habc.pade_coefficients(P)
    rng = np.random.default_rng(7)
    n = 5
    rpA, rpB, ps = rng.standard_normal((n, P)), rng.standard_normal((n, P)), rng.standard_normal((n, P, P))
    rmA, rmB = habc.edge_solve(rpA, rpB, ps, c, M)
    for i in range(n):
        pA, pB = rmA[i] + rpA[i], rmB[i] + rpB[i]          # fluxed 2D pressures at the edge
        zvA, zvB = rpA[i] - rmA[i], rpB[i] - rmB[i]          # rho c v of the 2D fields
        pab = np.empty((P, P))
        for a in range(P):
            for b in range(P):
                pab[a, b] = ((1 + c[a] + c[b]) * ps[i, a, b] + (1 + c[b]) * pA[a] + (1 + c[a]) * pB[b]) / (1 + c[a] + c[b])
        for a in range(P):   # L^y p_i00 = 0 on the edge, face A sets
            assert abs((pA[a] - zvA[a]) - (2.0 / M) * sum(c[b] * (pab[a, b] - pA[a]) for b in range(P))) < 1e-12
        for b in range(P):   # L^x p_0j0 = 0 on the edge, face B sets
            assert abs((pB[b] - zvB[b]) - (2.0 / M) * sum(c[a] * (pab[a, b] - pB[b]) for a in range(P))) < 1e-12


@pytest.mark.parametrize("P", [1, 2, 3])
def test_corner_solution_satisfies_integrated_bcs(P):
    """Corner: build p_ijk from the 0D relation (eq. lev3:ijkCorner) and check
    the integrated corner BCs (eqs. bc3:1-3):  p - rho c u = (2/M) sum c (p_ijk - p)."""
    c, M = habc.pade_coefficients(P)
    rng = np.random.default_rng(11)
    rYZ, rXZ, rXY = (rng.standard_normal(P * P) for _ in range(3))
    xYZ, xXZ, xXY = habc.corner_solve(rYZ, rXZ, rXY, c, M)
    p0jk = (xYZ + rYZ).reshape(P, P)
    pi0k = (xXZ + rXZ).reshape(P, P)
    pij0 = (xXY + rXY).reshape(P, P)
    zu = [(rYZ - xYZ).reshape(P, P), (rXZ - xXZ).reshape(P, P), (rXY - xXY).reshape(P, P)]
    pijk = np.empty((P, P, P))
    for i in range(P):
        for j in range(P):
            for k in range(P):
                pijk[i, j, k] = ((1 + c[i]) * p0jk[j, k] + (1 + c[j]) * pi0k[i, k] + (1 + c[k]) * pij0[i, j]) / (1 + c[i] + c[j] + c[k])
    for j in range(P):
        for k in range(P):
            assert abs(p0jk[j, k] - zu[0][j, k] - (2 / M) * sum(c[i] * (pijk[i, j, k] - p0jk[j, k]) for i in range(P))) < 1e-12
    for i in range(P):
        for k in range(P):
            assert abs(pi0k[i, k] - zu[1][i, k] - (2 / M) * sum(c[j] * (pijk[i, j, k] - pi0k[i, k]) for j in range(P))) < 1e-12
    for i in range(P):
        for j in range(P):
            assert abs(pij0[i, j] - zu[2][i, j] - (2 / M) * sum(c[k] * (pijk[i, j, k] - pij0[i, j]) for k in range(P))) < 1e-12


# ------------------------------------------------------------------ LSERK4
def test_lserk_stability_polynomial():
    """s <- a s + dt*lam*y, y <- y + b s on y' = lam y: the amplification
    factor is 1 + z + z^2/2 + z^3/6 + z^4/24 + z^5/200 (z = lam dt)."""
    P = np.polynomial.Polynomial
    y, s = P([1.0]), P([0.0])
    z = P([0.0, 1.0])
    for a, b in zip(LSERK_A, LSERK_B):
        s = a * s + z * y
        y = y + b * s
    assert np.allclose(y.coef, [1, 1, 1 / 2, 1 / 6, 1 / 24, 1 / 200], atol=1e-14)


def test_lserk_stage_times_and_order():
    # y' = f(t) integrates t^3 exactly and stages see the right times
    for deg in range(4):
        y, s, t, dt = 0.0, 0.0, 0.3, 0.1
        for a, b, c in zip(LSERK_A, LSERK_B, LSERK_C):
            s = a * s + dt * (t + c * dt) ** deg
            y = y + b * s
        exact = ((t + dt) ** (deg + 1) - t ** (deg + 1)) / (deg + 1)
        assert abs(y - exact) < 1e-15
    # temporal order 4 on y' = -y + cos(t)
    def run(nsteps):
        y, t, dt = 1.0, 0.0, 1.0 / nsteps
        s = 0.0
        for _ in range(nsteps):
            for a, b, c in zip(LSERK_A, LSERK_B, LSERK_C):
                s = a * s + dt * (-y + math.cos(t + c * dt))
                y = y + b * s
            t += dt
        return y
    exact = 0.5 * (math.cos(1.0) + math.sin(1.0)) + 0.5 * math.exp(-1.0)
    e1, e2 = abs(run(10) - exact), abs(run(20) - exact)
    assert math.log2(e1 / e2) > 3.8


# ------------------------------------------------------------------ Table 3
def test_dof_count_matches_table3():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table3_dofs.txt")) if l.strip() and not l.startswith("#")]
    for P, Ktet, Ktri, Klin, N, total in (map(int, r) for r in rows):
        assert dof_count(Ktet, Ktri, Klin, N, P) == total


# ------------------------------------------ auxiliary fluxes (reading E15)
# With the full pressure equal to p* (q0 = 0), each set of a face or edge
# system is a plain acoustic system: (1 + c) p_t = -rho c^2 div v, rho v_t =
# -grad p, with c = c_a on faces and c_a + c_b on edges.  Its DG energy
#   E = sum over cells of int (1 + c) p^2 / (2 rho c^2) + rho |v|^2 / 2
# then changes at exactly
#   dE/dt = - sum over interior interfaces of int [p]^2 / (2 Z) + Z [v.n]^2 / 2
# when the interfaces use the upwind flux with impedance Z (summation by
# parts of the nodal operators plus the flux algebra; the integrals are
# exact); between cells of different impedance the integrand is
# ([p]^2 + Z- Z+ [v.n]^2) / (Z- + Z+).  Reading E15 takes Z = rho c of the 3D
# medium, and E18 gives each triangle and line cell the material of its tet:
# with three layers of rho c far from 1 the identity pins the auxiliary
# fluxes' signs, factors, lift and neighbour matching against those readings,
# and Z = 1 must miss it.  The fields are random and discontinuous, and zero
# on the cells that touch a domain edge (resp. corner), so that only interior
# interfaces contribute.

def _aux_setup(seed):
    from oracle.mesh import BC_HABC, CuboidMesh
    from oracle.solver import Solver
    from paper_1610_05023_b300 import workloads as W
    VX, EToV = W.kuhn_mesh(6, 1.0, 0.03, seed=seed)
    c, rho = W.layered_material(VX, EToV, [-1 / 3, 1 / 3], [1.6, 2.0, 1.2], [1.5, 1.8, 2.5])   # Z = 2.4, 3.6, 3.0
    m = CuboidMesh(VX, EToV, 3, 2, [BC_HABC] * 6, rho, c)
    return m, Solver(m)


def test_face_system_energy_rate_is_the_upwind_dissipation():
    m, o = _aux_setup(81)
    ref, T, P = m.ref2, m.Ktri, m.P
    rho, cc = m.rho2, m.c2
    Nfp = ref.Nfp
    interior = np.all(m.EToE2 >= 0, axis=1)
    assert 0 < interior.sum() < T
    q2 = np.random.default_rng(5).normal(size=(T, P, 3, ref.Np)) * interior[:, None, None, None]
    rhs = o._rhs2(q2, q2[:, :, 0].copy(), np.zeros((T, 3, P, Nfp)))
    J = np.abs(m.J2)
    Mr = np.einsum("nk,tpfk->tpfn", ref.M, rhs)
    w = 1.0 + o.cP
    dE = np.sum(J[:, None] * (w[None, :] / (rho * cc * cc)[:, None] * np.sum(q2[:, :, 0] * Mr[:, :, 0], axis=-1)
                              + rho[:, None] * np.sum(q2[:, :, 1:3] * Mr[:, :, 1:3], axis=(-1, -2))))
    E = ref.M @ ref.LIFT                       # edge mass blocks (Np x 3 Nfp)
    Z = rho * cc
    diss, diss1, jumps = 0.0, 0.0, 0
    for t in range(T):
        for e in range(3):
            t2 = m.EToE2[t, e]
            if t2 < 0:
                continue
            own = ref.Fmask[e]
            nb = ref.Fmask[m.EToF2[t, e]][m.nbr_perm2[t, e]]
            Ee = E[own][:, e * Nfp:(e + 1) * Nfp] * J[t] * m.Fscale2[t, e]
            jumps += Z[t] != Z[t2]
            for a in range(P):
                jp = q2[t, a, 0, own] - q2[t2, a, 0, nb]
                jv = m.n2[t, e] @ (q2[t, a, 1:3][:, own] - q2[t2, a, 1:3][:, nb])
                pp, vv = jp @ Ee @ jp, jv @ Ee @ jv
                diss += 0.5 * (pp + Z[t] * Z[t2] * vv) / (Z[t] + Z[t2])   # each edge seen from both sides
                diss1 += 0.5 * (pp + vv) / 2.0
    assert jumps > 0
    assert abs(dE + diss) <= 1e-10 * diss
    assert abs(dE + diss1) > 1e-2 * diss


def test_edge_system_energy_rate_is_the_upwind_dissipation():
    m, o = _aux_setup(82)
    ref, L, S = m.ref1, m.Klin, m.P ** 2
    rho, cc = m.rho1, m.c1
    interior = np.all(m.EToE1 >= 0, axis=1)
    assert 0 < interior.sum() < L
    q1 = np.random.default_rng(6).normal(size=(L, S, 2, ref.Np)) * interior[:, None, None, None]
    rhs = o._rhs1(q1, q1[:, :, 0].copy(), np.zeros((L, 2, S)))
    J = np.abs(m.J1)
    Mr = np.einsum("nk,lsfk->lsfn", ref.M, rhs)
    w = np.array([1.0 + o.cP[s % m.P] + o.cP[s // m.P] for s in range(S)])   # set s = a + P b
    dE = np.sum(J[:, None] * (w[None, :] / (rho * cc * cc)[:, None] * np.sum(q1[:, :, 0] * Mr[:, :, 0], axis=-1)
                              + rho[:, None] * np.sum(q1[:, :, 1] * Mr[:, :, 1], axis=-1)))
    end = [0, ref.Np - 1]
    tau = [-1.0, 1.0]                          # outward tangent at the r = -1 and r = +1 ends
    Z = rho * cc
    diss, diss1, jumps = 0.0, 0.0, 0
    for l in range(L):
        for e in range(2):
            l2 = m.EToE1[l, e]
            if l2 < 0:
                continue
            n2 = end[m.EToF1[l, e]]
            jp = q1[l, :, 0, end[e]] - q1[l2, :, 0, n2]
            jv = tau[e] * (q1[l, :, 1, end[e]] - q1[l2, :, 1, n2])
            pp, vv = np.sum(jp * jp), np.sum(jv * jv)
            diss += 0.5 * (pp + Z[l] * Z[l2] * vv) / (Z[l] + Z[l2])      # each point seen from both sides
            diss1 += 0.5 * (pp + vv) / 2.0
            jumps += Z[l] != Z[l2]
    assert jumps > 0
    assert abs(dE + diss) <= 1e-10 * diss
    assert abs(dE + diss1) > 1e-2 * diss


def test_face_system_energy_rate_with_domain_edges():
    """The same identity with fields on every triangle, p = 0 on two domain
    faces and a random incoming characteristic r- (rm2) at the domain edges of
    the HABC faces.  A domain edge then adds, per unit length,
    - (p^2 / (2Z) + Z (v.n)^2 / 2) + r- (p - Z v.n) / Z on an HABC edge
    (upwind with the exterior state built from r+ and r-), and - p^2 / Z on an
    edge shared with a p = 0 face (mirror state).  This pins how the face
    systems combine r+ and r- at domain edges (Sec. 2.3, Algorithm 1)."""
    from oracle.mesh import BC_DIRICHLET, BC_HABC, CuboidMesh
    from oracle.solver import Solver
    from paper_1610_05023_b300 import workloads as W
    VX, EToV = W.kuhn_mesh(3, 1.0, 0.03, seed=84)
    c, rho = W.layered_material(VX, EToV, [-1 / 3, 1 / 3], [1.6, 2.0, 1.2], [1.5, 1.8, 2.5])
    bc = (BC_DIRICHLET, BC_HABC, BC_HABC, BC_HABC, BC_HABC, BC_DIRICHLET)
    m = CuboidMesh(VX, EToV, 3, 2, bc, rho, c)
    o = Solver(m)
    ref, T, P, Nfp = m.ref2, m.Ktri, m.P, m.ref2.Nfp
    rng = np.random.default_rng(8)
    q2 = rng.normal(size=(T, P, 3, ref.Np))
    rm2 = rng.normal(size=(T, 3, P, Nfp))
    rhs = o._rhs2(q2, q2[:, :, 0].copy(), rm2)
    J, Z, w = np.abs(m.J2), m.rho2 * m.c2, 1.0 + o.cP
    Mr = np.einsum("nk,tpfk->tpfn", ref.M, rhs)
    dE = np.sum(J[:, None] * (w[None, :] / (m.rho2 * m.c2 ** 2)[:, None] * np.sum(q2[:, :, 0] * Mr[:, :, 0], axis=-1)
                              + m.rho2[:, None] * np.sum(q2[:, :, 1:3] * Mr[:, :, 1:3], axis=(-1, -2))))
    E = ref.M @ ref.LIFT
    rate, kinds = 0.0, set()
    for t in range(T):
        for e in range(3):
            own = ref.Fmask[e]
            Ee = E[own][:, e * Nfp:(e + 1) * Nfp] * J[t] * m.Fscale2[t, e]
            t2 = m.EToE2[t, e]
            for a in range(P):
                p = q2[t, a, 0, own]
                vn = m.n2[t, e] @ q2[t, a, 1:3][:, own]
                if t2 >= 0:
                    nb = ref.Fmask[m.EToF2[t, e]][m.nbr_perm2[t, e]]
                    jp = p - q2[t2, a, 0, nb]
                    jv = vn - m.n2[t, e] @ q2[t2, a, 1:3][:, nb]
                    rate -= 0.5 * (jp @ Ee @ jp + Z[t] * Z[t2] * (jv @ Ee @ jv)) / (Z[t] + Z[t2])
                    kinds.add("interior")
                elif m.bc[m.tri_edge_dom[t, e]] == BC_DIRICHLET:
                    rate -= (p @ Ee @ p) / Z[t]
                    kinds.add("p = 0")
                else:
                    r = rm2[t, e, a]
                    rate -= (p @ Ee @ p) / (2 * Z[t]) + Z[t] * (vn @ Ee @ vn) / 2
                    rate += (r @ Ee @ (p - Z[t] * vn)) / Z[t]
                    kinds.add("HABC")
    assert kinds == {"interior", "p = 0", "HABC"}
    assert abs(dE - rate) <= 1e-10 * abs(rate)


def test_edge_system_energy_rate_with_corner_ends():
    """The edge-system identity with fields on every line cell, p = 0 on two
    domain faces and a random incoming characteristic r- (rm1) at the line
    ends that reach a domain corner: an end at a corner whose third face has
    the HABC adds - (p^2 / (2Z) + Z w^2 / 2) + r- (p - Z w) / Z (w: the
    velocity along the outward tangent), an end whose third face is p = 0
    adds - p^2 / Z.  Pins the edge systems' corner fluxes (Sec. 2.3)."""
    from oracle.mesh import BC_DIRICHLET, BC_HABC, CuboidMesh
    from oracle.solver import Solver
    from paper_1610_05023_b300 import workloads as W
    VX, EToV = W.kuhn_mesh(3, 1.0, 0.03, seed=85)
    c, rho = W.layered_material(VX, EToV, [-1 / 3, 1 / 3], [1.6, 2.0, 1.2], [1.5, 1.8, 2.5])
    bc = (BC_DIRICHLET, BC_HABC, BC_HABC, BC_HABC, BC_HABC, BC_DIRICHLET)
    m = CuboidMesh(VX, EToV, 3, 2, bc, rho, c)
    o = Solver(m)
    ref, L, S, P = m.ref1, m.Klin, m.P ** 2, m.P
    rng = np.random.default_rng(9)
    q1 = rng.normal(size=(L, S, 2, ref.Np))
    rm1 = rng.normal(size=(L, 2, S))
    rhs = o._rhs1(q1, q1[:, :, 0].copy(), rm1)
    J, Z = np.abs(m.J1), m.rho1 * m.c1
    w = np.array([1.0 + o.cP[s % P] + o.cP[s // P] for s in range(S)])
    Mr = np.einsum("nk,lsfk->lsfn", ref.M, rhs)
    dE = np.sum(J[:, None] * (w[None, :] / (m.rho1 * m.c1 ** 2)[:, None] * np.sum(q1[:, :, 0] * Mr[:, :, 0], axis=-1)
                              + m.rho1[:, None] * np.sum(q1[:, :, 1] * Mr[:, :, 1], axis=-1)))
    end, tau = [0, ref.Np - 1], [-1.0, 1.0]
    rate, kinds = 0.0, set()
    for l in range(L):
        for e in range(2):
            p, wn = q1[l, :, 0, end[e]], tau[e] * q1[l, :, 1, end[e]]
            l2 = m.EToE1[l, e]
            if l2 >= 0:
                n2 = end[m.EToF1[l, e]]
                jp = p - q1[l2, :, 0, n2]
                jv = wn - tau[e] * q1[l2, :, 1, n2]
                rate -= 0.5 * np.sum(jp * jp + Z[l] * Z[l2] * jv * jv) / (Z[l] + Z[l2])
                kinds.add("interior")
            elif m.bc[m.lin_end_dom[l, e]] == BC_DIRICHLET:
                rate -= np.sum(p * p) / Z[l]
                kinds.add("p = 0")
            else:
                r = rm1[l, e]
                rate -= np.sum(p * p / (2 * Z[l]) + Z[l] * wn * wn / 2) - np.sum(r * (p - Z[l] * wn)) / Z[l]
                kinds.add("HABC")
    assert kinds == {"interior", "p = 0", "HABC"}
    assert abs(dE - rate) <= 1e-10 * abs(rate)


def test_face_boundary_algebra_closed_form():
    """Face BC of Algorithm 1 (eqs. proc:faceBC, proc:pi00Star) in closed form:
    with a 3D state of uniform p0 and u0 (so r+ = (p0 + Z n.u0)/2 on a face
    with outward normal n) and uniform p*_a = k_a, every face node gets
    r- = (1/M) sum_a c_a k_a with c_a = tan^2(a pi / M),
    M = 2P + 1, q0 = r- + r+ and the full pressures p_a = k_a + q0."""
    import math
    from oracle.mesh import BC_HABC, CuboidMesh
    from oracle.solver import Solver
    from paper_1610_05023_b300 import workloads as W
    P, rho, c = 3, 1.3, 0.9
    VX, EToV = W.kuhn_mesh(2, 1.0, 0.03, seed=87)
    m = CuboidMesh(VX, EToV, 2, P, [BC_HABC] * 6, rho, c)
    o = Solver(m)
    Y = o.zero_state()
    p0, u0 = 0.4, np.array([0.3, -0.2, 0.6])
    Y["q3"][:, 0] = p0
    Y["q3"][:, 1:] = u0[None, :, None]
    k = np.array([0.5, -1.0, 2.0])
    Y["q2"][:, :, 0] = k[None, :, None]
    cl = o.closure(Y)
    M = 2 * P + 1
    ca = np.array([math.tan(a * math.pi / M) ** 2 for a in range(1, P + 1)])
    rm = np.sum(ca * k) / M
    d = m.tri_d
    rp = (p0 + rho * c * np.where(d % 2 == 1, 1.0, -1.0) * u0[d // 2]) / 2.0     # per triangle
    assert np.abs(cl["rm3"][m.tri_bface] - rm).max() < 1e-13
    q0 = rm + rp
    assert np.abs(cl["p2"] - (k[None, :, None] + q0[:, None, None])).max() < 1e-13
