"""Semi-discrete DG + HABC system and LSERK4 time stepping (oracle, FP64).

The oracle integrates dY/dt = F(Y, t) where Y holds
  q3[k, (p,u,v,w), n]            3D fields on the tetrahedra
  q2[tri, a, (p*,v1,v2), n]      2D temporaries p*_a and in-plane velocities
                                 (v1, v2 along the two in-plane axes in
                                 increasing axis order) for every set a
  q1[lin, s, (p*,w), n]          1D temporaries p*_ab and the velocity along
                                 the edge axis, set s = a + P*b (a: set of the
                                 lower-numbered face A, b: face B)
F evaluates, in the order of Algorithm 1, the boundary algebra (face BC, edge
system, corner system) from the current Y and then the DG right-hand sides of
eq. (dgLocalRhs) on all levels.  This equals the paper's procedure, in which
the incoming characteristics used by a stage are those computed from the
fields at the end of the previous stage.

DG right-hand side (strong form of eqs. weakDG1-2, Hesthaven & Warburton):
  dp/dt = -rho c^2 div u - LIFT( Fscale rho c^2 ((n.u)* - n.u^-) )
  du/dt = -(1/rho) grad p - LIFT( Fscale (1/rho) (p* - p^-) n )
with the upwind fluxes of Sec. 3.2: the exact Riemann solver form
  p*     = ({p/Z} - n.[[u]]) / {1/Z},   (n.u)* = (n.{Z u} - [[p]]) / {Z},
Z = rho c, {X} = (X^ext + X^int)/2, [[X]] = (X^ext - X^int)/2; at boundaries
with an incoming characteristic r^-_ext (basic ABC: 0; HABC: from the face /
edge / corner algebra)   p* = r^+ + r^-_ext,  (n.u)* = (r^+ - r^-_ext)/Z,
r^+ = (p^- + Z n.u^-)/2; at p = 0 faces p* = 0, (n.u)* = n.u^- + p^-/Z.
The 2D and 1D auxiliary systems (eqs. proc:2Dpvsyst1-3, proc:1Dpvsyst1-2) use
the same fluxes applied to the full auxiliary pressure and the in-plane (edge)
normal velocity, with Z = rho c of the cell; the pressure equation is divided
by (1 + c_a) (2D) or (1 + c_a + c_b) (1D).

Time stepping: the 5-stage 2N-storage RK4 of Carpenter & Kennedy (eqs.
timeStepProc1-2 read with the time step):  s <- A_i s + dt F(q, t + C_i dt),
q <- q + B_i s.
"""
import math

import numpy as np

from . import habc
from .mesh import BC_DIRICHLET, BC_HABC, CuboidMesh

# Carpenter & Kennedy (1994), 5-stage 2N-storage fourth-order RK
LSERK_A = np.array([0.0,
                    -567301805773.0 / 1357537059087.0,
                    -2404267990393.0 / 2016746695238.0,
                    -3550918686646.0 / 2091501179385.0,
                    -1275806237668.0 / 842570457699.0])
LSERK_B = np.array([1432997174477.0 / 9575080441755.0,
                    5161836677717.0 / 13612068292357.0,
                    1720146321549.0 / 2090206949498.0,
                    3134564353537.0 / 4481467310338.0,
                    2277821191437.0 / 14882151754819.0])
LSERK_C = np.array([0.0,
                    1432997174477.0 / 9575080441755.0,
                    2526269341429.0 / 6820363962896.0,
                    2006345519317.0 / 3224310063776.0,
                    2802321613138.0 / 2924317926251.0])


def ricker(t, f_peak, t_s):
    """Ricker wavelet s(t) (eq. validBench:ricker)."""
    a = (math.pi * f_peak * (t - t_s)) ** 2
    return (1.0 - 2.0 * a) * math.exp(-a)


def ricker_integral(t, f_peak, t_s):
    """S(t) = integral of s, = (t - t_s) exp(-pi^2 f^2 (t - t_s)^2)."""
    return (t - t_s) * math.exp(-(math.pi * f_peak * (t - t_s)) ** 2)


def upwind(pm, unm, pp, unp, Zm, Zp):
    """Exact Riemann solver fluxes at an interface (Sec. 3.2).  unp is the
    exterior velocity projected on the interior normal."""
    avg_pZ = 0.5 * (pp / Zp + pm / Zm)
    jump_un = 0.5 * (unp - unm)
    avg_iZ = 0.5 * (1.0 / Zp + 1.0 / Zm)
    pstar = (avg_pZ - jump_un) / avg_iZ
    avg_Zun = 0.5 * (Zp * unp + Zm * unm)
    jump_p = 0.5 * (pp - pm)
    avg_Z = 0.5 * (Zp + Zm)
    unstar = (avg_Zun - jump_p) / avg_Z
    return pstar, unstar


class Solver:
    """FP64 reference solver on a CuboidMesh."""

    def __init__(self, mesh: CuboidMesh):
        self.m = mesh
        m = mesh
        self.cP, self.M = habc.pade_coefficients(m.P) if m.P >= 1 else (np.zeros(0), 1)
        self.sources = []      # (k, vector, f_peak, t_s, amp)
        if m.P >= 1:
            self._edge_A = habc.edge_matrix(self.cP, self.M)
            self._corner_A = habc.corner_matrix(self.cP, self.M) if m.Kpnt else None

    # ------------------------------------------------------------- state
    def zero_state(self):
        m = self.m
        return {
            "q3": np.zeros((m.K, 4, m.ref3.Np)),
            "q2": np.zeros((m.Ktri, m.P, 3, m.ref2.Np)),
            "q1": np.zeros((m.Klin, m.P * m.P, 2, m.ref1.Np)),
        }

    def gaussian_state(self, x0, width, amp=1.0):
        """p = amp exp(-|x - x0|^2 / width^2) at the nodes, u = 0, aux = 0."""
        Y = self.zero_state()
        d2 = np.sum((self.m.x - np.asarray(x0)) ** 2, axis=2)
        Y["q3"][:, 0] = amp * np.exp(-d2 / width ** 2)
        return Y

    def add_point_source(self, xs, f_peak, t_s, amp=1.0):
        """Ricker point source delta(x - xs) S(t) in the pressure equation,
        discretised as S(t) M_k^{-1} l(xs) in the cell containing xs (the
        lowest cell id when xs lies on a shared face)."""
        m = self.m
        xs = np.asarray(xs, float)
        for k in range(m.K):
            v = m.VX[m.EToV[k]]
            rst = m.drdx[k] @ (xs - 0.5 * (v[1] + v[2] + v[3] - v[0]))
            r, s, t = rst
            if min(r, s, t) >= -1 - 1e-12 and r + s + t <= -1 + 1e-12:
                row = m.ref3.interp_row(r, s, t)
                vec = (m.ref3.V @ (m.ref3.V.T @ row)) / abs(m.J[k])
                self.sources.append((k, vec, f_peak, t_s, amp))
                return k
        raise ValueError("source point outside the mesh")

    # ------------------------------------------------------ HABC algebra
    def closure(self, Y):
        """Boundary algebra of Algorithm 1 from the current fields.

        Returns a dict with
          rm3[bface, m]   incoming 3D characteristic at boundary face nodes
          p2[tri, a, n]   full 2D pressure p_a = p*_a + q0
          rm2[tri, e, a, m] incoming 2D characteristic at domain-edge edges
          p1[lin, s, n]   full 1D pressure
          rm1[lin, end, s] incoming 1D characteristic at corner ends
        """
        m = self.m
        ref3, ref2, ref1 = m.ref3, m.ref2, m.ref1
        P, c, M = m.P, self.cP, self.M
        q3 = Y["q3"]
        out = {}
        # ---- 2D solver: 3D outgoing characteristic, face BC, full 2D pressure
        k, f = m.bface_k, m.bface_f
        Fm = ref3.Fmask[f]                                       # [Nb, Nfp]
        pm = q3[k[:, None], 0, Fm]
        unm = np.einsum("bi,bim->bm", m.n[k, f], q3[k[:, None], 1:4, Fm].transpose(0, 2, 1))
        Z = (m.rho * m.c)[k][:, None]
        rp3 = (pm + Z * unm) / 2.0                               # eq. proc:charact1
        rm3 = np.zeros_like(rp3)
        p2 = np.zeros((m.Ktri, P, ref2.Np))
        if m.Ktri:
            ps2 = Y["q2"][:, :, 0, :]                             # p*_a
            rm_t = np.einsum("a,tan->tn", c, ps2) / M             # eq. proc:faceBC
            rm3[m.tri_bface] = rm_t
            q0 = rm_t + rp3[m.tri_bface]
            p2 = ps2 + q0[:, None, :]                            # eq. proc:pi00Star
        out["rm3"], out["p2"] = rm3, p2
        # ---- 1D solver: 2D outgoing characteristics, edge system, full 1D pressure
        rm2 = np.zeros((m.Ktri, 3, P, ref2.Nfp))
        p1 = np.zeros((m.Klin, P * P, ref1.Np))
        if m.Klin:
            L = m.Klin
            rp = []
            for tri, edge, mp in ((m.lin_triA, m.lin_edgeA, m.lin_mapA), (m.lin_triB, m.lin_edgeB, m.lin_mapB)):
                nodes = ref2.Fmask[edge][np.arange(L)[:, None], mp]              # [L, Np1] tri node ids
                pa = p2[tri[:, None, None], np.arange(P)[None, :, None], nodes[:, None, :]]  # [L,P,Np1]
                v = Y["q2"][tri[:, None, None], np.arange(P)[None, :, None], 1:3, nodes[:, None, :]]  # [L,P,Np1,2]
                nrm = m.n2[tri, edge]                                            # [L,2]
                vn = np.einsum("ld,lpnd->lpn", nrm, v)
                Zt = (m.rho2 * m.c2)[tri][:, None, None]
                rp.append((pa + Zt * vn) / 2.0)                                  # eq. proc:charact2
            rpA, rpB = rp
            ps1 = Y["q1"][:, :, 0, :].reshape(L, P, P, ref1.Np)                  # [L, a, b, n] (s = a + P b -> [b][a])
            ps1 = ps1.transpose(0, 2, 1, 3)                                      # [L, a, b, n]
            nn = L * ref1.Np
            rA = rpA.transpose(0, 2, 1).reshape(nn, P)
            rB = rpB.transpose(0, 2, 1).reshape(nn, P)
            psn = ps1.transpose(0, 3, 1, 2).reshape(nn, P, P)
            rhs = np.stack([-habc.edge_residual(np.zeros(2 * P), rA[i], rB[i], psn[i], c, M) for i in range(nn)], axis=1)
            x = np.linalg.solve(self._edge_A, rhs)
            rmA = x[:P].T.reshape(L, ref1.Np, P).transpose(0, 2, 1)              # [L,P,Np1]
            rmB = x[P:].T.reshape(L, ref1.Np, P).transpose(0, 2, 1)
            QA = (rmA + rpA).transpose(0, 2, 1)                                  # [L,Np1,P]
            QB = (rmB + rpB).transpose(0, 2, 1)
            pab = habc.edge_pressure(psn.reshape(L, ref1.Np, P, P), QA, QB, c)   # [L,Np1,a,b]
            p1 = pab.transpose(0, 3, 2, 1).reshape(L, P * P, ref1.Np)            # s = a + P b
            for l in range(L):
                rm2[m.lin_triA[l], m.lin_edgeA[l], :, m.lin_mapA[l]] = rmA[l].T
                rm2[m.lin_triB[l], m.lin_edgeB[l], :, m.lin_mapB[l]] = rmB[l].T
        out["rm2"], out["p1"] = rm2, p1
        # ---- 0D solver: 1D outgoing characteristics, corner system
        rm1 = np.zeros((m.Klin, 2, P * P))
        for faces, ends in m.corners:
            X, Yf, Zf = faces                      # sorted: axis 0, 1, 2 faces
            rp_by_edge = {}
            for l, end in ends:
                nd = ref1.Fmask[end][0]
                tau = -1.0 if end == 0 else 1.0    # outward tangent along +axis
                Zl = m.rho1[l] * m.c1[l]
                rp_by_edge[(m.lin_A[l], m.lin_B[l])] = (l, end, (p1[l, :, nd] + Zl * tau * Y["q1"][l, :, 1, nd]) / 2.0)
            lYZ, eYZ, rYZ = rp_by_edge[(Yf, Zf)]
            lXZ, eXZ, rXZ = rp_by_edge[(X, Zf)]
            lXY, eXY, rXY = rp_by_edge[(X, Yf)]
            # edge set s = a + P b  ->  [b][a] storage; the corner layout is [first][second]
            to_rc = lambda v: v.reshape(P, P).T.ravel()
            from_rc = lambda v: v.reshape(P, P).T.ravel()
            b = -habc.corner_residual(np.zeros(3 * P * P), to_rc(rYZ), to_rc(rXZ), to_rc(rXY), c, M)
            xsol = np.linalg.solve(self._corner_A, b)
            n = P * P
            rm1[lYZ, eYZ] = from_rc(xsol[:n])
            rm1[lXZ, eXZ] = from_rc(xsol[n:2 * n])
            rm1[lXY, eXY] = from_rc(xsol[2 * n:])
        out["rm1"] = rm1
        return out

    # ------------------------------------------------------------ RHS
    def rhs(self, Y, t, cl=None):
        m = self.m
        if cl is None:
            cl = self.closure(Y)
        return {"q3": self._rhs3(Y["q3"], cl["rm3"], t),
                "q2": self._rhs2(Y["q2"], cl["p2"], cl["rm2"]),
                "q1": self._rhs1(Y["q1"], cl["p1"], cl["rm1"])}

    def _rhs3(self, q3, rm3, t):
        m, ref = self.m, self.m.ref3
        K = m.K
        p, u = q3[:, 0], q3[:, 1:4]
        D = (ref.Dr, ref.Ds, ref.Dt)
        Dp = np.stack([p @ Dj.T for Dj in D], axis=1)                 # [K, j, n]
        Du = np.stack([u @ Dj.T for Dj in D], axis=1)                 # [K, j, i, n]
        grad_p = np.einsum("kji,kjn->kin", m.drdx, Dp)
        div_u = np.einsum("kji,kjin->kn", m.drdx, Du)
        rho, c = m.rho[:, None], m.c[:, None]
        rhs = np.zeros_like(q3)
        rhs[:, 0] = -rho * c ** 2 * div_u
        rhs[:, 1:4] = -(1.0 / rho[:, None]) * grad_p
        # traces
        Fm = ref.Fmask                                               # [4, Nfp]
        pm = p[:, Fm]                                                # [K,4,Nfp]
        um = u[:, :, Fm]                                             # [K,3,4,Nfp]
        unm = np.einsum("kfi,kifm->kfm", m.n, um)
        Zm = (m.rho * m.c)[:, None, None] * np.ones_like(pm)
        pstar = np.zeros_like(pm)
        unstar = np.zeros_like(pm)
        inter = m.EToE >= 0
        kk, ff = np.nonzero(inter)
        k2, f2 = m.EToE[kk, ff], m.EToF[kk, ff]
        idx = Fm[f2][np.arange(len(kk))[:, None], m.nbr_perm[kk, ff]]  # neighbour node ids
        pp = p[k2[:, None], idx]
        up = u[k2[:, None], :, idx]                                   # [n, Nfp, 3]
        unp = np.einsum("ni,nmi->nm", m.n[kk, ff], up)
        Zp = (m.rho * m.c)[k2][:, None] * np.ones_like(pp)
        ps_i, un_i = upwind(pm[kk, ff], unm[kk, ff], pp, unp, Zm[kk, ff], Zp)
        pstar[kk, ff], unstar[kk, ff] = ps_i, un_i
        # boundary faces
        bk, bf = m.bface_k, m.bface_f
        dirich = m.bc[m.bface_dom] == BC_DIRICHLET
        rp = (pm[bk, bf] + Zm[bk, bf] * unm[bk, bf]) / 2.0
        ps_b = rp + rm3
        un_b = (rp - rm3) / Zm[bk, bf]
        ps_b[dirich] = 0.0
        un_b[dirich] = unm[bk, bf][dirich] + pm[bk, bf][dirich] / Zm[bk, bf][dirich]
        pstar[bk, bf], unstar[bk, bf] = ps_b, un_b
        dUn = (m.Fscale[..., None] * (unstar - unm)).reshape(K, -1)
        dP = m.Fscale[..., None] * (pstar - pm)                      # [K,4,Nfp]
        rhs[:, 0] -= (rho * c ** 2) * (dUn @ ref.LIFT.T)
        for i in range(3):
            g = (dP * m.n[:, :, i][..., None]).reshape(K, -1)
            rhs[:, 1 + i] -= (1.0 / rho) * (g @ ref.LIFT.T)
        for k, vec, f_peak, t_s, amp in self.sources:
            rhs[k, 0] += amp * ricker_integral(t, f_peak, t_s) * vec
        return rhs

    def _rhs2(self, q2, p2, rm2):
        m, ref = self.m, self.m.ref2
        T, P = m.Ktri, m.P
        if T == 0:
            return np.zeros_like(q2)
        v = q2[:, :, 1:3]                                            # [T,P,2,Np]
        Dp = np.stack([p2 @ ref.Dr.T, p2 @ ref.Ds.T], axis=2)         # [T,P,j,n]
        Dv = np.stack([v @ ref.Dr.T, v @ ref.Ds.T], axis=2)           # [T,P,j,i,n]
        grad_p = np.einsum("tji,tpjn->tpin", m.drdx2, Dp)
        div_v = np.einsum("tji,tpjin->tpn", m.drdx2, Dv)
        rho = m.rho2[:, None, None]
        c = m.c2[:, None, None]
        wa = (1.0 + self.cP)[None, :, None]
        rhs = np.zeros_like(q2)
        rhs[:, :, 0] = -rho * c ** 2 * div_v / wa
        rhs[:, :, 1:3] = -(1.0 / rho[..., None]) * grad_p
        Fm = ref.Fmask                                               # [3, Nfp]
        pm = p2[:, :, Fm]                                            # [T,P,3,Nfp]
        vm = v[:, :, :, Fm]                                          # [T,P,2,3,Nfp]
        vnm = np.einsum("tei,tpiem->tpem", m.n2, vm)
        Z = (m.rho2 * m.c2)[:, None, None, None] * np.ones_like(pm)
        pstar = np.zeros_like(pm)
        vnstar = np.zeros_like(pm)
        tt, ee = np.nonzero(m.EToE2 >= 0)
        t2, e2 = m.EToE2[tt, ee], m.EToF2[tt, ee]
        idx = Fm[e2][np.arange(len(tt))[:, None], m.nbr_perm2[tt, ee]]   # [n, Nfp]
        pp = p2[t2[:, None], :, idx].transpose(0, 2, 1)               # [n,P,Nfp]
        vp = v[t2[:, None], :, :, idx].transpose(0, 2, 3, 1)          # [n,P,2,Nfp]
        vnp = np.einsum("ni,npim->npm", m.n2[tt, ee], vp)
        Zp = (m.rho2 * m.c2)[t2][:, None, None] * np.ones_like(pp)
        a, b = upwind(pm[tt, :, ee], vnm[tt, :, ee], pp, vnp, Z[tt, :, ee], Zp)
        pstar[tt, :, ee], vnstar[tt, :, ee] = a, b
        tb, eb = np.nonzero(m.EToE2 < 0)
        dirich = m.bc[m.tri_edge_dom[tb, eb]] == BC_DIRICHLET
        pmb, vnb, Zb = pm[tb, :, eb], vnm[tb, :, eb], Z[tb, :, eb]
        rmb = rm2[tb, eb]                                            # [n,P,Nfp]
        rp = (pmb + Zb * vnb) / 2.0
        psb = rp + rmb
        vsb = (rp - rmb) / Zb
        psb[dirich] = 0.0
        vsb[dirich] = vnb[dirich] + pmb[dirich] / Zb[dirich]
        pstar[tb, :, eb], vnstar[tb, :, eb] = psb, vsb
        Fs = m.Fscale2[:, None, :, None]
        dVn = (Fs * (vnstar - vnm)).reshape(T, P, -1)
        dP = Fs * (pstar - pm)                                       # [T,P,3,Nfp]
        rhs[:, :, 0] -= (rho * c ** 2 / wa) * (dVn @ ref.LIFT.T)
        for i in range(2):
            g = (dP * m.n2[:, None, :, i, None]).reshape(T, P, -1)
            rhs[:, :, 1 + i] -= (1.0 / rho) * (g @ ref.LIFT.T)
        return rhs

    def _rhs1(self, q1, p1, rm1):
        m, ref = self.m, self.m.ref1
        L, P = m.Klin, m.P
        if L == 0:
            return np.zeros_like(q1)
        w = q1[:, :, 1]                                              # [L,S,Np]
        rx = (1.0 / m.J1)[:, None, None]
        dp = rx * (p1 @ ref.Dr.T)
        dw = rx * (w @ ref.Dr.T)
        rho = m.rho1[:, None, None]
        c = m.c1[:, None, None]
        ca = np.tile(self.cP, P)                                     # s = a + P b
        cb = np.repeat(self.cP, P)
        wab = (1.0 + ca + cb)[None, :, None]
        rhs = np.zeros_like(q1)
        rhs[:, :, 0] = -rho * c ** 2 * dw / wab
        rhs[:, :, 1] = -(1.0 / rho) * dp
        ends = ref.Fmask[:, 0]                                       # node ids of r=-1, r=+1
        tau = np.array([-1.0, 1.0])
        pm = p1[:, :, ends]                                          # [L,S,2]
        wnm = w[:, :, ends] * tau
        Z = (m.rho1 * m.c1)[:, None, None] * np.ones_like(pm)
        pstar = np.zeros_like(pm)
        wnstar = np.zeros_like(pm)
        for l in range(L):
            for e in range(2):
                l2, e2 = m.EToE1[l, e], m.EToF1[l, e]
                if l2 >= 0:
                    pp = p1[l2, :, ends[e2]]
                    wnp = w[l2, :, ends[e2]] * tau[e]
                    Zp = m.rho1[l2] * m.c1[l2]
                    pstar[l, :, e], wnstar[l, :, e] = upwind(pm[l, :, e], wnm[l, :, e], pp, wnp, Z[l, :, e], Zp)
                else:
                    X = m.lin_end_dom[l, e]
                    if m.bc[X] == BC_DIRICHLET:
                        pstar[l, :, e] = 0.0
                        wnstar[l, :, e] = wnm[l, :, e] + pm[l, :, e] / Z[l, :, e]
                    else:
                        rp = (pm[l, :, e] + Z[l, :, e] * wnm[l, :, e]) / 2.0
                        pstar[l, :, e] = rp + rm1[l, e]
                        wnstar[l, :, e] = (rp - rm1[l, e]) / Z[l, :, e]
        Fs = (1.0 / np.abs(m.J1))[:, None, None]
        dWn = Fs * (wnstar - wnm)
        dP = Fs * (pstar - pm) * tau
        rhs[:, :, 0] -= (rho * c ** 2 / wab) * (dWn @ ref.LIFT.T)
        rhs[:, :, 1] -= (1.0 / rho) * (dP @ ref.LIFT.T)
        return rhs

    # ------------------------------------------------------- stepping
    def step(self, Y, res, t, dt):
        """One LSERK4 step; Y and res are updated in place."""
        for s in range(5):
            k = self.rhs(Y, t + LSERK_C[s] * dt)
            for key in Y:
                res[key] *= LSERK_A[s]
                res[key] += dt * k[key]
                Y[key] += LSERK_B[s] * res[key]
        return t + dt

    def run(self, Y, t, dt, nsteps, res=None):
        if res is None:
            res = {k: np.zeros_like(v) for k, v in Y.items()}
        for _ in range(nsteps):
            t = self.step(Y, res, t, dt)
        return Y, res, t

    # ------------------------------------------------------- read-back
    def energy(self, Y):
        """E = sum_k |J_k| [p^T M p / (2 rho c^2) + (rho/2) sum_i u_i^T M u_i]."""
        m, Mref = self.m, self.m.ref3.M
        q3 = Y["q3"]
        quad = np.einsum("kfn,nm,kfm->kf", q3, Mref, q3)
        e = quad[:, 0] / (2.0 * m.rho * m.c ** 2) + 0.5 * m.rho * quad[:, 1:].sum(axis=1)
        return float(np.sum(np.abs(m.J) * e))

    def full_fields(self, Y):
        """Fields with the full auxiliary pressures: q2[:, :, 0] = p_a and
        q1[:, :, 0] = p_ab (the state holds the temporaries p*)."""
        cl = self.closure(Y)
        q2 = Y["q2"].copy()
        q1 = Y["q1"].copy()
        if q2.size:
            q2[:, :, 0] = cl["p2"]
        if q1.size:
            q1[:, :, 0] = cl["p1"]
        return {"q3": Y["q3"].copy(), "q2": q2, "q1": q1}
