"""Pade HABC coefficients and the face / edge / corner algebra (oracle, FP64).

Sec. 2.1: the (2P+1)-th order Pade approximation of sqrt(1+X) is written
f_P(X) = 1 + (2/M) sum_n c_n (1 - (1+c_n)/(1+c_n+X)), c_n = tan^2(n pi/M),
M = 2P+1 (eq. approxRoot2).  Sec. 3.1 rewrites the boundary and compatibility
conditions with characteristic variables; with the reading
r^(+/-) = (p +/- rho c n.u) / 2 (the 1/2 makes eqs. proc:pi00Star,
proc:faceBC and fluxDG1 consistent with each other):

  face   r^-_000 = (1/M) sum_i c_i p*_i00                     (eq. proc:faceBC)
         p_i00   = p*_i00 + (r^-_000 + r^+_000)                (eq. proc:pi00Star)
  edge   the 2P equations proc:edgeBC1-2 for r^-_A (face A sets) and
         r^-_B (face B sets), and p_ab = p*_ab + C_ba Q_A,a + C_ab Q_B,b
         with Q = r^- + r^+ and C_ab = (1+c_a)/(1+c_a+c_b) (eq. proc:pij0Star)
  corner the 3P^2 equations proc:cornerBC1-3 (which carry (C-1), the sign
         that the 0D relation lev3:ijkCorner implies).

The edge and corner systems are solved here directly: each equation is written
as a residual R(x) = x - rhs(x) (affine in the unknowns x), its matrix is
assembled column by column from R, and the system is solved by LU.
"""
import math

import numpy as np


def pade_coefficients(P):
    """c_n = tan^2(n pi / M), n = 1..P, M = 2P+1 (eq. approxRoot2)."""
    M = 2 * P + 1
    return np.array([math.tan(n * math.pi / M) ** 2 for n in range(1, P + 1)]), M


def pade_sqrt(X, P):
    """f_P(X) of eq. approxRoot2."""
    c, M = pade_coefficients(P)
    X = np.asarray(X, float)
    out = np.ones_like(X)
    for cn in c:
        out = out + (2.0 / M) * cn * (1.0 - (1.0 + cn) / (1.0 + cn + X))
    return out


def pade_sqrt_ab(X, P):
    """f_P(X) in the first form, eq. approxRoot1: a_n = sin^2, b_n = cos^2."""
    M = 2 * P + 1
    X = np.asarray(X, float)
    out = np.ones_like(X)
    for n in range(1, P + 1):
        a = math.sin(n * math.pi / M) ** 2
        b = math.cos(n * math.pi / M) ** 2
        out = out + (2.0 / M) * a * X / (1.0 + b * X)
    return out


# ----------------------------------------------------------------------------
# Edge system, eqs. proc:edgeBC1-2 (face A sets a, face B sets b)
# ----------------------------------------------------------------------------
def edge_residual(x, rpA, rpB, ps, c, M):
    """Residual of the 2P edge equations at one node.

    x   = [r^-_A (P), r^-_B (P)]   unknown incoming 2D characteristics
    rpA, rpB                        outgoing 2D characteristics (P each)
    ps[a, b]                        1D temporary fields p*_ab
    """
    P = len(c)
    xA, xB = x[:P], x[P:]
    QA, QB = xA + rpA, xB + rpB
    R = np.zeros(2 * P)
    for a in range(P):
        acc = 0.0
        for b in range(P):
            Cab = (1 + c[a]) / (1 + c[a] + c[b])
            Cba = (1 + c[b]) / (1 + c[a] + c[b])
            acc += c[b] * (ps[a, b] + (Cba - 1.0) * QA[a] + Cab * QB[b])
        R[a] = xA[a] - acc / M
    for b in range(P):
        acc = 0.0
        for a in range(P):
            Cab = (1 + c[a]) / (1 + c[a] + c[b])
            Cba = (1 + c[b]) / (1 + c[a] + c[b])
            acc += c[a] * (ps[a, b] + Cba * QA[a] + (Cab - 1.0) * QB[b])
        R[P + b] = xB[b] - acc / M
    return R


def _affine_matrix(residual, nx, *args):
    """Matrix A and vector b of an affine residual R(x) = A x - b."""
    r0 = residual(np.zeros(nx), *args)
    A = np.zeros((nx, nx))
    for m in range(nx):
        e = np.zeros(nx)
        e[m] = 1.0
        A[:, m] = residual(e, *args) - r0
    return A, -r0


def edge_matrix(c, M):
    P = len(c)
    A, _ = _affine_matrix(edge_residual, 2 * P, np.zeros(P), np.zeros(P), np.zeros((P, P)), c, M)
    return A


def edge_solve(rpA, rpB, ps, c, M):
    """Solve the edge system for many nodes: rpA, rpB [n, P], ps [n, P, P].
    Returns r^-_A, r^-_B [n, P]."""
    P = len(c)
    A = edge_matrix(c, M)
    rhs = np.stack([-edge_residual(np.zeros(2 * P), rpA[i], rpB[i], ps[i], c, M)
                    for i in range(rpA.shape[0])], axis=1) if rpA.shape[0] else np.zeros((2 * P, 0))
    x = np.linalg.solve(A, rhs)
    return x[:P].T, x[P:].T


def edge_pressure(ps, QA, QB, c):
    """p_ab = p*_ab + C_ba Q_A,a + C_ab Q_B,b (eq. proc:pij0Star)."""
    ca = c[:, None]
    cb = c[None, :]
    Cab = (1 + ca) / (1 + ca + cb)
    Cba = (1 + cb) / (1 + ca + cb)
    return ps + Cba * QA[..., :, None] + Cab * QB[..., None, :]


# ----------------------------------------------------------------------------
# Corner system, eqs. proc:cornerBC1-3
# ----------------------------------------------------------------------------
def corner_residual(x, rpYZ, rpXZ, rpXY, c, M):
    """Residual of the 3P^2 corner equations.

    The corner joins the faces X, Y, Z (one per axis).  Unknowns
      x = [r^-_YZ[j,k], r^-_XZ[i,k], r^-_XY[i,j]]  (each P*P, row-major)
    are the incoming 1D characteristics of the edges YZ (fields p_0jk), XZ
    (p_i0k) and XY (p_ij0); rpYZ, rpXZ, rpXY are the outgoing ones (the
    paper's r^{+x}_{0jk}, r^{+y}_{i0k}, r^{+z}_{ij0}) in the same layout.
    """
    P = len(c)
    n = P * P
    xYZ, xXZ, xXY = (x[m * n:(m + 1) * n].reshape(P, P) for m in range(3))
    QYZ = xYZ + rpYZ.reshape(P, P)
    QXZ = xXZ + rpXZ.reshape(P, P)
    QXY = xXY + rpXY.reshape(P, P)
    R = np.zeros(3 * n)
    RYZ, RXZ, RXY = (R[m * n:(m + 1) * n].reshape(P, P) for m in range(3))

    def C3(i, j, k):
        return (1 + c[i]) / (1 + c[i] + c[j] + c[k])

    for j in range(P):
        for k in range(P):
            acc = 0.0
            for i in range(P):
                acc += c[i] * ((C3(i, j, k) - 1.0) * QYZ[j, k] + C3(j, k, i) * QXZ[i, k] + C3(k, i, j) * QXY[i, j])
            RYZ[j, k] = xYZ[j, k] - acc / M
    for i in range(P):
        for k in range(P):
            acc = 0.0
            for j in range(P):
                acc += c[j] * (C3(i, j, k) * QYZ[j, k] + (C3(j, k, i) - 1.0) * QXZ[i, k] + C3(k, i, j) * QXY[i, j])
            RXZ[i, k] = xXZ[i, k] - acc / M
    for i in range(P):
        for j in range(P):
            acc = 0.0
            for k in range(P):
                acc += c[k] * (C3(i, j, k) * QYZ[j, k] + C3(j, k, i) * QXZ[i, k] + (C3(k, i, j) - 1.0) * QXY[i, j])
            RXY[i, j] = xXY[i, j] - acc / M
    return R


def corner_matrix(c, M):
    P = len(c)
    z = np.zeros(P * P)
    A, _ = _affine_matrix(corner_residual, 3 * P * P, z, z, z, c, M)
    return A


def corner_solve(rpYZ, rpXZ, rpXY, c, M):
    """Incoming 1D characteristics at one corner (arguments P*P each)."""
    P = len(c)
    A = corner_matrix(c, M)
    b = -corner_residual(np.zeros(3 * P * P), rpYZ, rpXZ, rpXY, c, M)
    x = np.linalg.solve(A, b)
    n = P * P
    return x[:n], x[n:2 * n], x[2 * n:]
