"""Orthonormal Jacobi polynomials and Gauss-type points (oracle, FP64).

Textbook material used by the nodal DG construction that Sec. 3.2 of the
paper cites: P_n^{(a,b)} orthonormal on [-1,1] with weight (1-x)^a (1+x)^b,
Gauss-Jacobi points from the eigenvalues of the Jacobi matrix (Golub-Welsch),
and Gauss-Lobatto-Legendre points (the nodes of the reference line, which
must coincide with the edge nodes of the tetrahedron, Sec. 3.2).
"""
import math

import numpy as np


def _h0(a, b):
    """Squared norm of the constant 1 under the weight (1-x)^a (1+x)^b."""
    return 2.0 ** (a + b + 1) * math.gamma(a + 1) * math.gamma(b + 1) / math.gamma(a + b + 2)


def _recurrence(a, b, n):
    """Diagonal alpha_i and off-diagonal beta_i (i = 0..n-1) of the symmetric
    three-term recurrence x p_i = beta_i p_{i+1} + alpha_i p_i + beta_{i-1} p_{i-1}
    for the orthonormal Jacobi polynomials."""
    alpha = np.zeros(n)
    beta = np.zeros(n)
    for i in range(n):
        s = 2 * i + a + b
        if i == 0:
            alpha[i] = (b - a) / (a + b + 2.0)
        else:
            alpha[i] = (b * b - a * a) / (s * (s + 2.0))
        num = 4.0 * (i + 1) * (i + 1 + a + b) * (i + 1 + a) * (i + 1 + b)
        den = (s + 2.0) ** 2 * (s + 1.0) * (s + 3.0)
        beta[i] = math.sqrt(num / den)
    return alpha, beta


def jacobi_p(x, a, b, n):
    """Orthonormal Jacobi polynomial P_n^{(a,b)} evaluated at the points x."""
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.zeros_like(x)
    p = np.full_like(x, 1.0 / math.sqrt(_h0(a, b)))
    if n == 0:
        return p
    alpha, beta = _recurrence(a, b, n)
    for i in range(n):
        p_next = ((x - alpha[i]) * p - (beta[i - 1] * p_prev if i > 0 else 0.0)) / beta[i]
        p_prev, p = p, p_next
    return p


def grad_jacobi_p(x, a, b, n):
    """d/dx of the orthonormal P_n^{(a,b)}: sqrt(n(n+a+b+1)) P_{n-1}^{(a+1,b+1)}."""
    x = np.asarray(x, dtype=np.float64)
    if n == 0:
        return np.zeros_like(x)
    return math.sqrt(n * (n + a + b + 1.0)) * jacobi_p(x, a + 1, b + 1, n - 1)


def gauss_jacobi(a, b, n):
    """n-point Gauss-Jacobi rule (points ascending, weights) by Golub-Welsch."""
    if n == 1:
        return np.array([(b - a) / (a + b + 2.0)]), np.array([_h0(a, b)])
    alpha, beta = _recurrence(a, b, n)
    T = np.diag(alpha) + np.diag(beta[:-1], 1) + np.diag(beta[:-1], -1)
    x, vec = np.linalg.eigh(T)
    w = _h0(a, b) * vec[0, :] ** 2
    return x, w


def gll_points(n):
    """The n+1 Gauss-Lobatto-Legendre points on [-1,1], ascending."""
    if n == 1:
        return np.array([-1.0, 1.0])
    inner, _ = gauss_jacobi(1.0, 1.0, n - 1)
    return np.concatenate(([-1.0], inner, [1.0]))
