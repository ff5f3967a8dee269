"""FP64 reference of the learned-closure MLP (test infrastructure only).

The network 6 -> 64 (tanh) -> 64 (tanh) -> 1 and its loss
L = (1/2n) sum_r (MLP(x_r) - y_r)^2, forward pass and analytic gradient
(reverse-mode chain rule written out layer by layer), plus central finite
differences of L.  The parameter vector is W1 [64][6], b1 [64], W2 [64][64],
b2 [64], w3 [64], b3, in that order.  The paper has no learned component;
this checks the project's own training and inference kernels.

ClosureSolver is the FP64 reference of the closure's effect on the solver:
the plain oracle solver whose 3D boundary takes r^- + y at every HABC face
node.  y is the network's correction (`correction`) of the node's features:
the own 3D trace (p, n.u), the full pressures p_1, p_2 of sets 1 and 2
(p*_a + q0), and dp*_1/dt, dp*_2/dt.  Those derivatives are the
face-level right-hand sides of the previous stage's evaluation; they are zero
before the first one.  Only the 3D exterior state changes; q0 and the face,
edge and corner levels keep the plain boundary algebra.  Pins (CPU tests):
- a network with zero output gives the plain solver bit for bit;
- the homogeneous form is of degree one in the fields;
- the features of a uniform state have a closed form.
"""
import numpy as np

NIN, NH = 6, 64
NPARAM = NH * NIN + NH + NH * NH + NH + NH + 1


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    assert w.shape == (NPARAM,)
    o = 0
    W1 = w[o:o + NH * NIN].reshape(NH, NIN); o += NH * NIN
    b1 = w[o:o + NH]; o += NH
    W2 = w[o:o + NH * NH].reshape(NH, NH); o += NH * NH
    b2 = w[o:o + NH]; o += NH
    w3 = w[o:o + NH]; o += NH
    b3 = w[o]
    return W1, b1, W2, b2, w3, b3


def forward(w, X):
    """MLP(X) for rows X [n][6] (FP64)."""
    W1, b1, W2, b2, w3, b3 = unpack(w)
    h1 = np.tanh(np.asarray(X, np.float64) @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ w3 + b3


def loss_grad(w, X, Y):
    """(L, dL/dw) with L = mean((MLP(X) - Y)^2) / 2, by the chain rule."""
    W1, b1, W2, b2, w3, b3 = unpack(w)
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    n = X.shape[0]
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    y = h2 @ w3 + b3
    e = y - Y
    L = 0.5 * np.mean(e * e)
    dy = e / n                              # dL/dy
    dw3 = h2.T @ dy
    db3 = dy.sum()
    dz2 = np.outer(dy, w3) * (1.0 - h2 * h2)
    dW2 = dz2.T @ h1
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (1.0 - h1 * h1)
    dW1 = dz1.T @ X
    db1 = dz1.sum(axis=0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, [db3]])
    return L, g


def loss(w, X, Y):
    e = forward(w, X) - np.asarray(Y, np.float64)
    return 0.5 * np.mean(e * e)


def finite_difference_grad(w, X, Y, idx, h=1e-6):
    """Central differences of the loss for the parameters idx."""
    w = np.asarray(w, np.float64)
    out = np.empty(len(idx))
    for k, p in enumerate(idx):
        wp, wm = w.copy(), w.copy()
        wp[p] += h
        wm[p] -= h
        out[k] = (loss(wp, X, Y) - loss(wm, X, Y)) / (2 * h)
    return out


def correction(w, X, scales=None):
    """The closure's correction per feature row (FP64).  Plain form:
    MLP(x) - MLP(0), so that no fields give no correction.  Homogeneous form
    (scales = 1/sigma_1..6 of the features, then sigma_y): with x~ = x / sigma,
    y = sigma_y |x~| MLP(x~ / |x~|), and 0 at x~ = 0 -- of degree one in the
    fields, as the linear wave equation asks of a boundary closure."""
    X = np.asarray(X, np.float64)
    if scales is None:
        return forward(w, X) - forward(w, np.zeros((1, NIN)))[0]
    scales = np.asarray(scales, np.float64)
    Xt = X * scales[:NIN]
    s = np.linalg.norm(Xt, axis=1)
    y = np.zeros(len(X))
    nz = s > 0.0
    y[nz] = scales[NIN] * s[nz] * forward(w, Xt[nz] / s[nz, None])
    return y


class ClosureSolver:
    """The oracle solver (oracle.solver.Solver, P >= 1) with the learned
    closure on its HABC faces; see the module docstring."""

    def __init__(self, solver, w, scales=None):
        self.s = solver
        self.w = np.asarray(w, np.float64)
        self.scales = None if scales is None else np.asarray(scales, np.float64)
        m = solver.m
        self.dps = np.zeros((m.Ktri, 2, m.ref2.Np))   # dp*_a/dt, a = 1, 2, of the last evaluation

    def features(self, Y, cl):
        """Feature rows [K^tri * Np2][6] (triangle-major, the triangle's own
        node order) from the fields Y and their boundary algebra cl."""
        m = self.s.m
        k, f = m.tri_k, m.tri_f
        Fm = m.ref3.Fmask[f]                                          # [T, Nfp]
        q3 = Y["q3"]
        p = q3[k[:, None], 0, Fm]
        un = np.einsum("ti,tin->tn", m.n[k, f], q3[k[:, None], 1:4, Fm].transpose(0, 2, 1))
        zero = np.zeros_like(p)
        p1 = cl["p2"][:, 0] if m.P >= 1 else zero
        p2 = cl["p2"][:, 1] if m.P >= 2 else zero
        X = np.stack([p, un, p1, p2, self.dps[:, 0], self.dps[:, 1]], axis=-1)
        return X.reshape(-1, NIN)

    def rhs(self, Y, t):
        m = self.s.m
        cl = self.s.closure(Y)
        y = correction(self.w, self.features(Y, cl), self.scales).reshape(m.Ktri, m.ref2.Np)
        cl["rm3"][m.tri_bface] += y
        k = self.s.rhs(Y, t, cl)
        a = min(m.P, 2)
        self.dps = np.zeros_like(self.dps)
        self.dps[:, :a] = k["q2"][:, :a, 0, :]
        return k

    def step(self, Y, res, t, dt):
        """One LSERK4 step (Appendix A); Y and res are updated in place."""
        from .solver import LSERK_A, LSERK_B, LSERK_C
        for st in range(5):
            k = self.rhs(Y, t + LSERK_C[st] * dt)
            for key in Y:
                res[key] *= LSERK_A[st]
                res[key] += dt * k[key]
                Y[key] += LSERK_B[st] * res[key]
        return t + dt

    def run(self, Y, t, dt, nsteps, res=None):
        if res is None:
            res = {k: np.zeros_like(v) for k, v in Y.items()}
        for _ in range(nsteps):
            t = self.step(Y, res, t, dt)
        return Y, res, t
