"""FP64 reference of the learned-closure MLP (test infrastructure only).

The network 6 -> 64 (tanh) -> 64 (tanh) -> 1 and its loss
L = (1/2n) sum_r (MLP(x_r) - y_r)^2, forward pass and analytic gradient
(reverse-mode chain rule written out layer by layer), plus central finite
differences of L.  The parameter vector is W1 [64][6], b1 [64], W2 [64][64],
b2 [64], w3 [64], b3, in that order.  The paper has no learned component;
this checks the project's own training and inference kernels.  Parity of
the closure's effect on the boundary is unpinned (no analytic target).
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
