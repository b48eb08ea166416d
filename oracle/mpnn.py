"""CPU oracle of the learned preconditioner network -- TEST INFRASTRUCTURE ONLY.

Plain numpy, FP64, written for reading rather than speed.  Only the test
suite and the bench's CPU leg may import it; the CUDA library shares no code
with it.

The network (a message-passing network over the GFD stencil graph, the
learned part of the solver; the paper itself has no learned component):

  * System.  Ahat = A D^-1, the Jacobi-scaled GFD Poisson matrix (Section
    3.2 step 2; D = diag(A)), so Ahat_jj = 1.  E_j = {i != j : Ahat_ji != 0}
    are node j's stencil neighbours (boundary rows have none).
  * Aggregation.  W = |Ahat_off| + |Ahat_off|^T (the stencil graph made
    symmetric: a node also hears the nodes whose stencils use it), P = W
    normalised by its row sums (P_ji = W_ji / sum_i' W_ji'), 0 rows for
    isolated nodes.
  * Node features F (16): 1, boundary flag, row sums over E_j of |Ahat_ji|,
    Ahat_ji and Ahat_ji^2, column sums over i != j of Ahat_ij^2 and |Ahat_ij|
    (the WLS weights other stencils give node j) -- these five through
    sign(f) log(1 + |f|) -- then with P: mean offset
    sum P_ji d_ji (3, d_ji = (x_i - x_j)/h_j, h_j the cell edge),
    sum P_ji |d_ji|^2, mean level offset sum P_ji (l_i - l_j), b_j / max|b|,
    sum P_ji b_i / max|b|, and the W-degree / 64.
  * Layers l = 0, 1, 2: H_{l+1} = relu([H_l | P H_l] W_l + b_l), H_0 = F,
    width 64 (W_0: 32 x 64, W_1, W_2: 128 x 64).
  * Head: t = H_3 W_o + b_o (64 x 2); s = exp(alpha tanh t_0), alpha = ln 8
    (s in [1/8, 8]), on interior nodes, s = 1 on boundary nodes (their rows
    are identity rows), the learned column scaling of the preconditioner
    (Ahat S replaces Ahat); gamma = exp(tanh t_1), the initial guess
    u0 = gamma * b of Ahat u = b.
  * Loss L = Lp + Lg.  Lp = (1/n_int) sum over interior columns of
    ||e_j - Ahat S e_j||^2 (the approximate-inverse objective for a diagonal
    right preconditioner; column j contributes 1 - 2 s_j + s_j^2 c_j with
    c_j = sum_i Ahat_ij^2), Lg = ||b - Ahat u0||^2 / ||b||^2 (the relative
    initial residual of the proposed guess).

Parameters travel as one flat FP32/FP64 vector in the order
W0 (32x64, row-major), b0 (64), W1 (128x64), b1, W2 (128x64), b2,
Wo (64x2), bo (2).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

NF = 16
WIDTH = 64
ALPHA = float(np.log(8.0))
SHAPES = [("W0", (2 * NF, WIDTH)), ("b0", (WIDTH,)), ("W1", (2 * WIDTH, WIDTH)), ("b1", (WIDTH,)),
          ("W2", (2 * WIDTH, WIDTH)), ("b2", (WIDTH,)), ("Wo", (WIDTH, 2)), ("bo", (2,))]
N_PARAMS = int(sum(np.prod(s) for _, s in SHAPES))


def unflatten(theta):
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def flatten(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def scaled_matrix(rp, col, val):
    """Ahat = A D^-1 as a scipy CSR matrix (D = diag(A))."""
    n = len(rp) - 1
    A = sp.csr_matrix((val, col, rp), shape=(n, n))
    d = A.diagonal()
    return (A @ sp.diags(1.0 / d)).tocsr()


def features(Ah, xyz, level, kind, b, ext):
    """Node features F (n x 16) and the aggregation matrix P."""
    n = Ah.shape[0]
    off = (Ah - sp.diags(Ah.diagonal())).tocsr()
    off.eliminate_zeros()
    absv = abs(off)
    W = (absv + absv.T).tocsr()
    S = np.asarray(W.sum(axis=1)).ravel()
    inv = np.where(S > 0, 1.0 / np.where(S > 0, S, 1.0), 0.0)
    P = (sp.diags(inv) @ W).tocsr()
    lvl = level.astype(np.float64)
    h = ext * 2.0 ** (-lvl)
    F = np.zeros((n, NF))
    F[:, 0] = 1.0
    F[:, 1] = kind
    F[:, 2] = np.asarray(absv.sum(axis=1)).ravel()
    F[:, 3] = np.asarray(off.sum(axis=1)).ravel()
    F[:, 4] = np.asarray(off.multiply(off).sum(axis=1)).ravel()
    F[:, 5] = np.asarray(off.multiply(off).sum(axis=0)).ravel()
    F[:, 6] = np.asarray(absv.sum(axis=0)).ravel()
    rows = np.repeat(np.arange(n), np.diff(P.indptr))
    d = (xyz[P.indices] - xyz[rows]) / h[rows, None]
    for a in range(3):
        F[:, 7 + a] = np.bincount(rows, weights=P.data * d[:, a], minlength=n)
    F[:, 10] = np.bincount(rows, weights=P.data * (d ** 2).sum(1), minlength=n)
    F[:, 11] = P @ lvl - (P @ np.ones(n)) * lvl
    B = np.abs(b).max()
    if B > 0:
        F[:, 12] = b / B
        F[:, 13] = (P @ b) / B
    F[:, 14] = np.diff(W.indptr) / 64.0
    # the sums of WLS weights are heavy-tailed: signed log1p keeps them O(1)
    F[:, 2:7] = np.sign(F[:, 2:7]) * np.log1p(np.abs(F[:, 2:7]))
    return F, P


def forward(theta, F, P):
    """Forward pass; F[:, 1] is the boundary flag."""
    p = unflatten(theta)
    H = [F]
    X = []
    for l in range(3):
        x = np.concatenate([H[l], P @ H[l]], axis=1)
        X.append(x)
        H.append(np.maximum(x @ p["W%d" % l] + p["b%d" % l], 0.0))
    t = H[3] @ p["Wo"] + p["bo"]
    interior = F[:, 1] == 0.0
    s = np.where(interior, np.exp(ALPHA * np.tanh(t[:, 0])), 1.0)
    gamma = np.exp(np.tanh(t[:, 1]))
    return dict(H=H, X=X, t=t, s=s, gamma=gamma, interior=interior)


def loss(Ah, b, s, gamma, interior):
    c = np.asarray(Ah.multiply(Ah).sum(axis=0)).ravel()   # 1 + the raw column feature
    Lp = float(np.sum((1.0 - 2.0 * s + s * s * c)[interior])) / max(1, int(interior.sum()))
    u0 = gamma * b
    r = b - Ah @ u0
    Lg = float(r @ r) / float(b @ b)
    return Lp + Lg, Lp, Lg, c, r


def loss_and_grad(theta, Ah, F, P, b):
    """(L, Lp, Lg), flat gradient dL/dtheta, and the forward record."""
    p = unflatten(theta)
    fw = forward(theta, F, P)
    interior = fw["interior"]
    L, Lp, Lg, c, r = loss(Ah, b, fw["s"], fw["gamma"], interior)
    s, gamma, t = fw["s"], fw["gamma"], fw["t"]
    ds = np.where(interior, (2.0 / max(1, int(interior.sum()))) * (s * c - 1.0), 0.0)
    dgamma = -2.0 * b * (Ah.T @ r) / float(b @ b)
    dt = np.zeros_like(t)
    th0, th1 = np.tanh(t[:, 0]), np.tanh(t[:, 1])
    dt[:, 0] = ds * s * ALPHA * (1.0 - th0 * th0)
    dt[:, 1] = dgamma * gamma * (1.0 - th1 * th1)
    g = {"Wo": fw["H"][3].T @ dt, "bo": dt.sum(0)}
    dH = dt @ p["Wo"].T
    for l in (2, 1, 0):
        dZ = dH * (fw["H"][l + 1] > 0)
        g["W%d" % l] = fw["X"][l].T @ dZ
        g["b%d" % l] = dZ.sum(0)
        dX = dZ @ p["W%d" % l].T
        k = dX.shape[1] // 2
        dH = dX[:, :k] + P.T @ dX[:, k:]
    return (L, Lp, Lg), flatten(g), fw


def init_params(seed=0):
    """Glorot-uniform layers from numpy's generator; a zero head, so that the
    untrained network is exactly Jacobi (s = 1) with the guess u0 = b."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in SHAPES:
        if name.startswith("W") and name != "Wo":
            lim = np.sqrt(6.0 / (shape[0] + shape[1]))
            p[name] = rng.uniform(-lim, lim, size=shape)
        else:
            p[name] = np.zeros(shape)
    return flatten(p)
