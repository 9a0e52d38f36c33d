"""Learned initial guesses: data generation, training and evaluation driver.

Host orchestration only: every arithmetic step runs in libtmnd (multi-shift CG
with its scalar history, Gram matrices, network features, forward/backward
kernels, Adam, BF16 inference, linear combinations).  The guess for a target
shift sigma_t is sum_j w_j x_j over the solutions of the 8 solved shifts just
above it, with w from Lagrange interpolation (Sec. 4.2.1) or from the network,
whose two predicted poles p_k give
    w_j = l_j(sigma_t) prod_k (p_k + sigma_j) / (p_k + sigma_t);
the network is trained on
    loss = mean log(w^T H w + floor),  H = Re(D G D),  G_jk = <x_j, x_k>/|b|^2,
    D = diag(sigma_t - sigma_j),
the squared relative residual of the guess when the x_j are exact (App. B);
floor = rho^2 of the solves stands for the residuals the x_j still carry.
"""
from __future__ import annotations

import numpy as np

import paper_1805_09584_gb300 as tm

NODES = 8


def solve_nodes(g, b_dev, sigma, rho=1e-10, maxiter=20000, prec=None):
    """Solutions of every shift, the way the hybrid solve produces them: one
    multi-shift CG on the 8 largest shifts (its scalar history and iteration count
    are the network's features) and one on the rest.  Returns (solutions of all
    shifts, info of the first solve, its scalar history).  prec = TMND_S16 gives
    the history of the sloppy solve, as the mixed hybrid solve sees it."""
    import torch
    pr = tm.TMND_F64 if prec is None else prec
    xs = [g.spinor() for _ in sigma]
    hist = np.zeros(2 * min(maxiter, 4096), np.float64)
    info = tm.mms_cg_solve(g.handle, b_dev, 1, sigma[:NODES], xs[:NODES], rho=rho, maxiter=maxiter, ab_hist=hist,
                           prec=pr)
    if len(sigma) > NODES:
        tm.mms_cg_solve(g.handle, b_dev, 1, sigma[NODES:], xs[NODES:], rho=rho, maxiter=maxiter, prec=pr)
    torch.cuda.synchronize()
    return xs, info, hist


def samples(g, b_dev, sigma, xs, info, hist):
    """Network inputs X [T, 20] (float32), shifts S [T, 9] = (sigma_t, nodes) and loss
    matrices H [T, 8, 8] (float64) for the targets sigma[8:], each over the 8 shifts
    just above it (the nearest solved ones, as the Lagrange guess of Sec. 4.2.1 uses);
    the Lanczos features come from the history of the solve with base shift sigma[7]."""
    sigma = np.asarray(sigma, np.float64)
    bb = float(tm.tmnd_gram(g.handle, [b_dev])[0, 0].real)
    feats, Ss, Hs = [], [], []
    for q, t in enumerate(sigma[NODES:]):
        nodes = sigma[q:q + NODES]
        G = tm.tmnd_gram(g.handle, xs[q:q + NODES])
        feats.append(tm.tmnd_mlp_features(nodes, float(t), hist, info["iters"], float(sigma[NODES - 1])))
        Ss.append(np.concatenate([[float(t)], nodes]))
        Hs.append(tm.tmnd_guess_quadratic_form(G, nodes, float(t), bb))
    return np.stack(feats), np.stack(Ss), np.stack(Hs)


def lagrange_weights(nodes, target):
    """Lagrange weights of Sec. 4.2.1 (the library's host function, as lagrange_guess applies them)."""
    return tm.tmnd_lagrange_weights(nodes, target)[0]


def _dev(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype)).cuda()


def train(X, S, H, epochs=600, lr=3e-3, seed=0, floor=1e-20):
    """Train a fresh network on (X [N,20], S [N,9], H [N,8,8]) with full-batch Adam after
    fitting the input standardisation; returns (handle, per-epoch losses)."""
    m = tm.tmnd_mlp_create(X.shape[1], seed)
    Xd, Sd, Hd = _dev(X, np.float32), _dev(S, np.float64), _dev(H, np.float64)
    N = X.shape[0]
    tm.tmnd_mlp_fit_inputs(m, Xd, N)
    losses = [tm.tmnd_mlp_train_step(m, Xd, Sd, Hd, N, lr, floor) for _ in range(epochs)]
    return m, losses


def predict(m, X, S):
    """FP64 weights [N, 8] (BF16 network inference)."""
    import torch
    W = torch.empty((X.shape[0], NODES), dtype=torch.float64, device="cuda")
    tm.tmnd_mlp_predict(m, _dev(X, np.float32), _dev(S, np.float64), X.shape[0], W)
    return W.cpu().numpy()


def iterations_from_guess(g, b_dev, xs, w, sigma_t, rho=1e-10):
    """CG iterations to reach |b - (Qhat^2 + sigma_t) x| <= rho |b| from the guess
    sum_j w_j x_j: solve the defect system (Qhat^2 + sigma_t) e = r to
    rho |b| / |r| with the multi-shift CG on one shift."""
    import torch
    guess = g.spinor()
    tm.tmnd_lincomb(g.handle, np.asarray(w, np.float64), xs, guess)
    y = g.spinor()
    tm.tm_nd_apply(g.handle, y, guess, tm.OP_QHAT2, float(sigma_t))
    r = g.spinor()
    tm.tmnd_lincomb(g.handle, np.array([1.0, -1.0]), [b_dev, y], r)
    bb = float(tm.tmnd_gram(g.handle, [b_dev])[0, 0].real)
    rr = float(tm.tmnd_gram(g.handle, [r])[0, 0].real)
    rel = np.sqrt(rr / bb)
    if rel <= rho:
        return 0, rel
    e = g.spinor()
    info = tm.mms_cg_solve(g.handle, r, 1, [float(sigma_t)], [e], rho=min(0.99, rho / rel))
    torch.cuda.synchronize()
    return info["iters"], rel
