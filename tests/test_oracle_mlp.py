"""Pins for the oracle's learned-guess pieces (not in the paper; built on the
partition of unity of App. B): backpropagation against central differences,
the projection sum w = 1, the closed-form span-optimal weights, and the
residual identity that defines the loss, checked with exact dense solves."""
import numpy as np

import oracle
import synth


def _data(N=7, F=20, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((N, F))
    A = rng.standard_normal((N, 8, 8))
    H = np.einsum("nij,nkj->nik", A, A) + 0.1 * np.eye(8)
    n = sum(int(np.prod(s)) for s in oracle.mlp_sizes(F))
    theta = 0.3 * rng.standard_normal(n)
    return theta, X, H


def test_backprop_matches_central_differences():
    theta, X, H = _data()
    loss, g = oracle.mlp_loss_grad(theta, X, H)
    rng = np.random.default_rng(1)
    for idx in rng.choice(len(theta), 40, replace=False):
        e = np.zeros_like(theta)
        h = 1e-6
        e[idx] = h
        fd = (oracle.mlp_loss_grad(theta + e, X, H)[0] - oracle.mlp_loss_grad(theta - e, X, H)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_projection_and_span_optimum():
    theta, X, H = _data()
    w = oracle.mlp_forward(theta, X)
    assert np.allclose(w.sum(axis=1), 1.0, atol=1e-14)
    for n in range(len(H)):
        ws = oracle.span_optimal_weights(H[n])
        assert abs(ws.sum() - 1) < 1e-12
        # optimality: H w* is parallel to 1 (Lagrange condition), and w* beats the network's w
        hw = H[n] @ ws
        assert np.max(np.abs(hw - hw.mean())) < 1e-10 * np.abs(hw).max()
        assert ws @ H[n] @ ws <= w[n] @ H[n] @ w[n] + 1e-12


def test_loss_is_the_guess_residual_for_exact_solutions(oracle_lib):
    """With exact x_j (dense LU on a 4x2^3 lattice) and sum w = 1,
    |b - (Qhat^2 + sigma_t) sum_j w_j x_j|^2 / |b|^2 = w^T H w.  The LU
    solutions carry residuals r_j ~ 1e-14 |b| that enter as sum_j w_j r_j, i.e.
    ~1e-8 relative to a guess residual of ~4e-6: tolerance 1e-6 relative."""
    dims = (4, 2, 2, 2)
    U = synth.random_su3_field(dims, 0.5, 3)
    act = oracle.action(dims, 0.16, 0.1, 0.11)
    b = synth.gaussian_rhs(dims, 4)[0]
    Vh = 16
    Q2 = oracle.dense(lambda v: oracle.qhat2(act, U, v.reshape(Vh, 2, 4, 3)), Vh * 24)
    sig = synth.shift_set(10, 1e-4, 1.0)
    nodes, tgt = sig[:8], sig[8]
    xs = [np.linalg.solve(Q2 + s * np.eye(Q2.shape[0]), b.ravel()) for s in nodes]
    H = oracle.guess_quadratic_form(nodes, tgt, xs, np.vdot(b, b).real)
    rng = np.random.default_rng(2)
    for w in (oracle.lagrange_weights(nodes, tgt), rng.standard_normal(8)):
        w = w + (1 - w.sum()) / 8
        guess = sum(wi * xi for wi, xi in zip(w, xs))
        r = b.ravel() - (Q2 @ guess + tgt * guess)
        assert abs(np.vdot(r, r).real / np.vdot(b, b).real - w @ H @ w) < 1e-6 * (w @ H @ w)
