"""Pins for the oracle's learned-guess pieces (not in the paper; built on the
Lagrange weights of Sec. 4.2.1 and the partition of unity of App. B):
backpropagation against central differences, the rational (pole) weights
against their defining exactness property and their Lagrange limit, the
closed-form span-optimal weights, and the residual identity that defines the
loss, checked with exact dense solves."""
import numpy as np

import oracle
import synth

F = 20


def _nodes_targets(N, seed):
    rng = np.random.default_rng(seed)
    sig = synth.shift_set(12, 1e-5, 2.0)
    S = np.array([np.concatenate([[sig[8 + rng.integers(4)]], sig[:8]]) for _ in range(N)])
    return S


def _data(N=7, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((N, F))
    A = rng.standard_normal((N, 8, 8))
    H = np.einsum("nij,nkj->nik", A, A) + 0.1 * np.eye(8)
    n = sum(int(np.prod(s)) for s in oracle.mlp_sizes(F))
    theta = 0.3 * rng.standard_normal(n)
    theta[F:2 * F] = 0.5 + rng.random(F)          # isd > 0
    return theta, X, _nodes_targets(N, seed), H


def test_backprop_matches_central_differences():
    theta, X, S, H = _data()
    loss, g = oracle.mlp_loss_grad(theta, X, S, H, floor=1e-3)
    assert np.all(g[:2 * F] == 0)                  # input statistics are not trained
    rng = np.random.default_rng(1)
    for idx in rng.choice(np.arange(2 * F, len(theta)), 40, replace=False):
        e = np.zeros_like(theta)
        h = 1e-6
        e[idx] = h
        fd = (oracle.mlp_loss_grad(theta + e, X, S, H, 1e-3)[0] - oracle.mlp_loss_grad(theta - e, X, S, H, 1e-3)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_pole_weights_reproduce_rational_functions():
    """w_j = l_j(t) prod_k (p_k + s_j)/(p_k + t) reproduce f(s) = P(s) / prod_k (p_k + s)
    for every polynomial P of degree <= 7 (8 nodes), hence sum to 1 (P = prod_k (p_k + s)),
    and tend to the Lagrange weights of Sec. 4.2.1 as the poles grow."""
    rng = np.random.default_rng(3)
    S = _nodes_targets(5, 3)
    for n in range(len(S)):
        t, nodes = S[n, 0], S[n, 1:]
        poles = np.exp(rng.uniform(np.log(1e-3), np.log(1.0), 2))
        w = oracle.pole_weights(S[n:n + 1], poles[None])[0]
        assert abs(w.sum() - 1.0) < 1e-12 * np.abs(w).sum()
        for _ in range(3):
            c = rng.standard_normal(8)
            f = lambda s: np.polyval(c, s) / np.prod(poles + s)
            assert abs(sum(wj * f(sj) for wj, sj in zip(w, nodes)) - f(t)) < 1e-9 * max(1.0, abs(f(t)))
        wl = oracle.pole_weights(S[n:n + 1], np.array([[1e12, 1e12]]))[0]
        assert np.allclose(wl, oracle.lagrange_weights(nodes, t), rtol=1e-9, atol=1e-12)


def test_projection_and_span_optimum():
    theta, X, S, H = _data()
    w = oracle.mlp_forward(theta, X, S)
    assert np.allclose(w.sum(axis=1), 1.0, atol=1e-12)
    for n in range(len(H)):
        ws = oracle.span_optimal_weights(H[n])
        assert abs(ws.sum() - 1) < 1e-12
        # optimality: H w* is parallel to 1 (Lagrange condition), and w* beats the network's w
        hw = H[n] @ ws
        assert np.max(np.abs(hw - hw.mean())) < 1e-10 * np.abs(hw).max()
        assert ws @ H[n] @ ws <= w[n] @ H[n] @ w[n] + 1e-12


def _dense_problem():
    dims = (4, 2, 2, 2)
    U = synth.random_su3_field(dims, 0.5, 3)
    act = oracle.action(dims, 0.16, 0.1, 0.11)
    b = synth.gaussian_rhs(dims, 4)[0]
    Vh = 16
    Q2 = oracle.dense(lambda v: oracle.qhat2(act, U, v.reshape(Vh, 2, 4, 3)), Vh * 24)
    return Q2, b.ravel()


def test_loss_is_the_guess_residual_for_exact_solutions(oracle_lib):
    """With exact x_j (dense LU on a 4x2^3 lattice) and sum w = 1,
    |b - (Qhat^2 + sigma_t) sum_j w_j x_j|^2 / |b|^2 = w^T H w.  The LU
    solutions carry residuals r_j ~ 1e-14 |b| that enter as sum_j w_j r_j, i.e.
    ~1e-8 relative to a guess residual of ~4e-6: tolerance 1e-6 relative."""
    Q2, b = _dense_problem()
    sig = synth.shift_set(10, 1e-4, 1.0)
    nodes, tgt = sig[:8], sig[8]
    xs = [np.linalg.solve(Q2 + s * np.eye(Q2.shape[0]), b) for s in nodes]
    H = oracle.guess_quadratic_form(nodes, tgt, xs, np.vdot(b, b).real)
    rng = np.random.default_rng(2)
    S = np.concatenate([[tgt], nodes])[None]
    for w in (oracle.lagrange_weights(nodes, tgt), rng.standard_normal(8),
              oracle.pole_weights(S, np.array([[0.05, 0.3]]))[0]):
        w = w + (1 - w.sum()) / 8
        guess = sum(wi * xi for wi, xi in zip(w, xs))
        r = b - (Q2 @ guess + tgt * guess)
        assert abs(np.vdot(r, r).real / np.vdot(b, b).real - w @ H @ w) < 1e-6 * (w @ H @ w)


def test_poles_at_the_spectrum_give_the_exact_solution(oracle_lib):
    """If b has components on two eigenvectors of Qhat^2 only, x(s) = sum_k c_k v_k/(lambda_k + s)
    and prod_k (lambda_k + s) x(s) is linear in s: the pole weights with p_k = lambda_k
    reproduce x(sigma_t) exactly, where Lagrange weights leave a residual."""
    Q2, _ = _dense_problem()
    lam, V = np.linalg.eigh(Q2)
    b = V[:, 0] * (1 + 0.5j) + V[:, 5] * (0.3 - 1j)
    sig = synth.shift_set(12, 1e-5, 2.0)
    nodes, tgt = sig[:8], sig[11]
    xs = [np.linalg.solve(Q2 + s * np.eye(Q2.shape[0]), b) for s in nodes]
    S = np.concatenate([[tgt], nodes])[None]
    w = oracle.pole_weights(S, np.array([[lam[0], lam[5]]]))[0]
    wl = oracle.lagrange_weights(nodes, tgt)
    xt = np.linalg.solve(Q2 + tgt * np.eye(Q2.shape[0]), b)
    err = np.linalg.norm(sum(wi * xi for wi, xi in zip(w, xs)) - xt) / np.linalg.norm(xt)
    err_l = np.linalg.norm(sum(wi * xi for wi, xi in zip(wl, xs)) - xt) / np.linalg.norm(xt)
    assert err < 1e-11 and err_l > 1e3 * err, (err, err_l)
