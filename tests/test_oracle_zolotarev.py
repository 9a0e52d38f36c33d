"""Pins for the oracle's Zolotarev rational approximation (Sec. 4.1, Eqs.
"rational", "deviation", "zolotarev_shifts", "ratapp"): the closed-form maximal
deviation equals the maximum of |1 - sqrt(y) R(y)| over eps < y < 1 (the
definition), the error equioscillates (2n + 2 alternating extrema of size delta:
Chebyshev's alternation theorem for the optimal approximation), the
partial-fraction form of Eq. "ratapp" equals the product form, and the whole
chain reproduces the exact inverse square root of a dense Qhat^2 within delta."""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("n,eps", [(3, 1e-1), (6, 1e-3), (10, 65e-6 / 4.7), (14, 1e-6)])
def test_deviation_closed_form_and_equioscillation(n, eps):
    a, c, q, delta = oracle.zolotarev(n, eps)
    assert np.all(np.diff(c) < 0) and np.all(c > 0)
    y = np.geomspace(eps, 1.0, 400001)
    err = 1.0 - np.sqrt(y) * oracle.zolotarev_eval(a, c, y)
    assert abs(np.abs(err).max() - delta) <= 1e-4 * delta
    # alternation: local extrema of err of size ~delta with alternating signs, 2n + 2 of them (ends included)
    ext = [0] + [i for i in range(1, len(y) - 1) if (err[i] - err[i - 1]) * (err[i + 1] - err[i]) < 0] + [len(y) - 1]
    vals = err[ext]
    assert len(ext) == 2 * n + 2, len(ext)
    assert np.all(np.abs(np.abs(vals) - delta) <= 1e-3 * delta)
    assert np.all(np.sign(vals[1:]) == -np.sign(vals[:-1]))


@pytest.mark.parametrize("n,eps", [(4, 1e-2), (10, 1e-5)])
def test_partial_fractions_equal_product_form(n, eps):
    a, c, q, _ = oracle.zolotarev(n, eps)
    y = np.random.default_rng(1).uniform(eps, 1.0, 1000)
    pf = a * (1.0 + sum(q[i] / (y + c[2 * i + 1]) for i in range(n)))
    assert np.max(np.abs(pf / oracle.zolotarev_eval(a, c, y) - 1.0)) < 1e-12


def test_rational_apply_matches_dense_inverse_sqrt(oracle_lib):
    """(Qhat^2)^(-1/2) b from the eigendecomposition of the dense Qhat^2 on a 4x2^3 lattice:
    every eigen-component is off by at most delta, so the relative error is <= delta
    (+ the solves' residuals, rho = 1e-12)."""
    dims = (4, 2, 2, 2)
    U = synth.random_su3_field(dims, 0.5, 7)
    act = oracle.action(dims, 0.16, 0.1, 0.11)
    b = synth.gaussian_rhs(dims, 8)[0]
    Vh = 16
    Q2 = oracle.dense(lambda v: oracle.qhat2(act, U, v.reshape(Vh, 2, 4, 3)), Vh * 24)
    lam, V = np.linalg.eigh(Q2)
    exact = V @ ((V.conj().T @ b.ravel()) / np.sqrt(lam))
    for n in (6, 10):
        x, delta = oracle.rational_apply(act, U, b, n, lam[0] * 0.999, lam[-1] * 1.001)
        rel = np.linalg.norm(x.ravel() - exact) / np.linalg.norm(exact)
        assert rel <= delta * 1.01 + 1e-10, (n, rel, delta)
        assert rel >= 1e-3 * delta  # the approximation error is really there (not a trivial pass)
