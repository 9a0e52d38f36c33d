"""Pins for the oracle's equivalent solutions of App. A (error and residual of
solutions that agree in exact arithmetic), checked with dense linear algebra on
a 4x2^3 lattice, independent of the oracle's CG: the residual and error of every
method against the upper limits App. A derives (with the exact extreme
eigenvalues of Qhat^2), e = A^-1 r for each, and the identities that define the
residual and error of method C from those of the single systems."""
import numpy as np
import pytest

import oracle
import synth

DIMS = (4, 2, 2, 2)
KAPPA, MU_BAR, EPS_BAR = 0.16, 0.1, 0.11


@pytest.fixture(scope="module")
def problem(oracle_lib):
    act = oracle.action(DIMS, KAPPA, MU_BAR, EPS_BAR)
    U = synth.random_su3_field(DIMS, 0.5, 7)
    vh = int(np.prod(DIMS)) // 2
    n = vh * 24
    Q = oracle.dense(lambda v: oracle.qhat(act, U, v.reshape(vh, 2, 4, 3)), n)
    assert np.allclose(Q, Q.conj().T, atol=1e-13)          # gamma_5 tau_1 hermiticity (Sec. 2)
    lam = np.linalg.eigvalsh(Q @ Q)
    rng = np.random.default_rng(11)
    x = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).reshape(vh, 2, 4, 3)
    return act, U, Q, float(lam[0]), float(lam[-1]), x


@pytest.mark.parametrize("mu", [0.3, 0.03, 0.003])
@pytest.mark.parametrize("rho", [1e-3, 1e-6, 1e-9])
def test_squared_operator_methods_within_app_a_limits(problem, mu, rho):
    act, U, Q, lmin, lmax, x = problem
    n = Q.shape[0]
    A = Q @ Q + mu * mu * np.eye(n)
    b = (A @ x.ravel()).reshape(x.shape)
    bn = np.linalg.norm(b)
    sols = oracle.equivalent_solutions(act, U, b, mu, rho)
    lim = oracle.equivalent_bounds(rho, bn, lmin, lmax, mu)
    for case in "ABC":
        xc = sols[case].ravel()
        r = b.ravel() - A @ xc
        e = x.ravel() - xc
        assert np.linalg.norm(e - np.linalg.solve(A, r)) <= 1e-8 * max(np.linalg.norm(e), 1e-300) + 1e-12 * bn
        assert np.linalg.norm(r) <= lim[case][0] * (1 + 1e-6), (case, np.linalg.norm(r) / bn)
        assert np.linalg.norm(e) <= lim[case][1] * (1 + 1e-6), (case, np.linalg.norm(e))
    # method C from the single systems: with r_pm = b - (Q +- i mu) x_pm and
    # (Q^2 + mu^2) (Q +- i mu)^-1 = Q -+ i mu, r_C = i/(2 mu) ((Q - i mu) r_+ - (Q + i mu) r_-)
    # (App. A prints the two operators the other way round; the norm bound is the same), and
    # e_C = i/(2 mu) (e_+ - e_-)
    I = np.eye(n)
    xp, xm = sols["p"].ravel(), sols["m"].ravel()
    rp, rm = b.ravel() - (Q + 1j * mu * I) @ xp, b.ravel() - (Q - 1j * mu * I) @ xm
    rC = b.ravel() - A @ sols["C"].ravel()
    rC_id = 1j / (2 * mu) * ((Q - 1j * mu * I) @ rp - (Q + 1j * mu * I) @ rm)
    assert np.linalg.norm(rC - rC_id) <= 1e-10 * bn
    ep = np.linalg.solve(Q + 1j * mu * I, b.ravel()) - xp
    em = np.linalg.solve(Q - 1j * mu * I, b.ravel()) - xm
    eC = x.ravel() - sols["C"].ravel()
    assert np.linalg.norm(eC - 1j / (2 * mu) * (ep - em)) <= 1e-8 * np.linalg.norm(x)


@pytest.mark.parametrize("mu", [0.3, 0.003])
def test_single_system_methods_within_app_a_limits(problem, mu):
    """Methods D, E, F for (Qhat +- i mu) x = b: D and F meet |r| <= rho |b|, E only the
    limit inflated by the condition number (App. A, single flavour discussion)."""
    act, U, Q, lmin, lmax, x = problem
    n = Q.shape[0]
    rho = 1e-7
    b = x
    bn = np.linalg.norm(b)
    one = oracle.single_system_solves(act, U, b, mu, rho)
    lim = oracle.equivalent_bounds(rho, bn, lmin, lmax, mu)
    for sg in (+1, -1):
        M = Q + sg * 1j * mu * np.eye(n)
        xt = np.linalg.solve(M, b.ravel())
        for meth in "DEF":
            xs = one[(meth, sg)].ravel()
            r = b.ravel() - M @ xs
            assert np.linalg.norm(r) <= lim[meth][0] * (1 + 1e-6), (meth, sg, np.linalg.norm(r) / bn)
            assert np.linalg.norm(xt - xs) <= lim[meth][1] * (1 + 1e-6), (meth, sg)


def test_methods_agree_in_the_exact_limit(problem):
    """At rho = 1e-13 the three solutions coincide with x to the accuracy the bounds allow."""
    act, U, Q, lmin, lmax, x = problem
    mu = 0.05
    A = Q @ Q + mu * mu * np.eye(Q.shape[0])
    b = (A @ x.ravel()).reshape(x.shape)
    sols = oracle.equivalent_solutions(act, U, b, mu, 1e-13)
    for case in "ABC":
        assert np.linalg.norm(sols[case] - x) <= 1e-8 * np.linalg.norm(x), case


def test_library_limits_equal_oracle_limits():
    """The GPU package restates App. A's limits (relative to |b|) for its study; both
    restatements agree for a range of spectra and shifts."""
    from paper_1805_09584_gb300 import equivalent
    for lmin, lmax, mu, rho in [(1e-3, 2.4, 0.3, 1e-6), (0.011, 2.39, 3.2e-3, 1e-10), (0.0, 5.0, 1e-2, 1e-4)]:
        mine = equivalent.app_a_limits(rho, lmin, lmax, mu)
        ref = oracle.equivalent_bounds(rho, 1.0, lmin, lmax, mu)
        assert set(mine) == set(ref)
        for k in ref:
            assert np.allclose(mine[k], ref[k], rtol=1e-14, atol=0), k
