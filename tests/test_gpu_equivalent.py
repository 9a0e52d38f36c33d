"""Equivalent solutions of App. A on the GPU (paper_1805_09584_gb300.equivalent,
through the C-ABI) against the oracle: on a 4x2^3 lattice every method's residual
and error meet App. A's upper limits with the exact extreme eigenvalues of Qhat^2
(dense, oracle side) and r_C obeys its defining identity; on 8x4^3 the GPU solutions
of methods A, B, C agree with the oracle's within their error limits; the complex
combination and the site-norm range match numpy."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import EPS, KAPPA, MU, require_gpu, torch

pytestmark = pytest.mark.gpu


def _setup(dims, seed):
    tm = require_gpu()
    U = synth.random_su3_field(dims, 0.5, seed)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    act = oracle.action(dims, KAPPA, MU, EPS)
    return tm, U, g, act


def _host(g, v):
    return g.unpack(v)[0].cpu().numpy()


def test_lincomb_c_and_site_norm_range():
    tm, U, g, act = _setup((4, 4, 4, 4), 3)
    rng = np.random.default_rng(5)
    a, b = synth.gaussian_rhs((4, 4, 4, 4), 6)[0], synth.gaussian_rhs((4, 4, 4, 4), 7)[0]
    da, db = g.pack(torch.from_numpy(a[None]).cuda()), g.pack(torch.from_numpy(b[None]).cuda())
    w = rng.standard_normal(2) + 1j * rng.standard_normal(2)
    out = g.spinor()
    tm.tmnd_lincomb_c(g.handle, w, [da, db], out)
    assert np.allclose(_host(g, out), w[0] * a + w[1] * b, rtol=0, atol=1e-13)
    tm.tmnd_lincomb_c(g.handle, [1j], [da], da)          # in place: x <- i x
    assert np.allclose(_host(g, da), 1j * a, rtol=0, atol=1e-14)
    lo, hi = tm.tmnd_site_norm_range(g.handle, db)
    site = np.linalg.norm(b.reshape(b.shape[0], -1), axis=1)
    assert abs(lo - site.min()) <= 1e-13 * site.max() and abs(hi - site.max()) <= 1e-13 * site.max()
    g.close()


@pytest.mark.parametrize("mu", [0.3, 0.01])
def test_methods_meet_app_a_limits(mu):
    from paper_1805_09584_gb300 import equivalent
    dims = (4, 2, 2, 2)
    tm, U, g, act = _setup(dims, 7)
    vh = int(np.prod(dims)) // 2
    n = vh * 24
    Q = oracle.dense(lambda v: oracle.qhat(act, U, v.reshape(vh, 2, 4, 3)), n)
    lam = np.linalg.eigvalsh(Q @ Q)
    A = Q @ Q + mu * mu * np.eye(n)
    x = synth.gaussian_rhs(dims, 21)[0]
    bh = (A @ x.ravel()).reshape(x.shape)
    b = g.pack(torch.from_numpy(bh[None]).cuda())
    for rho in (1e-4, 1e-9):
        sols, one = equivalent.equivalent_solutions(g, b, mu, rho)
        lim = oracle.equivalent_bounds(rho, np.linalg.norm(bh), lam[0], lam[-1], mu)
        for case in "ABC":
            xc = _host(g, sols[case]).ravel()
            r, e = bh.ravel() - A @ xc, x.ravel() - xc
            assert np.linalg.norm(r) <= lim[case][0] * (1 + 1e-6), (case, rho)
            assert np.linalg.norm(e) <= lim[case][1] * (1 + 1e-6), (case, rho)
        I = np.eye(n)
        xp, xm = _host(g, sols["p"]).ravel(), _host(g, sols["m"]).ravel()
        rp, rm = bh.ravel() - (Q + 1j * mu * I) @ xp, bh.ravel() - (Q - 1j * mu * I) @ xm
        rC = bh.ravel() - A @ _host(g, sols["C"]).ravel()
        assert np.linalg.norm(rC - 1j / (2 * mu) * ((Q - 1j * mu * I) @ rp - (Q + 1j * mu * I) @ rm)) \
            <= 1e-10 * np.linalg.norm(bh)
        M = Q + 1j * mu * I
        for meth in "DEF":
            xs = _host(g, one[(meth, +1)]).ravel()
            assert np.linalg.norm(bh.ravel() - M @ xs) <= lim[meth][0] * (1 + 1e-6), (meth, rho)
            assert np.linalg.norm(np.linalg.solve(M, bh.ravel()) - xs) <= lim[meth][1] * (1 + 1e-6), (meth, rho)
        xm_single = equivalent.single_system_solves(g, b, mu, rho)
        for meth in "DEF":
            xs = _host(g, xm_single[(meth, -1)]).ravel()
            assert np.linalg.norm(bh.ravel() - (Q - 1j * mu * I) @ xs) <= lim[meth][0] * (1 + 1e-6), (meth, rho)
        rep = equivalent.residual_and_error(g, b, g.pack(torch.from_numpy(x[None]).cuda()), sols["A"], mu)
        xa = _host(g, sols["A"]).ravel()
        assert abs(rep["res"] - np.linalg.norm(bh.ravel() - A @ xa) / np.linalg.norm(bh)) <= 1e-6 * rep["res"]
        assert abs(rep["err"] - np.linalg.norm(x.ravel() - xa) / np.linalg.norm(bh)) <= 1e-6 * rep["err"]
        # the library's restatement of the limits equals the oracle's
        mine = equivalent.app_a_limits(rho, lam[0], lam[-1], mu)
        for k, (lr, le) in lim.items():
            assert np.allclose(np.array(mine[k]) * np.linalg.norm(bh), [lr, le], rtol=1e-14)
    g.close()


def test_gpu_methods_agree_with_oracle():
    from paper_1805_09584_gb300 import equivalent
    dims = (8, 4, 4, 4)
    tm, U, g, act = _setup(dims, 9)
    mu, rho = 0.05, 1e-10
    x = synth.gaussian_rhs(dims, 31)[0]
    bh = oracle.qhat2(act, U, x, mu * mu)
    b = g.pack(torch.from_numpy(bh[None]).cuda())
    sols, _ = equivalent.equivalent_solutions(g, b, mu, rho)
    ref = oracle.equivalent_solutions(act, U, bh, mu, rho)
    # every limit of App. A for |e| of A, B, C is at most 2 rho |b| / mu^2 (lambda_min >= 0)
    tol = 2 * rho * np.linalg.norm(bh) / (mu * mu)
    for case in "ABC":
        xg = _host(g, sols[case])
        assert np.linalg.norm(xg - ref[case]) <= 2 * tol, case
        assert np.linalg.norm(xg - x) <= tol, case
    g.close()
