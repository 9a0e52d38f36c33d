"""Pins for the oracle's solvers (Sec. 1 Eq. "shifted_linear"; Sec. 4.2.2 MMS-CG):
dense LU on tiny lattices, plain CG, MMS collinearity, true residuals."""
import numpy as np
import pytest

import oracle
import synth

KAPPA, MU, EPS = 0.16, 0.1, 0.11


@pytest.fixture(scope="module")
def tiny():
    dims = (4, 2, 2, 2)
    U = synth.random_su3_field(dims, 0.3, 1001)
    act = oracle.action(dims, KAPPA, MU, EPS)
    b = synth.gaussian_rhs(dims, 2001)[0]
    Vh = 16
    Q2 = oracle.dense(lambda v: oracle.qhat2(act, U, v.reshape(Vh, 2, 4, 3)), Vh * 24)
    return dims, U, act, b, Q2


def test_qhat2_dense_is_hermitian_positive(oracle_lib, tiny):
    _, _, _, _, Q2 = tiny
    assert np.max(np.abs(Q2 - Q2.conj().T)) < 1e-14 * np.abs(Q2).max()
    assert np.linalg.eigvalsh(Q2).min() > 0


def test_mms_cg_matches_dense_lu(oracle_lib, tiny):
    """Every shift of the MMS-CG equals numpy's dense solve of (Qhat^2 + sigma) x = b
    within the error the stopping rule allows (|dx| <= rho |b| / lambda_min(Qhat^2+sigma))."""
    dims, U, act, b, Q2 = tiny
    sig = synth.shift_set(10, 1e-4, 1.0)
    rho = 1e-12
    res = oracle.mms_cg(act, U, b, sig, rho=rho)
    assert res["iters"] > 0
    lam = np.linalg.eigvalsh(Q2).min()
    for i, s in enumerate(sig):
        xd = np.linalg.solve(Q2 + s * np.eye(Q2.shape[0]), b.ravel())
        err = np.linalg.norm(res["x"][i].ravel() - xd)
        # recursive-residual stop plus a small allowance for its drift from the true residual
        assert err <= 10 * rho * np.linalg.norm(b) / (lam + s)


def test_single_shift_mms_equals_cg(oracle_lib, tiny):
    """With one shift the MMS recursion collapses to plain CG (zeta = 1):
    same iteration count, same iterate."""
    dims, U, act, b, _ = tiny
    res = oracle.mms_cg(act, U, b, [0.01], rho=1e-10)
    x, it = oracle.cg(act, U, b, 0.01, rho=1e-10)
    assert res["iters"] == it
    assert np.max(np.abs(res["x"][0] - x)) < 1e-12 * np.abs(x).max()


def test_mms_collinear_residuals(oracle_lib):
    """Defining property of the multi-shift recursion: after k steps the
    residual of shift i is zeta_i times the base residual,
    b - (Qhat^2 + sigma_i) x_i = zeta_i (b - (Qhat^2 + sigma_0) x_0)."""
    dims = (4, 4, 4, 4)
    U = synth.random_su3_field(dims, 0.3, 1001)
    act = oracle.action(dims, KAPPA, MU, EPS)
    b = synth.gaussian_rhs(dims, 2001)[0]
    sig = synth.shift_set(6, 1e-3, 1.0)
    res = oracle.mms_cg(act, U, b, sig, rho=1e-30, maxiter=12)
    assert res["iters"] == -12
    r0 = b - oracle.qhat2(act, U, res["x"][-1], sig[-1])
    assert res["zeta"][-1] == 1.0
    for i in range(len(sig) - 1):
        ri = b - oracle.qhat2(act, U, res["x"][i], sig[i])
        assert np.linalg.norm(ri - res["zeta"][i] * r0) < 1e-11 * np.linalg.norm(b)
        assert 0 < res["zeta"][i] < 1


def test_mms_config1_true_residuals(oracle_lib):
    """4^4 doublet, kappa 0.16, mu 0.1, eps 0.11, roughness 0.3, 10 shifts log-spaced
    in 1e-4..1: every shift reaches true relative residual <= 1e-10, and agrees
    with a separate plain CG on that shift within 2 rho |b| / sigma."""
    dims = (4, 4, 4, 4)
    U = synth.random_su3_field(dims, 0.3, 1001)
    act = oracle.action(dims, KAPPA, MU, EPS)
    b = synth.gaussian_rhs(dims, 2001)[0]
    sig = synth.shift_set(10, 1e-4, 1.0)
    rho = 1e-10
    res = oracle.mms_cg(act, U, b, sig, rho=rho)
    assert res["iters"] > 0
    conv = res["conv_iter"]
    assert np.all(conv > 0) and np.all(np.diff(conv) >= 0)  # larger shifts converge first
    nb = np.linalg.norm(b)
    for i, s in enumerate(sig):
        assert oracle.true_residual(act, U, b, res["x"][i], s) <= 1.01 * rho
    for i in (0, 5, 9):
        x, _ = oracle.cg(act, U, b, sig[i], rho=rho)
        assert np.linalg.norm(x - res["x"][i]) <= 2 * rho * nb / sig[i]


def test_mms_guess_shifts(oracle_lib):
    """Guess shifts below the base (Sec. 4.2.2) ride along the base Krylov space:
    they stay collinear with the base residual and are not converged."""
    dims = (4, 4, 4, 4)
    U = synth.random_su3_field(dims, 0.3, 1001)
    act = oracle.action(dims, KAPPA, MU, EPS)
    b = synth.gaussian_rhs(dims, 2001)[0]
    sig = synth.shift_set(10, 1e-4, 1.0)
    res = oracle.mms_cg(act, U, b, sig, rho=1e-10, nsolve=7)
    assert res["iters"] > 0
    assert np.all(res["conv_iter"][7:] == -1)
    r0n = oracle.true_residual(act, U, b, res["x"][6], sig[6])
    for i in (7, 8):
        ri = oracle.true_residual(act, U, b, res["x"][i], sig[i])
        assert ri > r0n and ri < 1.0
        assert abs(ri - res["zeta"][i] * r0n) < 0.05 * ri + 1e-12
