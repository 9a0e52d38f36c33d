"""Parity of the CUDA multi-shift CG and the Lagrange guess with the FP64 oracle.

What "match" means for a solve (Sec. 3.1 stopping rule, App. A): each shift's
solution is certified by the ORACLE's operator, |b - (Qhat^2 + sigma_i) x_i| /
|b| <= 1e-10 (a factor 1.01 allows for the summation order of the two FP64
norms; the library finishes any shift whose true residual drifted above rho by FP64
defect correction), and differs from the oracle's own MMS-CG solution by
at most 2 rho |b| / sigma_i (lambda_min(Qhat^2 + sigma) >= sigma).
Element-wise agreement is NOT expected: two correct solutions may differ by
~rho/sigma relative."""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_common import EPS, KAPPA, MU, rel_err, require_gpu, torch

pytestmark = pytest.mark.gpu


def _solve(tm, g, b, sig, rho=1e-10, nsolve=0, nrhs=1, check_every=0, profile=False):
    bi = g.pack(torch.from_numpy(b).cuda(), nrhs=nrhs)
    xs = [g.spinor(nrhs) for _ in sig]
    info = tm.mms_cg_solve(g.handle, bi, nrhs, sig, xs, rho=rho, nsolve=nsolve, check_every=check_every,
                           profile=profile)
    return info, [g.unpack(x, nrhs).cpu().numpy() for x in xs]


@pytest.mark.parametrize("check_every", [0, 7])
def test_mms_config1_matches_oracle(check_every):
    """4^4, roughness 0.3, 10 shifts log-spaced in 1e-4..1, rho 1e-10."""
    tm = require_gpu()
    dims = (4, 4, 4, 4)
    U = synth.random_su3_field(dims, 0.3, 1001)
    b = synth.gaussian_rhs(dims, 2001)[0]
    act = oracle.action(dims, KAPPA, MU, EPS)
    sig = synth.shift_set(10, 1e-4, 1.0)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    info, xs = _solve(tm, g, b, sig, check_every=check_every, profile=check_every > 0)
    ref = oracle.mms_cg(act, U, b, sig, rho=1e-10)
    if check_every > 0:  # profiled: per-iteration event timings are real numbers
        assert np.isfinite(info["hop_ms"]) and info["hop_ms"] > 0
        assert np.isfinite(info["update_ms"]) and info["update_ms"] > 0
    nb = np.linalg.norm(b)
    # same algorithm in FP64: iteration counts agree up to rounding-order effects
    assert abs(info["iters"] - ref["iters"]) <= 2
    for i, s in enumerate(sig):
        x = xs[i][0]
        tr = oracle.true_residual(act, U, b, x, s)
        assert tr <= 1.01e-10, (i, tr)
        assert abs(info["true_res"][i] - tr) <= 1e-3 * tr + 1e-15
        assert np.linalg.norm(x - ref["x"][i]) <= 2e-10 * nb / s
        assert abs(info["conv_iter"][i] - ref["conv_iter"][i]) <= 2
    g.close()


def test_mms_ragged_lattice_multi_rhs_and_guess_shifts():
    """6^3x8 (ragged block tail), two right-hand sides, 2 guess shifts below the
    base that ride along the Krylov space (Sec. 4.2.2) and are not converged."""
    tm = require_gpu()
    dims = (8, 6, 6, 6)
    U = synth.random_su3_field(dims, 0.5, 77)
    act = oracle.action(dims, KAPPA, MU, EPS)
    b = synth.gaussian_rhs(dims, 99, nrhs=2)
    sig = synth.shift_set(8, 1e-3, 2.0)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    info, xs = _solve(tm, g, b, sig, nsolve=6, nrhs=2)
    for k in range(2):
        ref = oracle.mms_cg(act, U, b[k], sig, rho=1e-10, nsolve=6)
        for i in range(6):
            assert oracle.true_residual(act, U, b[k], xs[i][k], sig[i]) <= 1.01e-10
        for i in (6, 7):
            # guess shifts follow the same recursion as the oracle's
            assert rel_err(xs[i][k], ref["x"][i]) < 1e-6
    assert info["conv_iter"][6] == -1 and info["conv_iter"][7] == -1
    g.close()


def test_mms_maxiter_reports_noconv_and_zero_rhs():
    tm = require_gpu()
    dims = (4, 4, 4, 4)
    U = synth.random_su3_field(dims, 0.3, 1001)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    b = synth.gaussian_rhs(dims, 2001)[0]
    bi = g.pack(torch.from_numpy(b).cuda())
    xs = [g.spinor() for _ in range(3)]
    with pytest.raises(tm.TmndError) as e:
        tm.mms_cg_solve(g.handle, bi, 1, [1.0, 0.1, 1e-4], xs, rho=1e-10, maxiter=5)
    assert e.value.status == 4
    # b = 0 gives x = 0 exactly
    z = g.spinor()
    z.zero_()
    info = tm.mms_cg_solve(g.handle, z, 1, [1.0, 0.1], xs[:2], rho=1e-10)
    assert info["iters"] == 0
    assert all(torch.count_nonzero(x).item() == 0 for x in xs[:2])
    # invalid shifts are rejected
    with pytest.raises(tm.TmndError) as e:
        tm.mms_cg_solve(g.handle, bi, 1, [0.1, 1.0], xs[:2])
    assert e.value.status == 1
    g.close()


def test_lagrange_guess_matches_oracle():
    tm = require_gpu()
    dims = (6, 6, 6, 8)
    U = synth.random_su3_field(dims, 0.5, 3)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    rng = np.random.default_rng(5)
    k = 6
    vecs = [rng.standard_normal((g.vh, 2, 4, 3)) + 1j * rng.standard_normal((g.vh, 2, 4, 3)) for _ in range(k)]
    nodes = synth.shift_set(k, 1e-3, 1.0)
    tgt = 3e-4
    xs = [g.pack(torch.from_numpy(v[None]).cuda()) for v in vecs]
    out = g.spinor()
    leb = tm.lagrange_guess(g.handle, nodes, xs, tgt, out)
    got = g.unpack(out)[0].cpu().numpy()
    ref = oracle.lagrange_guess(nodes, vecs, tgt)
    assert leb == pytest.approx(oracle.lebesgue(nodes, tgt), rel=1e-14)
    assert np.max(np.abs(got - ref)) <= 1e-15 * k * leb * max(np.abs(v).max() for v in vecs)
    g.close()


def test_mms_bench_workload_certified_by_oracle():
    """The bench workload itself: 16^3x32, roughness 0.5, 12 shifts log-spaced in
    1e-5..2, one Gaussian RHS, rho 1e-10, in the launch configuration bench.py
    times.  Every shift certified by the oracle's true residual."""
    tm = require_gpu()
    dims = (32, 16, 16, 16)
    U = synth.random_su3_field(dims, 0.5, 1002)
    b = synth.gaussian_rhs(dims, 2032)[0]
    act = oracle.action(dims, KAPPA, MU, EPS)
    sig = synth.shift_set(12, 1e-5, 2.0)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    info, xs = _solve(tm, g, b, sig, profile=True)
    for i, s in enumerate(sig):
        tr = oracle.true_residual(act, U, b, xs[i][0], s)
        assert tr <= 1.01e-10, (i, tr, info)
    # the oracle's own solve of this workload (stored by tests/golden/make_golden.py)
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "mms_16x16x16x32.json")))
    assert abs(info["iters"] - gold["iters"]) <= 2
    assert all(abs(a - b2) <= 2 for a, b2 in zip(info["conv_iter"], gold["conv_iter"]))
    g.close()


def test_fp64_solve_enforces_rho_by_defect_correction():
    """rho = 1e-12 on the 4^4 workload: the recursively updated residual of the multi-shift
    recursion drifts from the true one by more than rho allows, and any shift left above
    rho is finished by FP64 defect correction (Sec. 3.1 stopping rule on the true residual).
    The library's own FP64 true residual of every shift is <= rho; the oracle's evaluation
    of it differs by rounding of order eps |Qhat^2 + sigma| |x| ~ 1e-13 |b| here, so the
    oracle certifies at 1.2 rho."""
    tm = require_gpu()
    dims = (4, 4, 4, 4)
    U = synth.random_su3_field(dims, 0.3, 1001)
    b = synth.gaussian_rhs(dims, 2001)[0]
    act = oracle.action(dims, KAPPA, MU, EPS)
    sig = synth.shift_set(10, 1e-4, 1.0)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    info, xs = _solve(tm, g, b, sig, rho=1e-12)
    for i, s in enumerate(sig):
        tr = oracle.true_residual(act, U, b, xs[i][0], s)
        assert tr <= 1.2e-12, (i, tr, info["refine_rounds"], info["true_res"])
        assert info["true_res"][i] <= 1e-12
    g.close()
