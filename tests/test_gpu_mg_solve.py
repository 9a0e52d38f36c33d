"""Two-level MG solve of the case-C systems on the GPU (Sec. 3, Eq.
"error_propagation"; Sec. 3.1 Eq. "lindif") against the FP64 oracle.

FP32 solve to tol 1e-4 (an FP32 Krylov solve attains ~ eps_32 * cond(D') ~ 1e-5
here, so the multigrid is a preconditioner-level solver; the hybrid driver
finishes every shift with FP64 defect correction): the oracle's FP64 residual
of the returned vector must be below 2e-4, and the odd part must solve
(Qhat + i s) y = b to 1e-3, since with the right-hand side (0_e, gamma_5 tau_1 b)
the odd Schur complement of D_ND + i s gamma_5 tau_1 Pi_odd is gamma_5 tau_1 (Qhat + i s)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import EPS, KAPPA, MU, require_gpu, torch
from test_gpu_mg import from_mg_layout, to_mg_layout

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("s,smoother", [(0.05, 0), (-0.05, 0), (0.05, 1), (-0.05, 1)])
def test_mg_solve_case_c(s, smoother):
    """smoother 0: minimal residual on the whole lattice; 1: SAP on the 2^4 aggregation blocks."""
    tm = require_gpu()
    dims, bdims, nv = (8, 4, 4, 4), (2, 2, 2, 2), 6
    V = int(np.prod(dims))
    U = synth.random_su3_field(dims, 0.5, 31)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    act = oracle.action(dims, KAPPA, MU, EPS)
    rng = np.random.default_rng(1)
    tv = rng.standard_normal((nv, V, 12)) + 1j * rng.standard_normal((nv, V, 12))
    tvd = torch.from_numpy(to_mg_layout(dims, tv.astype(np.complex64), 12)).cuda().contiguous()
    tm.tmnd_mg_smooth_vectors(g.handle, tvd, nv, 6)
    mg = tm.tmnd_mg_create(g.handle, bdims, nv, tvd, smoother=smoother)
    b = synth.gaussian_rhs(dims, 5)[0]                      # odd-site doublet [V/2, 2, 4, 3]
    g5t1 = (b[:, ::-1] * np.array([1, 1, -1, -1])[None, None, :, None])
    rhs = np.zeros((V, 2, 4, 3), np.complex128)
    rhs[synth.odd_sites(dims)] = g5t1
    rd = torch.from_numpy(to_mg_layout(dims, rhs.reshape(V, 24).astype(np.complex64), 24)).cuda().contiguous()
    x = torch.zeros_like(rd)
    info = tm.tmnd_mg_solve(mg, x, rd, s, tol=1e-4, maxiter=300, restart=8, nu=4)
    xs = from_mg_layout(dims, x.cpu().numpy().reshape(2, 24, V // 2), 24).reshape(V, 2, 4, 3)
    r = rhs - oracle.dnd_odd_shift(act, U, xs, s)
    assert info["res"] <= 1e-4, info
    assert np.linalg.norm(r) / np.linalg.norm(rhs) < 2e-4, info
    yo = xs[synth.odd_sites(dims)]
    qy = oracle.qhat(act, U, yo) + 1j * s * yo
    assert np.linalg.norm(qy - b) / np.linalg.norm(b) < 1e-3
    # the coarse-grid correction must help: fewer outer iterations than without it
    x2 = torch.zeros_like(rd)
    info0 = tm.tmnd_mg_solve(mg, x2, rd, s, tol=1e-4, maxiter=300, restart=8, nu=0)
    assert info["iters"] <= info0["iters"]
    tm.tmnd_mg_destroy(mg)
    g.close()


def test_full_operator_matches_oracle():
    tm = require_gpu()
    dims = (4, 4, 2, 6)
    V = int(np.prod(dims))
    U = synth.random_su3_field(dims, 0.5, 8)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    act = oracle.action(dims, KAPPA, MU, EPS)
    rng = np.random.default_rng(2)
    v = rng.standard_normal((V, 24)) + 1j * rng.standard_normal((V, 24))
    vd = torch.from_numpy(to_mg_layout(dims, v.astype(np.complex64), 24)).cuda().contiguous()
    out = torch.zeros_like(vd)
    for s in (0.0, 0.07):
        tm.tmnd_dnd_full_apply(g.handle, out, vd, s)
        got = from_mg_layout(dims, out.cpu().numpy().reshape(2, 24, V // 2), 24)
        ref = oracle.dnd_odd_shift(act, U, v.reshape(V, 2, 4, 3), s).reshape(V, 24)
        assert np.max(np.abs(got - ref)) < 2e-6 * np.abs(ref).max()
    g.close()


def test_bootstrap_setup_then_case_c_certified():
    """Adaptive setup (tmnd_mg_bootstrap: test vectors improved by the two-level method itself,
    SAP smoothing), then a case-C solve with the new hierarchy, certified by the oracle as above."""
    tm = require_gpu()
    dims, bdims, nv, s = (8, 4, 4, 4), (2, 2, 2, 2), 6, 0.05
    V = int(np.prod(dims))
    U = synth.random_su3_field(dims, 0.5, 31)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    act = oracle.action(dims, KAPPA, MU, EPS)
    rng = np.random.default_rng(1)
    tv = rng.standard_normal((nv, V, 12)) + 1j * rng.standard_normal((nv, V, 12))
    tvd = torch.from_numpy(to_mg_layout(dims, tv.astype(np.complex64), 12)).cuda().contiguous()
    tm.tmnd_mg_smooth_vectors(g.handle, tvd, nv, 6)
    mg0 = tm.tmnd_mg_create(g.handle, bdims, nv, tvd, smoother=1)
    mg1 = tm.tmnd_mg_bootstrap(mg0, tvd, 3, bdims, nv, smoother=1)
    assert torch.isfinite(torch.view_as_real(tvd)).all()
    b = synth.gaussian_rhs(dims, 5)[0]
    g5t1 = (b[:, ::-1] * np.array([1, 1, -1, -1])[None, None, :, None])
    rhs = np.zeros((V, 2, 4, 3), np.complex128)
    rhs[synth.odd_sites(dims)] = g5t1
    rd = torch.from_numpy(to_mg_layout(dims, rhs.reshape(V, 24).astype(np.complex64), 24)).cuda().contiguous()
    its = []
    for mg in (mg0, mg1):
        x = torch.zeros_like(rd)
        info = tm.tmnd_mg_solve(mg, x, rd, s, tol=1e-4, maxiter=300, restart=8, nu=2)
        xs = from_mg_layout(dims, x.cpu().numpy().reshape(2, 24, V // 2), 24).reshape(V, 2, 4, 3)
        r = rhs - oracle.dnd_odd_shift(act, U, xs, s)
        assert np.linalg.norm(r) / np.linalg.norm(rhs) < 2e-4, info
        its.append(info["iters"])
    assert all(0 < i < 300 for i in its), its   # both hierarchies converge; bench --study mg compares them
    tm.tmnd_mg_destroy(mg1)
    tm.tmnd_mg_destroy(mg0)
    g.close()
