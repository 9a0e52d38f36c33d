"""Rational approximation of the inverse square root on the GPU (Sec. 4.1,
Eq. "ratapp"): tmnd_rational_apply against the exact (Qhat^2)^(-1/2) b of a dense
Qhat^2 (relative error within delta + the solves'), and against the oracle's
chain on a larger lattice (same approximation: agreement to the solves'
tolerance), in FP64 and with the mixed-precision solve."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import EPS, KAPPA, MU, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [6, 10])
def test_rational_apply_vs_dense_inverse_sqrt(n):
    tm = require_gpu()
    dims = (4, 2, 2, 2)
    U = synth.random_su3_field(dims, 0.5, 7)
    act = oracle.action(dims, KAPPA, MU, EPS)
    b = synth.gaussian_rhs(dims, 8)[0]
    Vh = 16
    Q2 = oracle.dense(lambda v: oracle.qhat2(act, U, v.reshape(Vh, 2, 4, 3)), Vh * 24)
    lam, V = np.linalg.eigh(Q2)
    exact = V @ ((V.conj().T @ b.ravel()) / np.sqrt(lam))
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    bi = g.pack(torch.from_numpy(b[None]).cuda())
    out = g.spinor()
    info = tm.tmnd_rational_apply(g.handle, bi, 1, n, lam[0] * 0.999, lam[-1] * 1.001, out, rho=1e-12)
    x = g.unpack(out)[0].cpu().numpy().ravel()
    rel = np.linalg.norm(x - exact) / np.linalg.norm(exact)
    assert rel <= info["delta"] * 1.01 + 1e-9, (rel, info)
    g.close()


@pytest.mark.parametrize("prec", [0, 2])
def test_rational_apply_matches_oracle_chain(prec):
    tm = require_gpu()
    dims = (8, 4, 4, 4)
    U = synth.random_su3_field(dims, 0.5, 17)
    act = oracle.action(dims, KAPPA, MU, EPS)
    b = synth.gaussian_rhs(dims, 18, nrhs=2)
    lmin, lmax, n = 1e-3, 1.2, 10
    ref = [oracle.rational_apply(act, U, b[k], n, lmin, lmax, rho=1e-12)[0] for k in range(2)]
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    bi = g.pack(torch.from_numpy(b).cuda(), nrhs=2)
    out = g.spinor(2)
    info = tm.tmnd_rational_apply(g.handle, bi, 2, n, lmin, lmax, out, rho=1e-11, prec=prec)
    x = g.unpack(out, 2).cpu().numpy()
    for k in range(2):
        # each x_i has relative residual <= 1e-11; the combination weights lmax q_i / (Qhat^2 + sigma_i)
        # amplify that by at most sum_i |lmax q_i| / sigma_i relative to |x|
        rel = np.linalg.norm(x[k] - ref[k]) / np.linalg.norm(ref[k])
        assert rel <= 1e-8, (k, rel, info)
    assert max(info["true_res"]) <= 1.01e-11
    g.close()
