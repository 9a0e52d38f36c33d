"""Parity of the sloppy operator (FP32 arithmetic on 16-bit links and
spinors) and of the precision conversions with the FP64 oracle.

Tolerances, from the arithmetic: a 16-bit fixed-point site stores every
component to within half a step of (site max)/32767, i.e. a norm-wise
relative error of about 2^-16 * sqrt(48)/sqrt(48) ~ 1.5e-5 per rounding;
the 12-real links carry the same step, and the FP32 sums add ~1e-7.  Mhat
rounds its input, the even intermediate and its output (3 roundings plus
link error): norm-wise relative error below 1e-4.  Qhat^2 has 7 roundings:
below 2e-4.  The F64 -> S16 -> F64 round trip is bounded component-wise by
half a quantisation step (plus FP32 rounding of the value, 6e-8 relative)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import EPS, KAPPA, MU, rel_err, require_gpu, torch

pytestmark = pytest.mark.gpu


def _gauge(dims, r=0.5, seed=1):
    tm = require_gpu()
    U = synth.random_su3_field(dims, r, 1000 + seed)
    return tm, U, tm.Gauge(U, dims, KAPPA, MU, EPS)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 6, 6, 8), (8, 4, 6, 2)])
def test_s16_roundtrip_bound(dims):
    tm, U, g = _gauge(dims)
    b = synth.gaussian_rhs(dims, 3, nrhs=2)
    bi = g.pack(torch.from_numpy(b).cuda(), nrhs=2)
    q = g.convert(bi, tm.TMND_F64, tm.TMND_S16, nrhs=2)
    back = g.unpack(g.convert(q, tm.TMND_S16, tm.TMND_F64, nrhs=2), nrhs=2).cpu().numpy()
    site_max = np.maximum(np.abs(b.real), np.abs(b.imag)).reshape(2, g.vh, -1).max(axis=2)
    step = site_max / 32767.0
    err = np.maximum(np.abs((back - b).real), np.abs((back - b).imag)).reshape(2, g.vh, -1).max(axis=2)
    assert np.all(err <= 0.5 * step * (1 + 1e-5) + 1e-7 * site_max)
    # F64 -> F32 -> F64 is FP32 rounding
    f = g.convert(bi, tm.TMND_F64, tm.TMND_F32, nrhs=2)
    back32 = g.unpack(g.convert(f, tm.TMND_F32, tm.TMND_F64, nrhs=2), nrhs=2).cpu().numpy()
    assert np.max(np.abs(back32 - b) / np.abs(b).max()) < 1.2e-7
    g.close()


# Shapes: X = T = 2, Y = 2, rows of Z/2 = 1, 2, 4, 8, 12, 16 sites (parts of, one
# and several 8-site blocks of the 16-bit layout), 58 time slices.
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 6, 6, 8), (8, 4, 6, 2), (2, 2, 2, 4), (32, 16, 16, 16),
                                  (58, 16, 16, 16), (4, 4, 32, 32), (4, 2, 48, 24), (4, 2, 40, 32), (4, 4, 2, 8),
                                  (2, 2, 4, 8)])
@pytest.mark.parametrize("op,tol", [("mhat", 1e-4), ("mhat_dag", 1e-4), ("qhat2", 2e-4)])
def test_s16_apply_matches_oracle(dims, op, tol):
    tm, U, g = _gauge(dims)
    act = oracle.action(dims, KAPPA, MU, EPS)
    b = synth.gaussian_rhs(dims, 11)[0]
    sigma = 0.0137
    ref = {"mhat": lambda: oracle.schur(act, U, b),
           "mhat_dag": lambda: oracle.schur(act, U, b, dagger=True),
           "qhat2": lambda: oracle.qhat2(act, U, b, sigma)}[op]()
    code = {"mhat": tm.OP_MHAT, "mhat_dag": tm.OP_MHAT_DAG, "qhat2": tm.OP_QHAT2}[op]
    q = g.convert(g.pack(torch.from_numpy(b).cuda()), tm.TMND_F64, tm.TMND_S16)
    out = g.spinor(prec=tm.TMND_S16)
    tm.tm_nd_apply(g.handle, out, q, code | tm.OP_S16, sigma)
    got = g.unpack(g.convert(out, tm.TMND_S16, tm.TMND_F64))[0].cpu().numpy()
    assert rel_err(got, ref) <= tol
    g.close()


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 6, 6, 8)])
def test_f32_operator_matches_oracle(dims):
    """The FP32 operator (TMND_OP_F32: the FP64 stencil instantiated in FP32 with FP32 links,
    used for the inner residuals of the defect correction) against the oracle: FP32 rounding
    of inputs, links and ~100 summed products per component gives a norm-wise relative error
    of a few 1e-7; bound 2e-6 for Mhat, Mhat^+ and Qhat^2 + sigma, two right-hand sides."""
    tm, U, g = _gauge(dims, seed=7)
    act = oracle.action(dims, KAPPA, MU, EPS)
    b = synth.gaussian_rhs(dims, 31, nrhs=2)
    bi = g.pack(torch.from_numpy(b).cuda(), nrhs=2)
    f = g.convert(bi, tm.TMND_F64, tm.TMND_F32, nrhs=2)
    for op, ref_fn in ((tm.OP_MHAT, lambda v: oracle.schur(act, U, v)),
                       (tm.OP_MHAT_DAG, lambda v: oracle.schur(act, U, v, dagger=True)),
                       (tm.OP_QHAT2, lambda v: oracle.qhat2(act, U, v, 0.021))):
        o = g.spinor(2, prec=tm.TMND_F32)
        tm.tm_nd_apply(g.handle, o, f, op | tm.OP_F32, 0.021, nrhs=2)
        got = g.unpack(g.convert(o, tm.TMND_F32, tm.TMND_F64, nrhs=2), nrhs=2).cpu().numpy()
        for k in range(2):
            assert rel_err(got[k], ref_fn(b[k])) < 2e-6, (op, k)
    g.close()
