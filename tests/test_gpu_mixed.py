"""Mixed-precision multi-shift solve (sloppy FP32/16-bit MMS-CG + FP64 defect
correction) against the FP64 oracle.  The certification is the oracle's own
true residual |b - (Qhat^2 + sigma_i) x_i| / |b| <= 1e-10 for every required
shift (the library stops each shift on its FP64 true residual, so no drift
allowance is needed beyond FP64 summation-order effects: factor 1.01)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import EPS, KAPPA, MU, require_gpu, torch

pytestmark = pytest.mark.gpu


def _mixed(tm, g, b, sig, nrhs=1, nsolve=0, rho=1e-10, rho_inner=0.0):
    bi = g.pack(torch.from_numpy(b).cuda(), nrhs=nrhs)
    xs = [g.spinor(nrhs) for _ in sig]
    info = tm.mms_cg_solve(g.handle, bi, nrhs, sig, xs, rho=rho, nsolve=nsolve, prec=tm.TMND_S16,
                           rho_inner=rho_inner)
    return info, [g.unpack(x, nrhs).cpu().numpy() for x in xs]


def test_mixed_config1_certified():
    tm = require_gpu()
    dims = (4, 4, 4, 4)
    U = synth.random_su3_field(dims, 0.3, 1001)
    b = synth.gaussian_rhs(dims, 2001)[0]
    act = oracle.action(dims, KAPPA, MU, EPS)
    sig = synth.shift_set(10, 1e-4, 1.0)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    info, xs = _mixed(tm, g, b, sig)
    for i, s in enumerate(sig):
        tr = oracle.true_residual(act, U, b, xs[i][0], s)
        assert tr <= 1.01e-10, (i, tr, info)
        assert abs(info["true_res"][i] - tr) <= 1e-3 * tr + 1e-16
    # one defect-correction round per pair: the FP64 defect after the multi-shift solve and the
    # final check; the inner refinement in between checks itself with the FP32 operator
    assert len(sig) <= info["fp64_applies"] <= 2 * len(sig), info
    assert info["f32_applies"] > 0, info
    g.close()


def test_mixed_multi_rhs_ragged_and_guess_shifts():
    tm = require_gpu()
    dims = (8, 6, 6, 6)
    U = synth.random_su3_field(dims, 0.5, 77)
    act = oracle.action(dims, KAPPA, MU, EPS)
    b = synth.gaussian_rhs(dims, 99, nrhs=2)
    sig = synth.shift_set(8, 1e-3, 2.0)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    info, xs = _mixed(tm, g, b, sig, nrhs=2, nsolve=6)
    for k in range(2):
        for i in range(6):
            assert oracle.true_residual(act, U, b[k], xs[i][k], sig[i]) <= 1.01e-10
        for i in (6, 7):  # guess shifts: sloppy iterates, better than the zero vector
            assert oracle.true_residual(act, U, b[k], xs[i][k], sig[i]) < 1.0
    g.close()


def test_mixed_bench_lattice_certified():
    """16^3x32, roughness 0.5, 12 shifts in 1e-5..2: every shift certified."""
    tm = require_gpu()
    dims = (32, 16, 16, 16)
    U = synth.random_su3_field(dims, 0.5, 1002)
    b = synth.gaussian_rhs(dims, 2032)[0]
    act = oracle.action(dims, KAPPA, MU, EPS)
    sig = synth.shift_set(12, 1e-5, 2.0)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    info, xs = _mixed(tm, g, b, sig)
    for i, s in enumerate(sig):
        tr = oracle.true_residual(act, U, b, xs[i][0], s)
        assert tr <= 1.01e-10, (i, tr, info)
    g.close()


@pytest.mark.parametrize("nrhs,batch", [(3, 0), (5, 2)])
def test_mixed_batched_rhs_match_one_at_a_time(nrhs, batch):
    """Batched sloppy solve (all right-hand sides in every stencil launch, each
    with its own scalars and stopping point; 5 RHS in batches of 2 leaves a
    ragged last batch): every shift of every RHS certified by the oracle, and
    the solutions agree with the one-at-a-time solve to the certified accuracy."""
    tm = require_gpu()
    dims = (8, 6, 6, 6)
    U = synth.random_su3_field(dims, 0.5, 78)
    act = oracle.action(dims, KAPPA, MU, EPS)
    b = synth.gaussian_rhs(dims, 101, nrhs=nrhs)
    b[1] *= 1e-3   # right-hand sides of very different size converge at different iterations
    sig = synth.shift_set(8, 1e-3, 2.0)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    bi = g.pack(torch.from_numpy(b).cuda(), nrhs=nrhs)
    xb = [g.spinor(nrhs) for _ in sig]
    x1 = [g.spinor(nrhs) for _ in sig]
    tm.mms_cg_solve(g.handle, bi, nrhs, sig, xb, prec=tm.TMND_S16, batch=batch)
    tm.mms_cg_solve(g.handle, bi, nrhs, sig, x1, prec=tm.TMND_S16, batch=1)
    for i, s in enumerate(sig):
        a = g.unpack(xb[i], nrhs).cpu().numpy()
        c = g.unpack(x1[i], nrhs).cpu().numpy()
        for k in range(nrhs):
            assert oracle.true_residual(act, U, b[k], a[k], s) <= 1.01e-10, (i, k)
            # both are certified solutions: they differ by at most ~ rho |b| / sigma
            assert np.linalg.norm(a[k] - c[k]) <= 2e-10 * np.linalg.norm(b[k]) / s
    g.close()


@pytest.mark.parametrize("dims", [(8, 6, 6, 6), (6, 4, 8, 16)])
def test_s16_multi_rhs_apply_equals_single(dims):
    """One 16-bit stencil launch over 3 right-hand sides gives, bit for bit, the
    three single applications (same arithmetic per right-hand side)."""
    tm = require_gpu()
    U = synth.random_su3_field(dims, 0.4, 79)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    b = synth.gaussian_rhs(dims, 103, nrhs=3)
    q = g.convert(g.pack(torch.from_numpy(b).cuda(), nrhs=3), tm.TMND_F64, tm.TMND_S16, nrhs=3)
    for op in (tm.OP_MHAT, tm.OP_QHAT2):
        out3 = g.spinor(3, prec=tm.TMND_S16)
        tm.tm_nd_apply(g.handle, out3, q, op | tm.OP_S16, 0.0213, nrhs=3)
        nb = tm.tmnd_spinor_bytes_prec(g.handle, tm.TMND_S16)
        q8, o8 = q.view(torch.uint8), out3.view(torch.uint8)
        for k in range(3):
            one = g.spinor(1, prec=tm.TMND_S16)
            tm.tm_nd_apply(g.handle, one, q8[k * nb:(k + 1) * nb], op | tm.OP_S16, 0.0213, nrhs=1)
            assert torch.equal(one.view(torch.uint8), o8[k * nb:(k + 1) * nb]), (op, k)
    g.close()


def test_mixed_batch_with_zero_rhs_and_argument_limits():
    """A zero right-hand side inside a batch gives x = 0 while the others are
    certified; batch > 16 and 16-bit applies of more than 16 RHS are rejected."""
    tm = require_gpu()
    dims = (4, 4, 4, 4)
    U = synth.random_su3_field(dims, 0.4, 81)
    act = oracle.action(dims, KAPPA, MU, EPS)
    b = synth.gaussian_rhs(dims, 82, nrhs=3)
    b[1] = 0
    sig = synth.shift_set(6, 1e-3, 1.0)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    bi = g.pack(torch.from_numpy(b).cuda(), nrhs=3)
    xs = [g.spinor(3) for _ in sig]
    tm.mms_cg_solve(g.handle, bi, 3, sig, xs, prec=tm.TMND_S16, batch=3)
    for i, s in enumerate(sig):
        x = g.unpack(xs[i], 3).cpu().numpy()
        assert np.all(x[1] == 0)
        for k in (0, 2):
            assert oracle.true_residual(act, U, b[k], x[k], s) <= 1.01e-10
    with pytest.raises(RuntimeError):
        tm.mms_cg_solve(g.handle, bi, 3, sig, xs, prec=tm.TMND_S16, batch=17)
    q = g.spinor(17, prec=tm.TMND_S16)
    o = g.spinor(17, prec=tm.TMND_S16)
    with pytest.raises(RuntimeError):
        tm.tm_nd_apply(g.handle, o, q, tm.OP_MHAT | tm.OP_S16, 0.0, nrhs=17)
    g.close()
