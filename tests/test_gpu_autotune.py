"""The launch-shape autotuner of the 16-bit stencil: every compiled shape gives the same
operator bit for bit (a site's arithmetic does not depend on the launch shape), the
tuner picks one of them from measured times, and a mixed solve under each forced shape
(different block counts, hence different reduction partials) is still certified by the
oracle at 1e-10."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import EPS, KAPPA, MU, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,nrhs", [((8, 6, 6, 6), 1), ((8, 6, 6, 6), 3), ((6, 6, 6, 4), 3)])
def test_shapes_agree_bitwise_and_tuner_picks_one(dims, nrhs):
    """(6, 6, 6, 4): V/2 = 432 odd sites, not a whole number of 32-site groups (ragged tail of
    the per-warp loop order)."""
    tm = require_gpu()
    g = tm.Gauge(synth.random_su3_field(dims, 0.5, 606), dims, KAPPA, MU, EPS)
    b = g.pack(torch.from_numpy(synth.gaussian_rhs(dims, 707, nrhs=nrhs)).cuda(), nrhs=nrhs)
    q = g.convert(b, tm.TMND_F64, tm.TMND_S16, nrhs=nrhs)
    outs = []
    try:
        for sh in range(tm.S16_SHAPES):
            tm.tmnd_s16_force_shape(sh)
            o = g.spinor(nrhs, prec=tm.TMND_S16)
            tm.tm_nd_apply(g.handle, o, q, tm.OP_QHAT2 | tm.OP_S16, 0.013, nrhs=nrhs)
            torch.cuda.synchronize()
            outs.append(o.cpu().numpy().copy())
    finally:
        tm.tmnd_s16_force_shape(-1)
    for sh in range(1, tm.S16_SHAPES):
        assert np.array_equal(outs[sh], outs[0]), sh
    shape, ms = tm.tmnd_autotune(g.handle, nrhs)
    assert 0 <= shape < tm.S16_SHAPES and np.all(ms > 0) and ms[shape] == ms.min()
    # the sloppy multi-shift iteration's objective, tuned in the same pass
    shm, msm = tm.tmnd_autotune_mms(g.handle, nrhs)
    assert 0 <= shm < tm.S16_SHAPES and np.all(msm > 0) and msm[shm] == msm.min()
    g.close()


@pytest.mark.parametrize("shape", [1, 2, 3, 12, 14])
def test_mixed_solve_certified_under_each_shape(shape):
    tm = require_gpu()
    dims = (4, 4, 4, 4)
    U = synth.random_su3_field(dims, 0.3, 1001)
    act = oracle.action(dims, KAPPA, MU, EPS)
    b = synth.gaussian_rhs(dims, 2001, nrhs=2)
    sig = synth.shift_set(10, 1e-4, 1.0)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    bi = g.pack(torch.from_numpy(b).cuda(), nrhs=2)
    xs = [g.spinor(2) for _ in sig]
    try:
        tm.tmnd_s16_force_shape(shape)
        tm.mms_cg_solve(g.handle, bi, 2, sig, xs, prec=tm.TMND_S16, batch=2)
    finally:
        tm.tmnd_s16_force_shape(-1)
    for i, s in enumerate(sig):
        x = g.unpack(xs[i], 2).cpu().numpy()
        for k in range(2):
            assert oracle.true_residual(act, U, b[k], x[k], s) <= 1.01e-10, (shape, i, k)
    g.close()
