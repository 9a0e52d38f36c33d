"""Failure paths, exercised without a GPU fault, trap or hang:
  * a bounded wait of the tensor-core coarse kernel runs out: the handle's test hook
    makes the MMA warp of every block wait, after its first MMAs, on a barrier that
    nothing completes, with a 20 ms limit.  tmnd_mg_status reports TMND_ERR_TIMEOUT,
    the kernel has drained its copies and MMAs and freed its tensor memory, and the
    next apply on the same handle matches the oracle;
  * a NaN in the host right-hand side: mms_cg_solve returns TMND_ERR_NAN from its
    FP64 reductions (FP64 and mixed forms) instead of iterating on, and the handle
    then solves a clean system to the oracle-certified 1e-10."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import EPS, KAPPA, MU, require_gpu, torch
from test_gpu_mg import to_mg_layout

pytestmark = pytest.mark.gpu


def test_coarse_tc_wait_timeout_reported_and_recovers():
    tm = require_gpu()
    dims, bdims, nv = (4, 4, 4, 4), (2, 2, 2, 2), 4
    U = synth.random_su3_field(dims, 0.5, 99)
    V = int(np.prod(dims))
    rng = np.random.default_rng(3)
    vecs = (rng.standard_normal((nv, V, 12)) + 1j * rng.standard_normal((nv, V, 12))).astype(np.complex64)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    tv = torch.from_numpy(to_mg_layout(dims, vecs, 12)).cuda()
    mg = tm.tmnd_mg_create(g.handle, bdims, nv, tv, wait_limit_s=0.02, stall_test=1)
    nb = V // 16
    R = 2
    xv = rng.standard_normal((R, nb * 4 * nv)) + 1j * rng.standard_normal((R, nb * 4 * nv))
    xin = torch.from_numpy(xv.astype(np.complex64).ravel()).cuda()
    y = torch.zeros_like(xin)
    tm.mg_coarse_apply(mg, y, xin, R, 0.03)          # the stalled launch
    with pytest.raises(tm.TmndError) as e:
        tm.tmnd_mg_status(mg)
    assert e.value.status == 6, e.value              # TMND_ERR_TIMEOUT
    tm.tmnd_mg_status(mg)                            # the flag was cleared
    # the same handle, next launch: parity with the oracle's P_ND^+ D' P_ND
    tm.mg_coarse_apply(mg, y, xin, R, 0.03)
    tm.tmnd_mg_status(mg)
    act = oracle.action(dims, KAPPA, MU, EPS)
    P = oracle.mg_prolongator(dims, bdims, vecs.astype(np.complex128).reshape(nv, V, 4, 3))
    Dnd = oracle.mg_coarse_nd_odd_shift(act, U, P, nv, 0.03)
    got = y.cpu().numpy().reshape(R, -1)
    for r in range(R):
        ref = Dnd @ xv[r]
        assert np.max(np.abs(got[r] - ref)) < 4e-3 * np.abs(ref).max(), r
    tm.tmnd_mg_destroy(mg)
    g.close()


@pytest.mark.parametrize("prec", [0, 2])
def test_nan_rhs_reported_and_handle_recovers(prec):
    tm = require_gpu()
    dims = (4, 4, 4, 4)
    U = synth.random_su3_field(dims, 0.3, 1001)
    act = oracle.action(dims, KAPPA, MU, EPS)
    sig = synth.shift_set(10, 1e-4, 1.0)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    b = synth.gaussian_rhs(dims, 2001)
    bad = b.copy()
    bad[0, 5, 1, 2, 1] = np.nan
    xs = [g.spinor() for _ in sig]
    with pytest.raises(tm.TmndError) as e:
        tm.mms_cg_solve(g.handle, g.pack(torch.from_numpy(bad).cuda()), 1, sig, xs, prec=prec)
    assert e.value.status == 5, e.value              # TMND_ERR_NAN
    tm.mms_cg_solve(g.handle, g.pack(torch.from_numpy(b).cuda()), 1, sig, xs, prec=prec)
    for i, s in enumerate(sig):
        x = g.unpack(xs[i])[0].cpu().numpy()
        assert oracle.true_residual(act, U, b[0], x, s) <= 1.01e-10, (prec, i)
    g.close()
