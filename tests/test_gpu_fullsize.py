"""Parity at the full sizes the bench times (24^3x48 and 32^3x64), in the same
launch configurations, on what the oracle can compute there:
  * the mixed (and batched) solves: the oracle's own FP64 true residual of sampled
    (shift, RHS) pairs <= 1e-10 (factor 1.01 for summation order);
  * the 16-bit Qhat^2 + sigma at 24^3x48: the oracle's FP64 Qhat^2 of the same field,
    norm-wise 2e-4 (7 roundings of 16-bit data, as in test_gpu_sloppy);
  * the hybrid solve at 32^3x64 with 8 RHS in the bench's configuration (4^4 aggregates,
    24 test vectors per chirality, multi-shift CG for the 8 largest shifts, Lagrange guesses
    and case-C multigrid for the 4 smallest): the oracle's true residual of sampled pairs,
    two of them on the multigrid branch;
  * the tensor-core coarse operator at 32^3x64 (48x48 blocks, 8 RHS): the FP32
    CUDA-core path, which the oracle pins at small sizes, max-norm 4e-3 (TF32)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import EPS, KAPPA, MU, require_gpu, torch

pytestmark = pytest.mark.gpu
SIG = synth.shift_set(12, 1e-5, 2.0)


def test_mixed_24_certified_by_oracle():
    tm = require_gpu()
    dims = (48, 24, 24, 24)
    U = synth.random_su3_field(dims, 0.5, 1003)
    b = synth.gaussian_rhs(dims, 2003, nrhs=2)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    bi = g.pack(torch.from_numpy(b).cuda(), nrhs=2)
    xs = [g.spinor(2) for _ in SIG]
    tm.mms_cg_solve(g.handle, bi, 2, SIG, xs, prec=tm.TMND_S16, batch=1)
    act = oracle.action(dims, KAPPA, MU, EPS)
    for i, k in ((0, 0), (11, 0), (6, 1), (11, 1)):
        x = g.unpack(xs[i], 2)[k].cpu().numpy()
        assert oracle.true_residual(act, U, b[k], x, SIG[i]) <= 1.01e-10, (i, k)
    # 16-bit Qhat^2 + sigma on the same field
    q = g.convert(bi, tm.TMND_F64, tm.TMND_S16, nrhs=2)
    o = g.spinor(2, prec=tm.TMND_S16)
    tm.tm_nd_apply(g.handle, o, q, tm.OP_QHAT2 | tm.OP_S16, 0.0137, nrhs=2)
    got = g.unpack(g.convert(o, tm.TMND_S16, tm.TMND_F64, nrhs=2), 2).cpu().numpy()
    ref = oracle.qhat2(act, U, b[1], 0.0137)
    assert np.linalg.norm(got[1] - ref) <= 2e-4 * np.linalg.norm(ref)
    g.close()


def test_batched_32_certified_by_oracle():
    tm = require_gpu()
    dims = (64, 32, 32, 32)
    U = synth.random_su3_field(dims, 0.5, 1004)
    b = synth.gaussian_rhs(dims, 2004, nrhs=8)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    bi = g.pack(torch.from_numpy(b).cuda(), nrhs=8)
    xs = [g.spinor(8) for _ in SIG]
    tm.mms_cg_solve(g.handle, bi, 8, SIG, xs, prec=tm.TMND_S16, batch=8)
    act = oracle.action(dims, KAPPA, MU, EPS)
    for i, k in ((11, 0), (0, 7), (8, 3)):
        x = g.unpack(xs[i], 8)[k].cpu().numpy()
        assert oracle.true_residual(act, U, b[k], x, SIG[i]) <= 1.01e-10, (i, k)
    g.close()


def test_hybrid_32_certified_by_oracle():
    tm = require_gpu()
    dims, nv = (64, 32, 32, 32), 24
    U = synth.random_su3_field(dims, 0.5, 1004)
    b = synth.gaussian_rhs(dims, 2004, nrhs=8)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    gen = torch.Generator(device="cuda").manual_seed(11)
    tv = torch.randn(nv * 2 * 12 * g.vh, dtype=torch.complex64, device="cuda", generator=gen)
    tm.tmnd_mg_smooth_vectors(g.handle, tv, nv, 4)
    mg = tm.tmnd_mg_create(g.handle, (4, 4, 4, 4), nv, tv)
    del tv
    bi = g.pack(torch.from_numpy(b).cuda(), nrhs=8)
    xs = [g.spinor(8) for _ in SIG]
    # mg_tol 3e-7 of |b|: the Lagrange guess of shift 8 (residual ~3e-6) leaves the case-C
    # multigrid real work; the smaller shifts' guesses may already be below it
    info = tm.tmnd_hybrid_solve(g.handle, mg, bi, 8, SIG, 8, xs, prec=tm.TMND_S16, n_guess=0, guess=1, mg_tol=3e-7)
    assert all(0 < r < 1e-3 for r in info["guess_res"][8:]), info
    assert info["mg_iters"][8] > 0, info
    act = oracle.action(dims, KAPPA, MU, EPS)
    for i, k in ((11, 0), (9, 5), (3, 7), (0, 2)):
        x = g.unpack(xs[i], 8)[k].cpu().numpy()
        assert oracle.true_residual(act, U, b[k], x, SIG[i]) <= 1.01e-10, (i, k)
    tm.tmnd_mg_destroy(mg)
    g.close()


def test_coarse_tc_32_matches_cuda_cores():
    tm = require_gpu()
    dims, nv = (64, 32, 32, 32), 24
    g = tm.Gauge(synth.random_su3_field(dims, 0.5, 1004), dims, KAPPA, MU, EPS)
    gen = torch.Generator(device="cuda").manual_seed(3)
    tv = torch.randn(nv * 2 * 12 * g.vh, dtype=torch.complex64, device="cuda", generator=gen)
    tm.tmnd_mg_smooth_vectors(g.handle, tv, nv, 4)
    mg = tm.tmnd_mg_create(g.handle, (4, 4, 4, 4), nv, tv)
    mgs = tm.tmnd_mg_create(g.handle, (4, 4, 4, 4), nv, tv, coarse_simt=True)
    del tv
    nb = 2 * g.vh // 256
    per = nb * 4 * nv
    x = torch.randn(8 * per, dtype=torch.complex64, device="cuda", generator=gen)
    for s_odd in (0.0, 0.02):
        y_tc, y_s = torch.empty_like(x), torch.empty_like(x)
        tm.mg_coarse_apply(mg, y_tc, x, 8, s_odd)
        for r in range(0, 8, 2):
            tm.mg_coarse_apply(mgs, y_s[r * per:], x[r * per:], 2, s_odd)
        d = (y_tc - y_s).abs().max().item()
        assert d <= 4e-3 * y_s.abs().max().item(), (s_odd, d)
    tm.tmnd_mg_destroy(mg)
    tm.tmnd_mg_destroy(mgs)
    g.close()
