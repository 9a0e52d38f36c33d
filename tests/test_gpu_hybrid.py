"""Hybrid solve (Sec. 4.3): multi-shift CG for the largest shifts with guess
shifts iterated along (Sec. 4.2.2), Lagrange guesses (Sec. 4.2.1) and case-C
multigrid solves (Sec. 3.1, Eq. "lindif"; Sec. 3) for the smallest, every shift
finished by FP64 defect correction.  Certified by the oracle's true residual."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import EPS, KAPPA, MU, require_gpu, torch
from test_gpu_mg import to_mg_layout

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,lebesgue_max", [(0, 0.0), (2, 0.0), (2, 1.5)])
def test_hybrid_certified(prec, lebesgue_max):
    tm = require_gpu()
    dims, bdims, nv = (8, 4, 4, 4), (2, 2, 2, 2), 6
    V = int(np.prod(dims))
    U = synth.random_su3_field(dims, 0.5, 41)
    act = oracle.action(dims, KAPPA, MU, EPS)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    rng = np.random.default_rng(4)
    tv = rng.standard_normal((nv, V, 12)) + 1j * rng.standard_normal((nv, V, 12))
    tvd = torch.from_numpy(to_mg_layout(dims, tv.astype(np.complex64), 12)).cuda().contiguous()
    tm.tmnd_mg_smooth_vectors(g.handle, tvd, nv, 6)
    mg = tm.tmnd_mg_create(g.handle, bdims, nv, tvd)
    b = synth.gaussian_rhs(dims, 9)
    sig = synth.shift_set(10, 1e-4, 1.0)
    bi = g.pack(torch.from_numpy(b).cuda())
    xs = [g.spinor() for _ in sig]
    info = tm.tmnd_hybrid_solve(g.handle, mg, bi, 1, sig, 6, xs, prec=prec, lebesgue_max=lebesgue_max)
    # Lagrange nodes of shifts 8, 9 (after 6 multi-shift and 2 guess shifts): the nearest solved
    # shifts, truncated where the Lebesgue function exceeds lebesgue_max (App. B), as the oracle picks
    for i in (8, 9):
        cand = sig[:i][::-1][:8]
        k_ref, g_ref = oracle.lagrange_degree(cand, sig[i], lebesgue_max or 4.0)
        assert info["lag_nodes"][i] == k_ref and abs(info["lebesgue"][i] - g_ref) < 1e-12 * g_ref, info
    if lebesgue_max == 1.5:
        assert info["lag_nodes"][8] < 8
    for i, s in enumerate(sig):
        x = g.unpack(xs[i])[0].cpu().numpy()
        tr = oracle.true_residual(act, U, b[0], x, s)
        assert tr <= 1.01e-10, (i, tr, info)
    # the guesses of the MG shifts are better than the zero start (Sec. 4.2.1: bound < 1)
    assert all(0 < r < 1 for r in info["guess_res"][6:]), info
    tm.tmnd_mg_destroy(mg)
    g.close()


def test_hybrid_learned_and_lagrange_guesses_without_mg():
    """No multigrid: the 4 smallest shifts start from Lagrange (guess 1) or
    learned (guess 2, a network trained here on solves of other fields) guesses
    and finish by FP64 defect correction; every shift certified by the oracle."""
    tm = require_gpu()
    from paper_1805_09584_gb300 import learned
    dims = (4, 4, 4, 4)
    sig = synth.shift_set(12, 1e-5, 2.0)
    Xs, Ss, Hs = [], [], []
    for fs in range(4):
        gauge = tm.Gauge(synth.random_su3_field(dims, 0.3 + 0.1 * fs, 300 + fs), dims, KAPPA, MU, EPS)
        for k, bk in enumerate(synth.gaussian_rhs(dims, 400 + fs, nrhs=2)):
            bd = gauge.pack(torch.from_numpy(bk[None]).cuda())
            xs, info, hist = learned.solve_nodes(gauge, bd, sig, prec=tm.TMND_S16)
            X, S, H = learned.samples(gauge, bd, sig, xs, info, hist)
            Xs.append(X); Ss.append(S); Hs.append(H)
        gauge.close()
    net, _ = learned.train(np.concatenate(Xs), np.concatenate(Ss), np.concatenate(Hs), epochs=300)
    U = synth.random_su3_field(dims, 0.45, 333)
    act = oracle.action(dims, KAPPA, MU, EPS)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    b = synth.gaussian_rhs(dims, 444, nrhs=2)
    bi = g.pack(torch.from_numpy(b).cuda(), nrhs=2)
    for guess, kw in ((1, {}), (2, {"net": net})):
        xs = [g.spinor(2) for _ in sig]
        info = tm.tmnd_hybrid_solve(g.handle, None, bi, 2, sig, 8, xs, prec=tm.TMND_S16, n_guess=0, guess=guess, **kw)
        for i, s in enumerate(sig):
            x = g.unpack(xs[i], 2).cpu().numpy()
            for k in range(2):
                tr = oracle.true_residual(act, U, b[k], x[k], s)
                assert tr <= 1.01e-10, (guess, i, k, tr, info)
        assert all(0 < r < 1e-3 for r in info["guess_res"][8:]), (guess, info)
    tm.tmnd_mlp_destroy(net)
    g.close()
