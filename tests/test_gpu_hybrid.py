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


@pytest.mark.parametrize("prec", [0, 2])
def test_hybrid_certified(prec):
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
    info = tm.tmnd_hybrid_solve(g.handle, mg, bi, 1, sig, 6, xs, prec=prec)
    for i, s in enumerate(sig):
        x = g.unpack(xs[i])[0].cpu().numpy()
        tr = oracle.true_residual(act, U, b[0], x, s)
        assert tr <= 1.01e-10, (i, tr, info)
    # the guesses of the MG shifts are better than the zero start (Sec. 4.2.1: bound < 1)
    assert all(0 < r < 1 for r in info["guess_res"][6:]), info
    tm.tmnd_mg_destroy(mg)
    g.close()
