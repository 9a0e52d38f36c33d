"""The library's hybrid cost model and fits (host code, Sec. 4.3) against the
oracle's: c_HY(n), n_opt (the paper's constants and 10-term Zolotarev shifts
give n_opt = 7), and the parameters fitted to noise-free closed-form data."""
import numpy as np

import oracle

CG = (5.88, -1.06, 0.000065, 4.7)
MG = (5.0, -0.059, 0.024, 4.7)


def _lib():
    from paper_1805_09584_gb300 import _build
    _build.build()
    import paper_1805_09584_gb300 as tm
    return tm


def test_cost_and_fits_match_oracle():
    tm = _lib()
    a, c, q, d = oracle.zolotarev(10, CG[2] / CG[3])
    sig = CG[3] * c[1::2]
    cost, n = tm.tmnd_hybrid_cost(sig, CG, MG)
    cref, nref = oracle.hybrid_cost(sig, CG, MG)
    assert n == nref == 7
    assert np.max(np.abs(cost - cref) / np.abs(cref)) < 1e-13
    fa, fb = tm.tmnd_fit_cg_time(sig, oracle.t_cg(sig, *CG), CG[2], CG[3])
    assert abs(fa - CG[0]) < 1e-9 and abs(fb - CG[1]) < 1e-9
    A, B, C = tm.tmnd_fit_mg_time(sig, oracle.t_mg(sig, *MG), MG[3], 4001)
    Ar, Br, Cr = oracle.fit_mg_time(sig, oracle.t_mg(sig, *MG), MG[3], grid=4001)
    assert abs(C - Cr) <= 1e-6 * Cr and abs(A - Ar) < 1e-6 and abs(B - Br) < 1e-6
