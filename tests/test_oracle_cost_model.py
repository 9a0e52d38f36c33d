"""Pins for the oracle's hybrid cost model (Sec. 4.3, Eqs. "CGtime2",
"MGtime2", "costwo"): with the paper's fitted constants (heavy ND doublet:
lambda_max 4.7, lambda_min 6.5e-5, a = 5.88, b = -1.06; A = 5.0, B = -0.059,
C = 0.024) and its 10-term Zolotarev shifts, the model's optimum is the
printed n_opt = 7; the fits recover the parameters of noise-free data made from
the closed forms."""
import numpy as np

import oracle

CG = (5.88, -1.06, 0.000065, 4.7)
MG = (5.0, -0.059, 0.024, 4.7)


def _paper_shifts():
    a, c, q, d = oracle.zolotarev(10, CG[2] / CG[3])
    return CG[3] * c[1::2]


def test_paper_constants_give_the_printed_optimum():
    cost, n_opt = oracle.hybrid_cost(_paper_shifts(), CG, MG)
    assert n_opt == 7
    # all-CG (n = N) and one MMS shift (n = 1) are both clearly worse
    assert cost[-1] > 1.5 * cost[n_opt - 1] and cost[0] > 1.3 * cost[n_opt - 1]


def test_fits_recover_closed_form_parameters():
    sig = _paper_shifts()
    a, b = oracle.fit_cg_time(sig, oracle.t_cg(sig, *CG), CG[2], CG[3])
    assert abs(a - CG[0]) < 1e-9 and abs(b - CG[1]) < 1e-9
    A, B, C = oracle.fit_mg_time(sig, oracle.t_mg(sig, *MG), MG[3], grid=4001)
    assert abs(C - MG[2]) < 2e-2 * MG[2] and abs(A - MG[0]) < 2e-2 and abs(B - MG[1]) < 2e-2 * abs(MG[1])
