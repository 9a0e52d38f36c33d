"""The library's Zolotarev coefficients (host code: arithmetic-geometric-mean
Jacobi elliptic functions) against the oracle's (scipy's elliptic functions from
the closed forms of Sec. 4.1): a, c_k, q_i and delta to 1e-11 relative."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("n,eps", [(1, 0.5), (4, 1e-2), (10, 65e-6 / 4.7), (16, 1e-7), (32, 1e-4)])
def test_zolotarev_coefficients_match_oracle(n, eps):
    from paper_1805_09584_gb300 import _build
    _build.build()
    import paper_1805_09584_gb300 as tm
    a, c, q, d = tm.tmnd_zolotarev(n, eps)
    ar, cr, qr, dr = oracle.zolotarev(n, eps)
    assert abs(a - ar) <= 1e-11 * abs(ar)
    assert np.max(np.abs(c - cr) / np.abs(cr)) <= 1e-11
    assert np.max(np.abs(q - qr) / np.abs(qr)) <= 1e-9
    assert abs(d - dr) <= 1e-9 * dr


def test_zolotarev_rejects_bad_arguments():
    from paper_1805_09584_gb300 import _build
    _build.build()
    import paper_1805_09584_gb300 as tm
    for n, eps in ((0, 0.1), (33, 0.1), (4, 0.0), (4, 1.0)):
        with pytest.raises(RuntimeError):
            tm.tmnd_zolotarev(n, eps)
