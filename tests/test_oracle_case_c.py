"""Pins for the oracle's case-C operators (Sec. 3.1, Eq. "lindif"; Sec. 3.2).

The multigrid solves (Qhat +- i s) y = b as the full-lattice system
D' = D_ND + i s (gamma_5 (x) tau_1) Pi_odd, whose odd Schur complement is
Mhat + i s gamma_5 tau_1 (reading of the even-odd reduction of Sec. 2), and
its coarse image P_ND^+ D' P_ND.  These tests fix both against the
independently pinned Qhat, the Eq. "non-degenerate_coarse" formula and
identities of the aggregation (Gamma_5 P = P Gamma_5,c, P^+ P = 1), so that a
wrong sign of i s, a missing flavour swap, the term on the wrong parity or a
transposed projection fails one of them."""
import numpy as np
import pytest

import oracle
import synth

KAPPA, MU, EPS = 0.16, 0.1, 0.11


def _parity(dims):
    T, X, Y, Z = dims
    t, x, y, z = np.meshgrid(np.arange(T), np.arange(X), np.arange(Y), np.arange(Z), indexing="ij")
    return ((t + x + y + z) & 1).ravel()


def _g5t1_odd(psi):
    """(gamma_5 (x) tau_1) on an odd-site vector [V/2, 2, 4, 3]."""
    g5 = np.array([1.0, 1.0, -1.0, -1.0])
    return g5[None, None, :, None] * psi[:, ::-1]


@pytest.mark.parametrize("s", [0.05, -0.05])
def test_schur_complement_of_odd_shift_is_qhat_plus_is(oracle_lib, s):
    """(gamma_5 (x) tau_1) [D'_oo - D'_oe D'_ee^-1 D'_eo] = Qhat + i s on a rough
    4x2x2x4 field: the odd-site term i s gamma_5 tau_1 becomes the shift of the
    hermitian Qhat after the even sites are eliminated (numpy inverse of the
    dense even-even block; Qhat from the oracle's own, separately pinned stencil)."""
    dims = (4, 2, 2, 4)
    U = synth.random_su3_field(dims, 0.5, 777)
    act = oracle.action(dims, KAPPA, MU, EPS)
    V = int(np.prod(dims))
    n = V * 24
    Dp = oracle.dense(lambda v: oracle.dnd_odd_shift(act, U, v.reshape(V, 2, 4, 3), s), n)
    par = np.repeat(_parity(dims), 24)
    o, e = np.nonzero(par == 1)[0], np.nonzero(par == 0)[0]
    schur = Dp[np.ix_(o, o)] - Dp[np.ix_(o, e)] @ np.linalg.solve(Dp[np.ix_(e, e)], Dp[np.ix_(e, o)])
    vh = V // 2
    g5t1 = oracle.dense(lambda v: _g5t1_odd(v.reshape(vh, 2, 4, 3)), vh * 24)
    Q = oracle.dense(lambda v: oracle.qhat(act, U, v.reshape(vh, 2, 4, 3)), vh * 24)
    lhs = g5t1 @ schur
    assert np.max(np.abs(lhs - (Q + 1j * s * np.eye(vh * 24)))) < 1e-12 * np.abs(Q).max()
    # the term acts on odd sites only: the even-even block is that of D_ND
    D0 = oracle.dense(lambda v: oracle.dnd(act, U, v.reshape(V, 2, 4, 3)), n)
    assert np.max(np.abs(Dp[np.ix_(e, e)] - D0[np.ix_(e, e)])) == 0.0
    assert np.max(np.abs(Dp[np.ix_(o, e)] - D0[np.ix_(o, e)])) == 0.0


DIMS, BDIMS, NV = (4, 4, 4, 4), (2, 2, 2, 2), 4


@pytest.fixture(scope="module")
def coarse(oracle_lib):
    U = synth.random_su3_field(DIMS, 0.5, 321)
    V = int(np.prod(DIMS))
    rng = np.random.default_rng(7)
    vecs = rng.standard_normal((NV, V, 4, 3)) + 1j * rng.standard_normal((NV, V, 4, 3))
    P = oracle.mg_prolongator(DIMS, BDIMS, vecs)
    act = oracle.action(DIMS, KAPPA, MU, EPS)
    Dcw = oracle.mg_coarse_wilson(act, U, P)
    nb = P.shape[1] // (2 * NV)
    return dict(U=U, P=P, act=act, Dcw=Dcw, nb=nb, V=V)


def _flavour_blockdiag(A, nb, nv, off=False):
    """A [nb 2nv, nb 2nv] (single-flavour coarse) -> doublet coarse layout, on the
    flavour diagonal (A (x) 1_2) or off it (A (x) tau_1)."""
    n2 = 2 * nv
    out = np.zeros((2 * nb * n2, 2 * nb * n2), np.complex128)
    b = np.repeat(np.arange(nb), n2)
    r = np.tile(np.arange(n2), nb)
    i0, i1 = b * 2 * n2 + r, b * 2 * n2 + n2 + r
    if off:
        out[np.ix_(i0, i1)] = A
        out[np.ix_(i1, i0)] = A
    else:
        out[np.ix_(i0, i0)] = A
        out[np.ix_(i1, i1)] = A
    return out


def test_coarse_odd_shift_at_zero_is_eq_non_degenerate_coarse(coarse):
    """s = 0: the probed P_ND^+ D_ND P_ND equals Eq. "non-degenerate_coarse"."""
    c = coarse
    Dc0 = oracle.mg_coarse_nd_odd_shift(c["act"], c["U"], c["P"], NV, 0.0)
    ref = oracle.mg_coarse_nd(c["Dcw"], c["nb"], NV, 2 * KAPPA * MU, 2 * KAPPA * EPS)
    assert np.max(np.abs(Dc0 - ref)) < 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("s", [0.03, -0.2])
def test_coarse_odd_shift_term(coarse, s):
    """D'_c(s) - D'_c(0) = i s tau_1 (x) (P^+ Pi_odd P) Gamma_5,c: aggregate-local,
    flavour off-diagonal, linear in s.  The right side uses Gamma_5 P = P Gamma_5,c
    (Sec. 3) to move gamma_5 past P, so it never applies gamma_5 on the fine grid."""
    c = coarse
    P, nb, V = c["P"], c["nb"], c["V"]
    Dcs = oracle.mg_coarse_nd_odd_shift(c["act"], c["U"], P, NV, s)
    Dc0 = oracle.mg_coarse_nd_odd_shift(c["act"], c["U"], P, NV, 0.0)
    odd = np.repeat(_parity(DIMS) == 1, 12)
    PoP = P.conj().T @ (odd[:, None] * P)
    g5c = np.tile(np.repeat([1.0, -1.0], NV), nb)
    term = _flavour_blockdiag(1j * s * PoP * g5c[None, :], nb, NV, off=True)
    assert np.max(np.abs((Dcs - Dc0) - term)) < 1e-13
    # aggregate-local: P^+ Pi_odd P couples a block only to itself
    n2 = 2 * NV
    for a in range(nb):
        for b in range(nb):
            if a != b:
                assert np.max(np.abs(PoP[a * n2:(a + 1) * n2, b * n2:(b + 1) * n2])) < 1e-15
    # half of each aggregate is odd: P^+ Pi_odd P + P^+ Pi_even P = P^+ P = 1
    PeP = P.conj().T @ ((~odd)[:, None] * P)
    assert np.max(np.abs(PoP + PeP - np.eye(P.shape[1]))) < 1e-13


def test_coarse_odd_shift_antihermitian_part(coarse):
    """(Gamma_5,c (x) tau_1) D'_c = hermitian + i s (1 (x) P^+ Pi_odd P): the fine
    gamma_5 tau_1 D_ND is hermitian (Eq. "g5tau1-hermiticity") and gamma_5 tau_1 times
    the shift term is i s Pi_odd, so the anti-hermitian part of the coarse product is
    i s P^+ Pi_odd P on both flavours (its sign fixes the sign of s)."""
    c = coarse
    P, nb = c["P"], c["nb"]
    s = 0.07
    Dcs = oracle.mg_coarse_nd_odd_shift(c["act"], c["U"], P, NV, s)
    g5c = np.tile(np.repeat([1.0, -1.0], NV), nb)
    G = _flavour_blockdiag(np.diag(g5c).astype(np.complex128), nb, NV, off=True)
    GD = G @ Dcs
    ah = (GD - GD.conj().T) / 2
    odd = np.repeat(_parity(DIMS) == 1, 12)
    PoP = P.conj().T @ (odd[:, None] * P)
    assert np.max(np.abs(ah - _flavour_blockdiag(1j * s * PoP, nb, NV))) < 1e-13


def test_coarse_odd_shift_exact_coarse_grid_correction(coarse):
    """(1 - P_ND D'_c^-1 P_ND^+ D') P_ND = 0 (Eq. "error_propagation" with the case-C
    operator): the probed coarse operator is the Galerkin projection of D'."""
    c = coarse
    P, V, nb = c["P"], c["V"], c["nb"]
    s = 0.05
    Dcs = oracle.mg_coarse_nd_odd_shift(c["act"], c["U"], P, NV, s)
    ncol = P.shape[1]
    # P_ND as a dense matrix on [V, 2 flavour, 12] fine vectors
    PND = np.zeros((V * 24, 2 * ncol), np.complex128)
    for j in range(2 * ncol):
        b, rem = divmod(j, 4 * NV)
        f, r = divmod(rem, 2 * NV)
        col = np.zeros((V, 2, 12), np.complex128)
        col[:, f] = P[:, b * 2 * NV + r].reshape(V, 12)
        PND[:, j] = col.ravel()
    DPND = np.stack([oracle.dnd_odd_shift(c["act"], c["U"], PND[:, j].reshape(V, 2, 4, 3), s).ravel()
                     for j in range(2 * ncol)], 1)
    E = PND - PND @ np.linalg.solve(Dcs, PND.conj().T @ DPND)
    assert np.max(np.abs(E)) < 1e-10
