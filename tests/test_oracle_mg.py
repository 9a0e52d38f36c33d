"""Pins for the oracle's aggregation multigrid (Sec. 3, 3.2)."""
import numpy as np
import pytest

import oracle
import synth

KAPPA, MU, EPS = 0.16, 0.1, 0.11
DIMS, BDIMS, NV = (4, 4, 4, 4), (2, 2, 2, 2), 4


@pytest.fixture(scope="module")
def setup():
    U = synth.random_su3_field(DIMS, 0.5, 321)
    V = int(np.prod(DIMS))
    rng = np.random.default_rng(7)
    vecs = rng.standard_normal((NV, V, 4, 3)) + 1j * rng.standard_normal((NV, V, 4, 3))
    P = oracle.mg_prolongator(DIMS, BDIMS, vecs)
    act = oracle.action(DIMS, KAPPA, MU, EPS)
    Dcw = oracle.mg_coarse_wilson(act, U, P)
    return U, P, act, Dcw


def _g5(V):
    return np.kron(np.eye(V), np.kron(np.diag([1, 1, -1, -1]), np.eye(3)))


def test_prolongator_orthonormal_and_gamma5_compatible(setup):
    """P^+ P = 1 and Gamma_5 P = P Gamma_5,c (Sec. 3)."""
    U, P, act, _ = setup
    nb = P.shape[1] // (2 * NV)
    assert np.max(np.abs(P.conj().T @ P - np.eye(P.shape[1]))) < 1e-13
    g5c = np.diag(np.tile(np.repeat([1.0, -1.0], NV), nb))
    assert np.max(np.abs(_g5(int(np.prod(DIMS))) @ P - P @ g5c)) < 1e-14


def test_coarse_wilson_gamma5_hermitian_and_stencil(setup):
    """D_c^+ = Gamma_5,c D_c Gamma_5,c (Sec. 3); blocks couple only to themselves
    and nearest-neighbour blocks (a 9-point coarse stencil)."""
    U, P, act, Dcw = setup
    nb = P.shape[1] // (2 * NV)
    g5c = np.diag(np.tile(np.repeat([1.0, -1.0], NV), nb))
    assert np.max(np.abs(Dcw.conj().T - g5c @ Dcw @ g5c)) < 1e-13 * np.abs(Dcw).max()
    nbd = [d // b for d, b in zip(DIMS, BDIMS)]
    coords = np.array(np.unravel_index(np.arange(nb), nbd)).T
    for a in range(nb):
        for b in range(nb):
            d = np.abs(coords[a] - coords[b])
            d = np.minimum(d, np.array(nbd) - d)
            blockab = Dcw[a * 2 * NV:(a + 1) * 2 * NV, b * 2 * NV:(b + 1) * 2 * NV]
            if d.sum() > 1:
                assert np.max(np.abs(blockab)) == 0.0


def test_coarse_nd_structure_and_hermiticity(setup):
    """P_ND = P (x) 1_2 makes the coarse doublet operator keep the fine
    structure (Eq. "non-degenerate_coarse"): P_ND^+ D_ND P_ND equals the formula,
    and it is (Gamma_5,c (x) tau_1)-hermitian (Eq. "g5-t1-hermiticity")."""
    U, P, act, Dcw = setup
    V = int(np.prod(DIMS))
    nb = P.shape[1] // (2 * NV)
    n = nb * 2 * NV
    mu_c, eps_c = 2 * KAPPA * MU, 2 * KAPPA * EPS
    Dnd_c = oracle.mg_coarse_nd(Dcw, nb, NV, mu_c, eps_c)
    # direct projection of the fine doublet operator
    cols = []
    for j in range(2 * n):
        b, rem = divmod(j, 4 * NV)
        f, r = divmod(rem, 2 * NV)
        fine = np.zeros((V, 2, 4, 3), np.complex128)
        fine[:, f] = P[:, b * 2 * NV + r].reshape(V, 4, 3)
        cols.append(oracle.dnd(act, U, fine))
    direct = np.zeros((2 * n, 2 * n), np.complex128)
    for i in range(2 * n):
        b, rem = divmod(i, 4 * NV)
        f, r = divmod(rem, 2 * NV)
        pcol = P[:, b * 2 * NV + r]
        for j in range(2 * n):
            direct[i, j] = np.vdot(pcol, cols[j][:, f].ravel())
    assert np.max(np.abs(direct - Dnd_c)) < 1e-13
    g5c = np.tile(np.repeat([1.0, -1.0], NV), nb)
    G = np.zeros((2 * n, 2 * n))
    for b in range(nb):
        for r in range(2 * NV):
            i0, i1 = b * 4 * NV + r, b * 4 * NV + 2 * NV + r
            G[i0, i1] = G[i1, i0] = g5c[b * 2 * NV + r]
    assert np.max(np.abs(G @ Dnd_c - (G @ Dnd_c).conj().T)) < 1e-13


def test_exact_coarse_grid_correction_annihilates_range_of_P(setup):
    """(1 - P D_c^-1 P^+ D) P = 0 (the coarse-grid correction of Eq.
    "error_propagation" is exact on the range of P)."""
    U, P, act, Dcw = setup
    V = int(np.prod(DIMS))
    DP = np.stack([oracle.wilson_apply(act, U, P[:, j].reshape(V, 4, 3)).ravel() for j in range(P.shape[1])], 1)
    E = P - P @ np.linalg.solve(Dcw, P.conj().T @ DP)
    assert np.max(np.abs(E)) < 1e-10
