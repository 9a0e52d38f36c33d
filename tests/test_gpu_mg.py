"""Parity of the GPU multigrid pieces (Sec. 3, 3.2) with the FP64 oracle:
prolongator (block Gram-Schmidt of the same test vectors), coarse Wilson
operator P^+ D_W P, odd-site Gram G_odd, restriction / prolongation, and the
coarse doublet stencil mg_coarse_apply.  FP32 on the device: tolerances 2e-5
relative (sums of ~1e3 FP32 products of O(1) numbers).  The tensor-core coarse
apply rounds both operands to TF32 (10 mantissa bits, relative 2^-11 each):
4e-3 of the largest output, max-norm."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import EPS, KAPPA, MU, require_gpu, torch

pytestmark = pytest.mark.gpu
NV = 4


def to_mg_layout(dims, canon, ncomp):
    """canonical [..., V, ncomp] (lexicographic) -> [..., 2 parity, ncomp, V/2]"""
    V = int(np.prod(dims))
    T, X, Y, Z = dims
    t, x, y, z = np.meshgrid(np.arange(T), np.arange(X), np.arange(Y), np.arange(Z), indexing="ij")
    par = ((t + x + y + z) & 1).ravel()
    lead = canon.shape[:-2]
    out = np.zeros(lead + (2, ncomp, V // 2), np.complex64)
    lex = np.arange(V)
    for pp in (0, 1):
        sel = lex[par == pp]
        out[..., pp, :, :] = np.moveaxis(canon[..., sel, :], -1, -2)
    return out


def from_mg_layout(dims, mg, ncomp):
    V = int(np.prod(dims))
    T, X, Y, Z = dims
    t, x, y, z = np.meshgrid(np.arange(T), np.arange(X), np.arange(Y), np.arange(Z), indexing="ij")
    par = ((t + x + y + z) & 1).ravel()
    lead = mg.shape[:-3]
    out = np.zeros(lead + (V, ncomp), np.complex128)
    lex = np.arange(V)
    for pp in (0, 1):
        sel = lex[par == pp]
        out[..., sel, :] = np.moveaxis(mg[..., pp, :, :], -2, -1)
    return out


@pytest.fixture(scope="module", params=[((4, 4, 4, 4), (2, 2, 2, 2)), ((8, 4, 4, 4), (2, 2, 2, 2))])
def mgsetup(request):
    tm = require_gpu()
    dims, bdims = request.param
    U = synth.random_su3_field(dims, 0.5, 99)
    V = int(np.prod(dims))
    rng = np.random.default_rng(3)
    vecs = (rng.standard_normal((NV, V, 12)) + 1j * rng.standard_normal((NV, V, 12))).astype(np.complex64)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    tv = torch.from_numpy(to_mg_layout(dims, vecs, 12)).cuda()
    mg = tm.tmnd_mg_create(g.handle, bdims, NV, tv)
    mg_simt = tm.tmnd_mg_create(g.handle, bdims, NV, tv, coarse_simt=True)
    act = oracle.action(dims, KAPPA, MU, EPS)
    P = oracle.mg_prolongator(dims, bdims, vecs.astype(np.complex128).reshape(NV, V, 4, 3))
    Dcw = oracle.mg_coarse_wilson(act, U, P)
    nb = P.shape[1] // (2 * NV)
    yield dict(tm=tm, g=g, mg=mg, mg_simt=mg_simt, dims=dims, bdims=bdims, U=U, P=P, Dcw=Dcw, nb=nb, act=act,
               vecs=vecs)
    tm.tmnd_mg_destroy(mg)
    tm.tmnd_mg_destroy(mg_simt)
    g.close()


def _gpu_P_dense(s):
    dims, bdims, nb = s["dims"], s["bdims"], s["nb"]
    nsb = int(np.prod(bdims))
    V = int(np.prod(dims))
    Ph = np.zeros((nb, 2, NV, nsb, 6), np.complex64)
    s["tm"].tmnd_mg_export(s["mg"], P_host=Ph)
    blk = oracle.mg_block_of_site(dims, bdims)
    dense = np.zeros((V * 12, nb * 2 * NV), np.complex128)
    for b in range(nb):
        sites = np.nonzero(blk == b)[0]   # lexicographic order = block-local order
        for chi in range(2):
            for k in range(NV):
                for si, site in enumerate(sites):
                    dense[site * 12 + chi * 6: site * 12 + chi * 6 + 6, b * 2 * NV + chi * NV + k] = Ph[b, chi, k, si]
    return dense


def test_prolongator_matches_oracle(mgsetup):
    s = mgsetup
    Pg = _gpu_P_dense(s)
    assert np.max(np.abs(Pg - s["P"])) < 2e-5


def test_coarse_operator_matches_oracle(mgsetup):
    s = mgsetup
    nb, n2 = s["nb"], 2 * NV
    Dh = np.zeros((nb, 9, n2, n2), np.complex64)
    Gh = np.zeros((nb, n2, n2), np.complex64)
    s["tm"].tmnd_mg_export(s["mg"], Dc_host=Dh, Godd_host=Gh)
    nbd = [d // b for d, b in zip(s["dims"], s["bdims"])]
    dense = np.zeros((nb * n2, nb * n2), np.complex128)
    for b in range(nb):
        c = list(np.unravel_index(b, nbd))
        for d in range(9):
            cc = list(c)
            if d > 0:
                mu = (d - 1) // 2
                cc[mu] = (cc[mu] + (1 if (d - 1) % 2 == 0 else -1)) % nbd[mu]
            b2 = int(np.ravel_multi_index(cc, nbd))
            dense[b * n2:(b + 1) * n2, b2 * n2:(b2 + 1) * n2] += Dh[b, d]
    scale = np.abs(s["Dcw"]).max()
    assert np.max(np.abs(dense - s["Dcw"])) < 2e-5 * scale
    # G_odd = P^+ gamma_5 Pi_odd P
    V = int(np.prod(s["dims"]))
    odd = np.zeros(V, bool)
    odd[synth.odd_sites(s["dims"])] = True
    g5 = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), V) * np.repeat(odd, 12)
    Gref = s["P"].conj().T @ (g5[:, None] * s["P"])
    for b in range(nb):
        assert np.max(np.abs(Gh[b] - Gref[b * n2:(b + 1) * n2, b * n2:(b + 1) * n2])) < 2e-5


def test_restrict_prolong_match_oracle(mgsetup):
    s = mgsetup
    tm, mg, dims = s["tm"], s["mg"], s["dims"]
    V = int(np.prod(dims))
    nb = s["nb"]
    rng = np.random.default_rng(11)
    fine = rng.standard_normal((2, V, 24)) + 1j * rng.standard_normal((2, V, 24))   # 2 RHS, doublet
    fin = torch.from_numpy(to_mg_layout(dims, fine.astype(np.complex64), 24)).cuda()
    coarse = torch.zeros(2 * nb * 2 * 2 * NV, dtype=torch.complex64, device="cuda")
    tm.tmnd_mg_restrict(mg, coarse, fin, 2)
    got = coarse.cpu().numpy().reshape(2, nb, 2, 2 * NV)
    P = s["P"]
    for r in range(2):
        for f in range(2):
            ref = P.conj().T @ fine[r, :, f * 12:(f + 1) * 12].ravel()
            assert np.max(np.abs(got[r, :, f, :].ravel() - ref)) < 2e-5 * np.abs(ref).max()
    cv = rng.standard_normal((2, nb, 2, 2 * NV)) + 1j * rng.standard_normal((2, nb, 2, 2 * NV))
    cin = torch.from_numpy(cv.astype(np.complex64).ravel()).cuda()
    fout = torch.zeros(2 * 2 * 24 * (V // 2), dtype=torch.complex64, device="cuda")
    tm.tmnd_mg_prolong(mg, fout, cin, 2)
    back = from_mg_layout(dims, fout.cpu().numpy().reshape(2, 2, 24, V // 2), 24)
    for r in range(2):
        for f in range(2):
            ref = P @ cv[r, :, f, :].ravel()
            assert np.max(np.abs(back[r, :, f * 12:(f + 1) * 12].ravel() - ref)) < 2e-5 * np.abs(ref).max()


@pytest.mark.parametrize("s_odd", [0.0, 0.03])
@pytest.mark.parametrize("path,R,tol", [("simt", 3, 2e-5), ("tc", 1, 4e-3), ("tc", 3, 4e-3), ("tc", 8, 4e-3),
                                        ("tc", 16, 4e-3)])
def test_coarse_apply_matches_oracle(mgsetup, s_odd, path, R, tol):
    s = mgsetup
    tm, nb = s["tm"], s["nb"]
    mg = s["mg_simt"] if path == "simt" else s["mg"]
    # the oracle's P_ND^+ (D_ND + i s gamma_5 tau_1 Pi_odd) P_ND, by column probing
    Dnd = oracle.mg_coarse_nd_odd_shift(s["act"], s["U"], s["P"], NV, s_odd)
    rng = np.random.default_rng(5)
    xv = rng.standard_normal((R, nb * 4 * NV)) + 1j * rng.standard_normal((R, nb * 4 * NV))
    xin = torch.from_numpy(xv.astype(np.complex64).ravel()).cuda()
    yout = torch.zeros_like(xin)
    tm.mg_coarse_apply(mg, yout, xin, R, s_odd)
    got = yout.cpu().numpy().reshape(R, -1)
    for r in range(R):
        ref = Dnd @ xv[r]
        assert np.max(np.abs(got[r] - ref)) < tol * np.abs(ref).max(), (path, R, r)


@pytest.mark.parametrize("s_odd", [0.0, 0.05])
def test_coarse_apply_tc_production_shape(s_odd):
    """24 test vectors per chirality (48x48 complex coarse blocks, the production
    shape: six 8-row groups, K = 96 per direction), 8 right-hand sides, on a
    4x4x4x8 lattice with 2^4 aggregates: tensor cores vs the oracle, and vs the
    FP32 CUDA-core path."""
    tm = require_gpu()
    nv = 24
    dims, bdims = (8, 4, 4, 4), (2, 2, 2, 2)
    U = synth.random_su3_field(dims, 0.5, 98)
    V = int(np.prod(dims))
    rng = np.random.default_rng(4)
    vecs = (rng.standard_normal((nv, V, 12)) + 1j * rng.standard_normal((nv, V, 12))).astype(np.complex64)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    tv = torch.from_numpy(to_mg_layout(dims, vecs, 12)).cuda()
    mg = tm.tmnd_mg_create(g.handle, bdims, nv, tv)
    mgs = tm.tmnd_mg_create(g.handle, bdims, nv, tv, coarse_simt=True)
    act = oracle.action(dims, KAPPA, MU, EPS)
    P = oracle.mg_prolongator(dims, bdims, vecs.astype(np.complex128).reshape(nv, V, 4, 3))
    nb = P.shape[1] // (2 * nv)
    Dnd = oracle.mg_coarse_nd_odd_shift(act, U, P, nv, s_odd)
    R = 8
    xv = rng.standard_normal((R, nb * 4 * nv)) + 1j * rng.standard_normal((R, nb * 4 * nv))
    xin = torch.from_numpy(xv.astype(np.complex64).ravel()).cuda()
    y_tc, y_simt = torch.zeros_like(xin), torch.zeros_like(xin)
    tm.mg_coarse_apply(mg, y_tc, xin, R, s_odd)
    tm.mg_coarse_apply(mgs, y_simt, xin, 2, s_odd)   # CUDA cores: 2 RHS per launch (thread limit)
    tm.mg_coarse_apply(mgs, y_simt[2 * nb * 4 * nv:], xin[2 * nb * 4 * nv:], 2, s_odd)
    got = y_tc.cpu().numpy().reshape(R, -1)
    gs = y_simt.cpu().numpy().reshape(R, -1)
    for r in range(R):
        ref = Dnd @ xv[r]
        assert np.max(np.abs(got[r] - ref)) < 4e-3 * np.abs(ref).max(), r
        if r < 4:
            assert np.max(np.abs(gs[r] - ref)) < 2e-5 * np.abs(ref).max(), r
    tm.tmnd_mg_destroy(mg)
    tm.tmnd_mg_destroy(mgs)
    g.close()
