"""Parity of the CUDA stencil (tm_nd_apply) and the spinor packing with the
FP64 oracle, through the C ABI.

Tolerance (FP64): each output component is a sum of O(100) products of
O(1) numbers, so the rounding difference between two summation orders is a
few hundred ulp of the largest term; we require max |gpu - oracle| <=
1e-13 * max |oracle| and the norm-wise relative error <= 1e-14 * 10."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import EPS, KAPPA, MU, rel_err, require_gpu, torch

pytestmark = pytest.mark.gpu

# (dims, roughness): 2 in a direction makes the forward and backward neighbour
# coincide (and exactly one of the two crosses the time boundary); 6^3x8 has
# V/2 = 864, a ragged tail for 128-thread blocks and 32-site packing tiles.
CASES = [((4, 4, 4, 4), 0.3), ((2, 2, 2, 4), 0.7), ((6, 6, 6, 8), 0.5), ((8, 4, 6, 2), 0.5), ((8, 8, 8, 8), 0.5)]


def _setup(dims, r, seed=1):
    tm = require_gpu()
    U = synth.random_su3_field(dims, r, 1000 + seed)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    return tm, U, g


@pytest.mark.parametrize("dims,r", CASES)
def test_pack_unpack_roundtrip_bit_exact(dims, r):
    tm, U, g = _setup(dims, r)
    b = synth.gaussian_rhs(dims, 7, nrhs=2)
    bc = torch.from_numpy(b).cuda()
    bi = g.pack(bc, nrhs=2)
    # internal plane layout: element (c, h) of rhs k at k*24*Vh + c*Vh + h
    vh = g.vh
    host = bi.cpu().numpy().reshape(2, 24, vh)
    assert np.array_equal(host, b.reshape(2, vh, 24).transpose(0, 2, 1))
    back = g.unpack(bi, nrhs=2).cpu().numpy()
    assert np.array_equal(back, b)
    g.close()


@pytest.mark.parametrize("dims,r", CASES)
@pytest.mark.parametrize("op", ["mhat", "mhat_dag", "qhat2", "qhat"])
def test_apply_matches_oracle(dims, r, op):
    tm, U, g = _setup(dims, r)
    act = oracle.action(dims, KAPPA, MU, EPS)
    b = synth.gaussian_rhs(dims, 11)[0]
    sigma = 0.0137
    ref = {"mhat": lambda: oracle.schur(act, U, b),
           "mhat_dag": lambda: oracle.schur(act, U, b, dagger=True),
           "qhat2": lambda: oracle.qhat2(act, U, b, sigma),
           "qhat": lambda: oracle.qhat(act, U, b)}[op]()
    code = {"mhat": tm.OP_MHAT, "mhat_dag": tm.OP_MHAT_DAG, "qhat2": tm.OP_QHAT2, "qhat": tm.OP_QHAT}[op]
    bi = g.pack(torch.from_numpy(b).cuda())
    out = g.spinor()
    tm.tm_nd_apply(g.handle, out, bi, code, sigma)
    got = g.unpack(out)[0].cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    assert rel_err(got, ref) <= 1e-14 * 10
    g.close()


def test_apply_multi_rhs_and_periodic_time():
    tm = require_gpu()
    dims = (4, 4, 2, 6)
    U = synth.random_su3_field(dims, 0.5, 5)
    for apbc in (True, False):
        act = oracle.action(dims, KAPPA, MU, EPS, apbc=apbc)
        g = tm.Gauge(U, dims, KAPPA, MU, EPS, antiperiodic_t=apbc)
        b = synth.gaussian_rhs(dims, 3, nrhs=3)
        bi = g.pack(torch.from_numpy(b).cuda(), nrhs=3)
        out = g.spinor(3)
        tm.tm_nd_apply(g.handle, out, bi, tm.OP_QHAT2, 0.5, nrhs=3)
        got = g.unpack(out, nrhs=3).cpu().numpy()
        for k in range(3):
            ref = oracle.qhat2(act, U, b[k], 0.5)
            assert rel_err(got[k], ref) <= 1e-13
        g.close()


def test_apply_zero_and_unit_gauge():
    """Degenerate inputs: a zero vector maps to zero; the free field (U = 1)."""
    tm = require_gpu()
    dims = (4, 2, 2, 4)
    U = synth.unit_gauge_field(dims)
    act = oracle.action(dims, KAPPA, MU, EPS)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    z = g.spinor()
    z.zero_()
    out = g.spinor()
    tm.tm_nd_apply(g.handle, out, z, tm.OP_QHAT2, 1.0)
    assert torch.count_nonzero(out).item() == 0
    b = synth.gaussian_rhs(dims, 1)[0]
    tm.tm_nd_apply(g.handle, out, g.pack(torch.from_numpy(b).cuda()), tm.OP_MHAT)
    assert rel_err(g.unpack(out)[0].cpu().numpy(), oracle.schur(act, U, b)) < 1e-14
    g.close()


def test_full_size_qhat2_bench_lattice():
    """16^3x32, roughness 0.5 (the bench workload's lattice): every element of
    (Qhat^2 + sigma) b against the oracle."""
    tm = require_gpu()
    dims = (32, 16, 16, 16)
    U = synth.random_su3_field(dims, 0.5, 1002)
    act = oracle.action(dims, KAPPA, MU, EPS)
    b = synth.gaussian_rhs(dims, 2032)[0]
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    out = g.spinor()
    tm.tm_nd_apply(g.handle, out, g.pack(torch.from_numpy(b).cuda()), tm.OP_QHAT2, 1e-5)
    got = g.unpack(out)[0].cpu().numpy()
    ref = oracle.qhat2(act, U, b, 1e-5)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    g.close()
