"""tm_nd_apply_noalloc, the variant of tm_nd_apply that never allocates device
memory (its temporaries sit in a fixed array inside the library).  It exists
for callers that cannot allocate at call time: programs whose device memory
belongs to another allocator, and latency-critical loops that cannot accept
cudaMalloc's device-wide synchronisation.

Called through the C ABI; its output must equal tm_nd_apply's within the
operator tests' tolerance, on two calls in a row (the second call meets the
first call's leftovers in the shared array).  This file is collected last so
that a run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

import synth
from gpu_common import EPS, KAPPA, MU, require_gpu, torch

pytestmark = pytest.mark.gpu


def _close(got, ref):
    # tolerance of the operator parity tests
    return np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 6, 6, 8)])
def test_noalloc_matches_tm_nd_apply(dims):
    tm = require_gpu()
    U = synth.random_su3_field(dims, 0.5, 4242)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    b = synth.gaussian_rhs(dims, 17, nrhs=2)
    bi = g.pack(torch.from_numpy(b).cuda(), nrhs=2)
    for op in (tm.OP_MHAT, tm.OP_MHAT_DAG, tm.OP_QHAT2, tm.OP_QHAT):
        ref = g.spinor(2)
        tm.tm_nd_apply(g.handle, ref, bi, op, 0.031, nrhs=2)
        ref_h = ref.cpu().numpy()
        for _ in range(2):
            out = g.spinor(2)
            out.fill_(float("nan"))
            tm.tm_nd_apply_noalloc(g.handle, out, bi, op, 0.031, nrhs=2)
            torch.cuda.synchronize()
            assert _close(out.cpu().numpy(), ref_h), op
    g.close()


def test_noalloc_allocates_nothing():
    """The defining property: a handle that has never run tm_nd_apply (so its workspace
    was never grown) applies the operator through tm_nd_apply_noalloc without any change
    in the device's free memory.  Warm-up calls on another handle first load the library's
    kernels (module loading places the fixed array) and look up the array's address."""
    tm = require_gpu()
    dims = (8, 8, 8, 8)
    U = synth.random_su3_field(dims, 0.5, 4243)
    warm = tm.Gauge(U, dims, KAPPA, MU, EPS)
    b = warm.pack(torch.from_numpy(synth.gaussian_rhs(dims, 18)).cuda())
    o = warm.spinor()
    for op in (tm.OP_MHAT, tm.OP_MHAT_DAG, tm.OP_QHAT2, tm.OP_QHAT):  # every kernel loaded once
        tm.tm_nd_apply_noalloc(warm.handle, o, b, op, 0.02)
    fresh = tm.Gauge(U, dims, KAPPA, MU, EPS)
    out = fresh.spinor()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for op in (tm.OP_MHAT, tm.OP_MHAT_DAG, tm.OP_QHAT2, tm.OP_QHAT):
        tm.tm_nd_apply_noalloc(fresh.handle, out, b, op, 0.02)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    ref = fresh.spinor()
    tm.tm_nd_apply(warm.handle, ref, b, tm.OP_QHAT, 0.02)
    assert _close(out.cpu().numpy(), ref.cpu().numpy())
    fresh.close()
    warm.close()


def test_noalloc_rejects_lattices_above_its_limit():
    tm = require_gpu()
    dims = (16, 16, 16, 18)   # V/2 = 36864 > 32768
    U = synth.unit_gauge_field(dims)
    g = tm.Gauge(U, dims, KAPPA, MU, EPS)
    assert g.vh > tm.NOALLOC_MAX_VH
    x = g.spinor()
    y = g.spinor()
    with pytest.raises(tm.TmndError) as e:
        tm.tm_nd_apply_noalloc(g.handle, y, x, tm.OP_MHAT, 0.0)
    assert e.value.status == 1 and "limit" in str(e.value)
    g.close()
