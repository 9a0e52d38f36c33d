"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
and exports every entry point include/tmnd.h declares; argument validation
rejects bad input before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tmnd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w]+\s*\**\s*(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def tm():
    from paper_1805_09584_gb300 import _build
    _build.build()
    import paper_1805_09584_gb300 as tm
    return tm


def test_exports_match_header(tm):
    declared = _declared()
    assert set(declared) == set(tm.EXPORTS), declared
    L = tm.lib()
    for name in declared:
        assert hasattr(L, name), name
        # every entry point has its argument types declared: without them ctypes
        # would pass 64-bit device pointers as 32-bit ints
        assert getattr(L, name).argtypes is not None, name


def test_rejects_bad_arguments_without_gpu(tm):
    import numpy as np
    # odd dimension -> TMND_ERR_ARG before any CUDA call
    a = tm.make_action((4, 4, 4, 3), 0.16, 0.1, 0.11)
    with pytest.raises(tm.TmndError) as e:
        tm.tmnd_gauge_create(np.zeros((4, 4, 4, 4, 3, 3, 3), np.complex128), a)
    assert e.value.status == 1 and "even" in str(e.value)
    # non-SU(3) link -> TMND_ERR_NOTSU3 (host-side validation)
    dims = (2, 2, 2, 2)
    import synth
    U = synth.unit_gauge_field(dims)
    U[2, 1, 0, 1, 1] *= 1.5
    with pytest.raises(tm.TmndError) as e:
        tm.tmnd_gauge_create(U, tm.make_action(dims, 0.16, 0.1, 0.11))
    assert e.value.status == 7
    # NULL handle -> TMND_ERR_ARG
    with pytest.raises(tm.TmndError) as e:
        tm.tm_nd_apply(None, 16, 32, 0, 0.0, 1, stream=0)
    assert e.value.status == 1


def test_oracle_and_library_share_no_code():
    """The oracle is independent of the CUDA path: neither imports the other."""
    import ast
    for path, forbidden in ((os.path.join(ROOT, "oracle"), "paper_1805_09584_gb300"),
                            (os.path.join(ROOT, "paper_1805_09584_gb300"), "oracle")):
        for dp, _, fs in os.walk(path):
            for f in fs:
                if f.endswith(".py"):
                    tree = ast.parse(open(os.path.join(dp, f)).read())
                    for node in ast.walk(tree):
                        if isinstance(node, ast.Import):
                            assert all(not a.name.startswith(forbidden) for a in node.names), (f, forbidden)
                        if isinstance(node, ast.ImportFrom) and node.module:
                            assert not node.module.startswith(forbidden), (f, forbidden)
                if f.endswith((".cu", ".cuh", ".c", ".h")):
                    txt = open(os.path.join(dp, f)).read()
                    assert "tmnd_oracle" not in txt or path.endswith("oracle")


def test_s16_shape_table_host(tm):
    """The compiled launch shapes of the 16-bit stencil (host queries, no GPU needed)."""
    seen = set()
    for sh in range(tm.S16_SHAPES):
        t, b, pf, ro = tm.tmnd_s16_shape_info(sh)
        assert t % 32 == 0 and 1 <= b <= 8 and t * b <= 1024
        seen.add((t, b, pf, ro))
    assert len(seen) == tm.S16_SHAPES
    with pytest.raises(tm.TmndError):
        tm.tmnd_s16_shape_info(tm.S16_SHAPES)
    with pytest.raises(tm.TmndError):
        tm.tmnd_s16_force_shape(tm.S16_SHAPES)
    tm.tmnd_s16_force_shape(-1)
