"""C-ABI checks that need no GPU: the library loads, exports every symbol
include/tdse.h declares, and its host-only entry points validate input."""
import ctypes
import os
import re
from fractions import Fraction

import numpy as np
import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "tdse.h")


@pytest.fixture(scope="module")
def native():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2001_06113_gb300 import _native
    return _native


def _declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tdse_[a-z_0-9]+)\s*\(", text)) - {"tdse_field_fn"})


def test_header_declarations_listed(native):
    assert sorted(native.EXPORTS) == _declared_symbols()


def test_library_exports_every_declared_symbol(native):
    lib = ctypes.CDLL(native._LIB_PATH)
    for name in _declared_symbols():
        assert hasattr(lib, name), name


def test_adams_weights_match_table1(native, golden_dir):
    from paper_2001_06113_gb300 import adams_weights
    rows = [l.split() for l in open(os.path.join(golden_dir, "adams8_table1.txt")) if l.strip() and l[0] != "#"]
    table = [float(Fraction(int(n), int(d))) for _, n, d in rows]
    assert list(adams_weights(8)) == table
    assert list(adams_weights(2)) == [0.5, 0.5]


def _cfg(native, **kw):
    c = native.TdseConfig()
    c.dim, c.bc, c.batch, c.dt, c.nsteps, c.order, c.startup_steps, c.precision = 1, 0, 1, 0.01, 10, 8, -1, 0
    c.n[0], c.n[1] = 64, 1
    for k, v in kw.items():
        if k == "n":
            c.n[0], c.n[1] = v
        else:
            setattr(c, k, v)
    return c


@pytest.mark.parametrize("kw,status", [
    (dict(), 0),
    (dict(dim=2, n=(32, 16)), 0),
    (dict(dim=3), -1),
    (dict(n=(48, 1)), -1),             # not a power of two
    (dict(n=(16384, 1)), -7),          # 1D limit of this build (FP64 transform in shared memory)
    (dict(order=7), -1),
    (dict(order=10), -1),
    (dict(dt=0.0), -1),
    (dict(batch=0), -1),
    (dict(startup_steps=5), -1),       # fewer than order - 2
    (dict(bc=1), -7),                  # free space: not built
    (dict(precision=5), -1),
])
def test_create_validates(native, kw, status):
    lib = native.lib()
    ctx = ctypes.c_void_p()
    st = lib.tdse_create(ctypes.byref(_cfg(native, **kw)), ctypes.byref(ctx))
    assert st == status
    if st == 0:
        assert lib.tdse_workspace_bytes(ctx) > 0
        assert lib.tdse_step_index(ctx) == 0
        # calls that need the workspace fail cleanly before it is bound
        assert lib.tdse_step(ctx, 1, None) == -6
        lib.tdse_destroy(ctx)


def test_workspace_size_scales_with_batch(native):
    lib = native.lib()
    sizes = []
    for b in (1, 4):
        ctx = ctypes.c_void_p()
        assert lib.tdse_create(ctypes.byref(_cfg(native, batch=b, dim=2, n=(64, 64))), ctypes.byref(ctx)) == 0
        sizes.append(lib.tdse_workspace_bytes(ctx))
        lib.tdse_destroy(ctx)
    assert 3.5 * sizes[0] < sizes[1] < 4.5 * sizes[0]
