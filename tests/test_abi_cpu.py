"""C-ABI checks that need no GPU: the library loads, exports every symbol
include/tdse.h declares, and its host-only entry points validate input."""
import ctypes
import math
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
    return sorted(set(re.findall(r"\b(tdse_[A-Za-z_0-9]+)\s*\(", text)) - {"tdse_field_fn"})


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
        elif k == "nu":
            c.nu[0], c.nu[1] = v
        else:
            setattr(c, k, v)
    return c


@pytest.mark.parametrize("kw,status", [
    (dict(), 0),
    (dict(dim=2, n=(32, 16)), 0),
    (dict(dim=3), -1),                 # 3D needs n_z
    (dict(dim=3, n=(16, 8), n_z=32), 0),
    (dict(dim=3, n=(16, 8), n_z=32, precision=1), 0),
    (dict(dim=3, n=(16, 12), n_z=32), -1),            # not a power of two
    (dict(dim=3, n=(16, 512), n_z=32), -7),           # axis 1 at most 256
    (dict(dim=3, n=(1024, 256), n_z=1024), -7),       # more than 2^24 points
    (dict(dim=3, n=(32, 64), n_z=32, bc=1, nu=(128, 256), nu_z=128, H=1.5, gauss_q=10, n_r=1), 0),  # free space 3D
    (dict(dim=3, n=(32, 64), n_z=32, bc=1, nu=(128, 256), nu_z=128, H=1.5, gauss_q=10, n_r=1, precision=1), 0),
    (dict(dim=3, n=(32, 64), n_z=32, bc=1, nu=(128, 256), H=1.5, gauss_q=10, n_r=1), -1),   # no nu_z
    (dict(dim=3, n=(32, 64), n_z=16, bc=1, nu=(128, 256), nu_z=64, H=1.5, gauss_q=10, n_r=1), -7),  # n_z < 32
    (dict(dim=4), -1),
    (dict(n=(48, 1)), -1),             # not a power of two
    (dict(n=(16384, 1)), 0),           # 1D FP64 beyond one CTA: the four-step transform through the 2D passes
    (dict(n=(16384, 1), precision=1), 0),   # mixed: FP32 steps, FP64 four-step start and read-out
    (dict(n=(32768, 1), precision=1), 0),
    (dict(n=(65536, 1), precision=1), 0),
    (dict(n=(1 << 21, 1), precision=1), -7),
    (dict(n=(16384, 1), precision=1, layout_1d=2), 0),   # the four-step passes by choice
    (dict(n=(512, 1), layout_1d=2), 0),
    (dict(n=(32768, 1), precision=1, layout_1d=1), -7),  # one CTA per instance not built there
    (dict(n=(32, 1), layout_1d=2), -7),                  # the passes need n >= 64
    (dict(n=(512, 1), layout_1d=3), -1),
    (dict(order=7), -1),
    (dict(order=10), -1),
    (dict(dt=0.0), -1),
    (dict(batch=0), -1),
    (dict(startup_steps=5), -1),       # fewer than order - 2
    (dict(bc=1), -1),                  # free space without nu / H
    (dict(bc=1, nu=(512, 0), H=1.5, gauss_q=10, n_r=1), 0),
    (dict(bc=1, dim=2, n=(64, 32), nu=(512, 256), H=1.5, gauss_q=10, n_r=1), 0),
    (dict(bc=1, nu=(512, 0), H=1.5, gauss_q=10, n_r=1, precision=1), 0),    # free space, FP32 transforms
    (dict(bc=1, dim=2, n=(64, 64), nu=(512, 512), H=1.0, gauss_q=10, n_r=1, precision=1), 0),
    (dict(bc=1, n=(1024, 1), nu=(4096, 0), H=1.5, gauss_q=10, n_r=1), -7),  # n > 512
    (dict(bc=1, nu=(500, 0), H=1.5, gauss_q=10, n_r=1), -1),                # nu not a multiple of n
    (dict(bc=1, nu=(512, 0), H=0.0, gauss_q=10, n_r=1), -1),
    (dict(bc=1, nu=(512, 0), H=1.5, gauss_q=10, n_r=1, alpert_p=5), -1),
    (dict(bc=1, nu=(512, 0), H=1.5, gauss_q=10, n_r=5), -1),
    (dict(bc=1, nu=(512, 0), H=1.5, gauss_q=0, n_r=1), -1),
    (dict(bc=1, nu=(512, 0), H=1.5, gauss_q=32, n_r=4), -1),                # dense block > 128 modes
    (dict(precision=5), -1),
    (dict(potential=1), 0),                                                  # general V(x, t) table
    (dict(potential=2), 0),                                                  # one table for all instances
    (dict(potential=3), -1),
    (dict(bc=1, nu=(512, 0), H=1.5, gauss_q=10, n_r=1, potential=1), 0),
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


def test_shape_1d_validation(native):
    """The alternative 1D launch shape exists for mixed 1D contexts of n >= 512
    (one CTA per instance) and nowhere else; no CUDA call is made."""
    lib = native.lib()
    # (config, status of shape 1, status of shape 0)
    cases = [(dict(n=(512, 1), precision=1), 0, 0), (dict(n=(16384, 1), precision=1), 0, 0),
             (dict(n=(256, 1), precision=1), -7, 0), (dict(n=(512, 1)), -7, -7),
             (dict(n=(32768, 1), precision=1), -7, -7), (dict(dim=2, n=(64, 64), precision=1), -7, -7)]
    for kw, want, want0 in cases:
        ctx = ctypes.c_void_p()
        assert lib.tdse_create(ctypes.byref(_cfg(native, **kw)), ctypes.byref(ctx)) == 0
        assert lib.tdse_shape_1d(ctx) == 0
        assert lib.tdse_set_shape_1d(ctx, 1) == want, kw
        assert lib.tdse_shape_1d(ctx) == (1 if want == 0 else 0)
        assert lib.tdse_set_shape_1d(ctx, 2) == -1
        assert lib.tdse_set_shape_1d(ctx, 0) == want0
        lib.tdse_destroy(ctx)
    assert lib.tdse_shape_1d(None) == -1


def test_workspace_size_scales_with_batch(native):
    lib = native.lib()
    sizes = []
    for b in (1, 4):
        ctx = ctypes.c_void_p()
        assert lib.tdse_create(ctypes.byref(_cfg(native, batch=b, dim=2, n=(64, 64))), ctypes.byref(ctx)) == 0
        sizes.append(lib.tdse_workspace_bytes(ctx))
        lib.tdse_destroy(ctx)
    assert 3.5 * sizes[0] < sizes[1] < 4.5 * sizes[0]


# ------------------------------------------------------------ free-space rule
def _free_ctx(native, M=64, nu=512, H=1.7, p=8, q=10, n_r=2):
    lib = native.lib()
    ctx = ctypes.c_void_p()
    cfg = _cfg(native, bc=1, n=(M, 1), nu=(nu, 0), H=H, gauss_q=q, n_r=n_r, alpert_p=p)
    assert lib.tdse_create(ctypes.byref(cfg), ctypes.byref(ctx)) == 0
    return lib, ctx


@pytest.mark.parametrize("p,q,n_r", [(8, 10, 1), (8, 16, 2), (4, 6, 0), (8, 8, 3)])
def test_free_rule_matches_oracle_rule(native, p, q, n_r):
    """The library's contour rule (its own Gauss-Legendre and Alpert tables,
    derived by a different algorithm) equals the oracle's GammaRule node by node."""
    from oracle import gamma
    M, nu, H = 64, 512, 1.7
    lib, ctx = _free_ctx(native, M, nu, H, p, q, n_r)
    n = ctypes.c_int()
    assert lib.tdse_free_rule(ctx, 0, ctypes.byref(n), None, None) == 0
    z = np.empty(n.value, dtype=np.complex128)
    w = np.empty(n.value, dtype=np.complex128)
    dp = ctypes.POINTER(ctypes.c_double)
    assert lib.tdse_free_rule(ctx, 0, ctypes.byref(n), z.ctypes.data_as(dp), w.ctypes.data_as(dp)) == 0
    assert lib.tdse_free_rule(ctx, 1, ctypes.byref(n), None, None) == -1      # 1D: no axis 1
    lib.tdse_destroy(ctx)
    r = gamma.GammaRule.for_nu(M, nu, H, p=p, q=q, n_r=n_r)
    assert z.size == r.N
    assert np.max(np.abs(z - r.zeta) / np.maximum(1.0, np.abs(r.zeta))) < 4e-16
    assert np.max(np.abs(w - r.w)) < 2e-15      # Gauss-Legendre weights by two routes: a few ulps


def test_free_rule_3d_per_axis(native):
    """3D free space: each axis has its own contour rule (M, nu of that axis)
    and the mode state is their tensor product."""
    from oracle import gamma
    lib = native.lib()
    ctx = ctypes.c_void_p()
    M, nus, H = (32, 64, 32), (128, 256, 256), 1.5
    cfg = _cfg(native, dim=3, bc=1, n=M[:2], n_z=M[2], nu=nus[:2], nu_z=nus[2], H=H, gauss_q=10, n_r=1)
    assert lib.tdse_create(ctypes.byref(cfg), ctypes.byref(ctx)) == 0
    dp = ctypes.POINTER(ctypes.c_double)
    Ns = []
    for ax in range(3):
        n = ctypes.c_int()
        assert lib.tdse_free_rule(ctx, ax, ctypes.byref(n), None, None) == 0
        z = np.empty(n.value, dtype=np.complex128)
        w = np.empty(n.value, dtype=np.complex128)
        assert lib.tdse_free_rule(ctx, ax, ctypes.byref(n), z.ctypes.data_as(dp), w.ctypes.data_as(dp)) == 0
        r = gamma.GammaRule.for_nu(M[ax], nus[ax], H, q=10, n_r=1)
        assert z.size == r.N
        assert np.max(np.abs(z - r.zeta) / np.maximum(1.0, np.abs(r.zeta))) < 4e-16
        Ns.append(r.N)
    assert lib.tdse_free_rule(ctx, 3, ctypes.byref(ctypes.c_int()), None, None) == -1
    # the workspace holds at least u^ and the ring (7 slots) over N0 N1 N2 modes
    assert lib.tdse_workspace_bytes(ctx) >= 16 * 8 * Ns[0] * Ns[1] * Ns[2]
    lib.tdse_destroy(ctx)


@pytest.mark.parametrize("eps,vnorm,phimax,dim", [(1e-10, 20.0, 0.3, 2), (1e-12, 0.0, 0.0, 1), (1e-8, 5.0, 1.0, 2),
                                                (1e-4, 5.0, 0.5, 2), (1e-3, 0.0, 0.0, 1)])
def test_free_choose_H_matches_oracle(native, eps, vnorm, phimax, dim):
    from oracle import gamma
    from paper_2001_06113_gb300 import free_choose_H
    assert abs(free_choose_H(eps, vnorm, phimax, dim) - gamma.choose_H(eps, vnorm, phimax, dim)) < 1e-15
    if eps > 1e-6:
        # FP32 contour sums: eps_m = 2^-23, i.e. H smaller by log(2^29) / (2 d (1 + phimax))
        Hm = free_choose_H(eps, vnorm, phimax, dim, precision="mixed")
        assert abs(Hm - gamma.choose_H(eps, vnorm, phimax, dim, eps_m=2.0 ** -23)) < 1e-15
        assert abs(free_choose_H(eps, vnorm, phimax, dim) - Hm - 29 * math.log(2.0) / (2 * dim * (1 + phimax))) < 1e-13


def test_free_choose_H_rejects_nonpositive(native):
    from paper_2001_06113_gb300 import TdseError, free_choose_H
    with pytest.raises(TdseError):
        free_choose_H(1e-20, 100.0, 0.0, 1)         # eps below (1 + ||V||) eps_m: H < 0


def test_alpert_header_is_generator_output():
    """alpert_rules.h is exactly what its committed generator writes."""
    pytest.importorskip("mpmath")
    import subprocess
    import sys
    gen = os.path.join(ROOT, "paper_2001_06113_gb300", "csrc", "gen_alpert.py")
    out = subprocess.run([sys.executable, gen], capture_output=True, text=True, check=True).stdout
    assert out == open(os.path.join(ROOT, "paper_2001_06113_gb300", "csrc", "alpert_rules.h")).read()


def test_batch_create_validates_without_gpu(native):
    lib = native.lib()
    out = ctypes.c_void_p()
    assert lib.tdse_batch_create(None, 1, ctypes.byref(out)) == -1
    ctx = ctypes.c_void_p()
    assert lib.tdse_create(ctypes.byref(_cfg(native, precision=1)), ctypes.byref(ctx)) == 0
    arr = (ctypes.c_void_p * 1)(ctx.value)
    assert lib.tdse_batch_create(arr, 0, ctypes.byref(out)) == -1
    assert lib.tdse_batch_create(arr, 1, ctypes.byref(out)) == -1      # workspace not bound
    assert lib.tdse_batch_step(None, 1, None) == -1
    assert lib.tdse_batch_set_mode(None, 0) == -1
    lib.tdse_destroy(ctx)


def test_entry_points_refuse_before_binding(native):
    """Calls that need device memory fail with TDSE_ESTATE before the
    workspace is bound, and bad arguments with TDSE_EINVAL; no CUDA call."""
    lib = native.lib()
    ctx = ctypes.c_void_p()
    assert lib.tdse_create(ctypes.byref(_cfg(native, potential=1)), ctypes.byref(ctx)) == 0
    u = np.zeros(2 * 64)
    V = np.zeros(lib.tdse_potential_times(ctx, None) * 64)
    dp = ctypes.POINTER(ctypes.c_double)
    assert lib.tdse_set_initial_batch(ctx, u.ctypes.data_as(dp), 0, None) == -6
    assert lib.tdse_set_potential_table(ctx, -1, V.ctypes.data_as(dp), 0, None) == -6
    assert lib.tdse_set_initial_batch(None, u.ctypes.data_as(dp), 0, None) == -1
    assert lib.tdse_set_initial_batch(ctx, None, 0, None) == -1
    assert lib.tdse_set_potential_table(ctx, -1, None, 0, None) == -1
    d = (ctypes.c_double * 2)(1.0, 0.0)
    assert lib.tdse_set_pulse(ctx, -1, 1.0, 10.0, 0.0, d, None) == -1       # T_pulse must be > 0
    assert lib.tdse_set_pulse(ctx, -1, 1.0, 10.0, 1.0, d, None) == -6
    assert lib.tdse_set_residual_check(ctx, 5, 1e-6) == -7                 # FP64: nothing to check
    lib.tdse_destroy(ctx)


def test_checkpoint_size_query_without_gpu(native):
    lib = native.lib()
    ctx = ctypes.c_void_p()
    assert lib.tdse_create(ctypes.byref(_cfg(native)), ctypes.byref(ctx)) == 0
    n = ctypes.c_size_t()
    assert lib.tdse_save(ctx, None, ctypes.byref(n), None) == 0
    assert n.value > lib.tdse_workspace_bytes(ctx)
    buf = ctypes.create_string_buffer(n.value)
    assert lib.tdse_save(ctx, buf, ctypes.byref(n), None) == -6          # workspace not bound
    assert lib.tdse_load(ctx, buf, n.value, None) == -6
    lib.tdse_destroy(ctx)


@pytest.mark.parametrize("nsteps,startup,bc", [(20, -1, 0), (5, -1, 0), (30, 10, 1)])
def test_potential_times(native, nsteps, startup, bc):
    """Rows of a potential table: every dt/8 of the S start-up steps, then
    every Adams step (host-only query; -1 for a separable context)."""
    lib = native.lib()
    kw = dict(nsteps=nsteps, startup_steps=startup, potential=1, dt=0.01)
    if bc:
        kw.update(bc=1, nu=(512, 0), H=1.5, gauss_q=10, n_r=1)
    ctx = ctypes.c_void_p()
    assert lib.tdse_create(ctypes.byref(_cfg(native, **kw)), ctypes.byref(ctx)) == 0
    S = min(7 if startup < 0 else startup, nsteps)
    R = lib.tdse_potential_times(ctx, None)
    assert R == 8 * S + 1 + nsteps - S
    t = np.empty(R)
    assert lib.tdse_potential_times(ctx, t.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == R
    want = np.concatenate([np.arange(8 * S + 1) * 0.01 / 8, np.arange(S + 1, nsteps + 1) * 0.01])
    assert np.allclose(t, want, rtol=0, atol=1e-15)
    lib.tdse_destroy(ctx)
    sep = ctypes.c_void_p()
    assert lib.tdse_create(ctypes.byref(_cfg(native)), ctypes.byref(sep)) == 0
    assert lib.tdse_potential_times(sep, None) == -1
    lib.tdse_destroy(sep)
