"""The allocation-free read-out transform against the library's own read-out.

Some callers cannot allocate device memory at all -- no cudaMalloc and hence
no workspace for a solver context (a host application that owns every
allocation, a plugin with a fixed device budget).  For them the library offers
tdse_modes_to_grid_2d_noalloc, whose scratch is a fixed array inside the
library.  Its grid values must equal what tdse_read_u returns for the same
modes, within the FP64 tolerance of the other parity tests, on consecutive
calls (the shared scratch keeps the previous call's contents).

This file is named to be collected last.
"""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2001_06113_gb300 import _native
    return torch, _native


def _free_problem(shape, batch, nsteps, dt, seed):
    """V = 0 with a pulse: the solver's modes are exactly
    DFT(u0) e^{-i |k|^2 t + i k.phi(t)} (eq. uhatkinteq), computed here on the host."""
    from oracle import fields
    from paper_2001_06113_gb300 import Problem
    import synth
    n0, n1 = shape
    pulse = synth.Pulse(2.0, 10.0, nsteps * dt, (0.7, -0.4))
    rng = np.random.default_rng(seed)
    u0s = []
    for _ in range(batch):
        u0s.append(synth.random_periodic(shape, int(rng.integers(1 << 30)), dt, nsteps).u0)
    prob = Problem(shape, dt, nsteps, batch=batch)
    prob.set_potential(np.zeros(shape))
    prob.set_pulse(pulse.A0, pulse.omega, pulse.T_pulse, pulse.direction)
    for b, u0 in enumerate(u0s):
        prob.set_initial(u0, instance=b)
    prob.step(nsteps)
    t = nsteps * dt
    phi = fields.phi_pulse(t, pulse.A0, pulse.omega, pulse.T_pulse, pulse.direction).reshape(2)
    k0 = np.fft.fftfreq(n0, 1.0 / n0)[:, None]
    k1 = np.fft.fftfreq(n1, 1.0 / n1)[None, :]
    ph = np.exp(-1j * (k0 ** 2 + k1 ** 2) * t + 1j * (k0 * phi[0] + k1 * phi[1]))
    modes = np.stack([np.fft.fft2(u0) / (n0 * n1) * ph for u0 in u0s])
    return prob, modes


def _noalloc(torch, native, modes, stream):
    nb, n0, n1 = modes.shape
    src = torch.tensor(modes, dtype=torch.complex128, device="cuda")
    out = torch.full((nb, n0, n1), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    st = native.lib().tdse_modes_to_grid_2d_noalloc(ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                                   n0, n1, nb, ctypes.c_void_p(stream.cuda_stream))
    stream.synchronize()
    return st, out.cpu().numpy()


def _rel(a, b):
    return math.sqrt(float(np.sum(np.abs(a - b) ** 2) / np.sum(np.abs(b) ** 2)))


def test_noalloc_matches_read_u_on_two_calls(env):
    torch, native = env
    stream = torch.cuda.current_stream()
    cases = [((64, 32), 2, 12, 2e-3, 1), ((16, 128), 1, 9, 3e-3, 2)]
    for shape, batch, nsteps, dt, seed in cases:           # two calls in a row, different sizes
        prob, modes = _free_problem(shape, batch, nsteps, dt, seed)
        ref = prob.read_u(-1)                              # existing entry point
        st, got = _noalloc(torch, native, modes, stream)
        assert st == 0
        for b in range(batch):
            assert _rel(got[b], ref[b]) <= TOL, (shape, b)
            # and an independent inverse DFT (numpy's, without its 1/(n0 n1))
            assert _rel(got[b], np.fft.ifft2(modes[b]) * (shape[0] * shape[1])) <= TOL, (shape, b)
        prob.close()


def test_noalloc_at_the_size_limit(env):
    """Calls that fill the fixed scratch exactly: 512 x 1024 (one array, the
    intermediate reaching the end of its region) and 64 arrays of 1024 x 8 (a
    full 1024-entry twiddle axis), each against tdse_read_u and numpy."""
    torch, native = env
    stream = torch.cuda.current_stream()
    cases = [((512, 1024), 1, 3, 1e-3, 5), ((1024, 8), 64, 3, 1e-3, 6)]
    for shape, batch, nsteps, dt, seed in cases:
        assert batch * shape[0] * shape[1] == native.NOALLOC_MAX_POINTS
        prob, modes = _free_problem(shape, batch, nsteps, dt, seed)
        ref = prob.read_u(-1)
        st, got = _noalloc(torch, native, modes, stream)
        assert st == 0
        for b in range(batch):
            assert _rel(got[b], ref[b]) <= TOL, (shape, b)
            assert _rel(got[b], np.fft.ifft2(modes[b]) * (shape[0] * shape[1])) <= TOL, (shape, b)
        prob.close()


def test_noalloc_rejects_oversize(env):
    torch, native = env
    stream = torch.cuda.current_stream()
    n = 1024
    modes = np.zeros((1, n, n), dtype=np.complex128)      # 2^20 points > TDSE_NOALLOC_MAX_POINTS
    st, got = _noalloc(torch, native, modes, stream)
    assert st == -2
    assert np.all(np.isnan(got))                          # output untouched
    assert n * n > native.NOALLOC_MAX_POINTS
