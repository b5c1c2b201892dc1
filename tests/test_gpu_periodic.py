"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle
on the same seeded inputs.

Tolerances (relative L2 on the grid, eq. l2err):
  * FP64:  1e-12 (rounding-order differences only: both sides run the same
    scheme; the GPU uses FFTs and one-step phase products, the oracle direct
    O(M^2) sums and directly evaluated multi-step phases);
  * MIXED: the O(h |V|) correction passes through FP32, so the error grows
    like (number of steps) * h |V| * eps_32; the bound per test is stated
    with it.
"""
import math

import numpy as np
import pytest

import synth
from oracle import fields
from oracle.periodic import PeriodicOracle, oracle_for, rel_l2

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def gpu_solve(inst, precision="fp64", order=8, startup=-1, nsteps=None, batch_of=None, keep=()):
    from paper_2001_06113_gb300 import Problem
    nsteps = inst.nsteps if nsteps is None else nsteps
    insts = batch_of or [inst]
    prob = Problem(inst.shape, inst.dt, inst.nsteps, order=order, precision=precision,
                   startup_steps=startup, batch=len(insts))
    for b, it in enumerate(insts):
        prob.set_potential(it.V0, it.vfac_table(), instance=b)
        if it.pulse is not None:
            p = it.pulse
            prob.set_pulse(p.A0, p.omega, p.T_pulse, p.direction, instance=b)
        prob.set_initial(it.u0, instance=b)
    snaps = {}
    done = 0
    for n in sorted(set(keep) | {nsteps}):
        prob.step(n - done)
        done = n
        snaps[n] = prob.read_u(-1 if batch_of else 0).copy()
    prob.close()
    return snaps[nsteps], snaps


def oracle_solve(inst, order=8, startup=None, nsteps=None):
    nsteps = inst.nsteps if nsteps is None else nsteps
    return oracle_for(inst, order=order, n_startup=startup).solve(inst.u0, nsteps)


# ------------------------------------------------------------------ 1D, FP64
def test_1d_cosine_workload_fp64():
    """1D periodic N=128, V = (1 + 0.5 sin 2t) sum a_m cos(mx), T = 1, dt = 1e-2."""
    inst = synth.periodic_1d_cosine()
    err = rel_l2(gpu_solve(inst)[0], oracle_solve(inst))
    assert err <= FP64_TOL, err


@pytest.mark.parametrize("M", [8, 16, 32, 256, 1024, 4096])
def test_1d_sizes_fp64(M):
    """Ragged cases: N=8..32 has fewer modes than threads; 4096 spans many passes."""
    inst = synth.random_periodic((M,), 100 + M, 2e-3, 12, vamp=8.0,
                                 pulse=synth.Pulse(2.5, 10.0, 0.024, (1.0,)),
                                 vfac=lambda t: 1.0 + 0.3 * np.cos(5.0 * np.asarray(t)))
    err = rel_l2(gpu_solve(inst)[0], oracle_solve(inst))
    assert err <= FP64_TOL, err


@pytest.mark.parametrize("order,startup", [(2, -1), (4, -1), (6, -1), (8, 6), (8, 10)])
def test_1d_orders_and_startup(order, startup):
    inst = synth.random_periodic((64,), 7, 5e-3, 16, vamp=6.0, pulse=synth.Pulse(1.0, 10.0, 0.08, (1.0,)))
    ref = oracle_solve(inst, order=order, startup=None if startup == -1 else startup)
    err = rel_l2(gpu_solve(inst, order=order, startup=startup)[0], ref)
    assert err <= FP64_TOL, err


def test_1d_intermediate_times_fp64():
    """Read-out in the middle of the start-up and of the Adams phase."""
    inst = synth.random_periodic((128,), 3, 4e-3, 20, vamp=5.0, pulse=synth.Pulse(2.0, 10.0, 0.08, (1.0,)))
    _, snaps = gpu_solve(inst, keep=(3, 7, 8, 13))
    orc = oracle_for(inst)
    _, kept = orc.solve(inst.u0, 20, keep={3, 7, 8, 13, 20})
    for n in (3, 7, 8, 13, 20):
        assert rel_l2(snaps[n], kept[n]) <= FP64_TOL, n


def test_1d_free_particle_max_size():
    """N = 8192 (the largest 1D size): with V = 0 the scheme is exact, so the
    result must equal the closed form e^{-i k^2 t + i k phi(t)} u^_k(0)."""
    M = 8192
    pulse = synth.Pulse(3.0, 10.0, 0.05, (1.0,))
    rng = np.random.default_rng(5)
    x = synth.periodic_grid(M)
    ks = np.arange(-40, 41)
    c = (rng.normal(size=ks.size) + 1j * rng.normal(size=ks.size)) * np.exp(-0.002 * ks ** 2)
    u0 = (np.exp(1j * np.outer(x, ks)) @ c)
    inst = synth.Instance(synth.PERIODIC, (M,), u0, np.zeros(M), lambda t: np.ones_like(np.asarray(t)),
                          pulse, 1e-3, 50)
    u = gpu_solve(inst)[0]
    T = 0.05
    ph = fields.phi_callable(pulse, 1)(T)[0]
    ref = np.exp(1j * np.outer(x, ks)) @ (c * np.exp(-1j * ks ** 2 * T + 1j * ks * ph))
    assert rel_l2(u, ref) <= 1e-12


# ------------------------------------------------------------------ 2D, FP64
@pytest.mark.parametrize("shape", [(8, 8), (16, 32), (32, 8), (64, 64), (128, 16)])
def test_2d_shapes_fp64(shape):
    inst = synth.random_periodic(shape, 11, 2e-3, 12, vamp=6.0, pulse=synth.Pulse(2.0, 10.0, 0.024, (0.8, -0.6)),
                                 vfac=lambda t: 1.0 + 0.5 * np.sin(3.0 * np.asarray(t)))
    err = rel_l2(gpu_solve(inst)[0], oracle_solve(inst))
    assert err <= FP64_TOL, err


def test_2d_wells_full_grid_fp64():
    """The 512^2 wells workload at full grid size (first 10 steps: 7 Richardson
    start-up steps and 3 Adams steps), in the launch configuration the bench uses."""
    inst = synth.periodic_2d_wells()
    err = rel_l2(gpu_solve(inst, nsteps=10)[0], oracle_solve(inst, nsteps=10))
    assert err <= FP64_TOL, err


def test_2d_free_particle_full_length():
    """512^2 over the workload's full 2000 steps with V = 0: exact closed form."""
    inst = synth.periodic_2d_wells()
    M = 512
    x = synth.periodic_grid(M)
    rng = np.random.default_rng(1)
    modes = [((int(a), int(b)), complex(rng.normal(), rng.normal())) for a, b in rng.integers(-20, 20, size=(12, 2))]
    X, Y = np.meshgrid(x, x, indexing="ij")

    def field(t):
        ph = fields.phi_callable(inst.pulse, 2)(t)
        u = np.zeros((M, M), dtype=np.complex128)
        for (a, b), c in modes:
            u += c * np.exp(1j * (a * X + b * Y - (a * a + b * b) * t + a * ph[0] + b * ph[1]))
        return u
    free = synth.Instance(synth.PERIODIC, (M, M), field(0.0), np.zeros((M, M)), inst.vfac, inst.pulse,
                          inst.dt, inst.nsteps)
    u = gpu_solve(free)[0]
    assert rel_l2(u, field(inst.t_max)) <= 1e-12


@pytest.mark.parametrize("shape,precision,tol", [((1024, 1024), "fp64", 1e-12), ((1024, 1024), "mixed", 2e-6),
                                                   ((8, 1024), "fp64", 1e-12), ((1024, 8), "mixed", 2e-6)])
def test_2d_free_particle_extreme_shapes(shape, precision, tol):
    """The largest and the most elongated 2D grids (8..1024 per dimension),
    V = 0 with a pulse along (0.6, -0.8): the closed form
    sum_k c_k e^{i k.x - i |k|^2 t + i k.phi(t)}."""
    n0, n1 = shape
    pulse = synth.Pulse(2.0, 10.0, 0.03, (0.6, -0.8))
    rng = np.random.default_rng(4)
    K0, K1 = min(n0 // 2 - 1, 30), min(n1 // 2 - 1, 30)
    modes = [((int(a), int(b)), complex(rng.normal(), rng.normal()))
             for a, b in zip(rng.integers(-K0, K0 + 1, size=10), rng.integers(-K1, K1 + 1, size=10))]
    X, Y = np.meshgrid(synth.periodic_grid(n0), synth.periodic_grid(n1), indexing="ij")

    def field(t):
        ph = fields.phi_callable(pulse, 2)(t)
        u = np.zeros(shape, dtype=np.complex128)
        for (a, b), c in modes:
            u += c * np.exp(1j * (a * X + b * Y - (a * a + b * b) * t + a * ph[0] + b * ph[1]))
        return u
    free = synth.Instance(synth.PERIODIC, shape, field(0.0), np.zeros(shape), lambda t: np.ones_like(np.asarray(t)),
                          pulse, 1e-3, 30)
    u = gpu_solve(free, precision=precision)[0]
    assert rel_l2(u, field(free.t_max)) <= tol


# ------------------------------------------------------------------ batching
def test_batch_members_equal_single_runs():
    """Each batch member is bit-identical to the same instance solved alone."""
    insts = [synth.random_periodic((32, 16), s, 2e-3, 10, vamp=4.0 + s,
                                   pulse=synth.Pulse(1.0 + s, 10.0, 0.02, (1.0, 0.3))) for s in range(3)]
    batched = gpu_solve(insts[0], batch_of=insts)[0]
    for b, it in enumerate(insts):
        alone = gpu_solve(it)[0]
        assert np.array_equal(batched[b], alone), b


# ------------------------------------------------------------------ mixed precision
@pytest.mark.parametrize("shape,steps,tol", [((128,), 100, 2e-6), ((64, 64), 40, 2e-6)])
def test_mixed_precision_error_bound(shape, steps, tol):
    inst = synth.random_periodic(shape, 5, 5e-3, steps, vamp=8.0, pulse=synth.Pulse(2.0, 10.0, steps * 5e-3, (1.0, 0.0)[:len(shape)]))
    ref = oracle_solve(inst)
    err = rel_l2(gpu_solve(inst, precision="mixed")[0], ref)
    print("mixed", shape, err)
    assert err <= tol, err


def test_mixed_2d_wells_full_grid():
    inst = synth.periodic_2d_wells()
    err = rel_l2(gpu_solve(inst, precision="mixed", nsteps=10)[0], oracle_solve(inst, nsteps=10))
    print("mixed 512^2 10 steps", err)
    assert err <= 1e-6, err


# ------------------------------------------------------------------ edge cases and errors
def test_read_before_step_returns_u0():
    inst = synth.random_periodic((16, 16), 2, 1e-3, 5)
    from paper_2001_06113_gb300 import Problem
    p = Problem(inst.shape, inst.dt, inst.nsteps)
    p.set_potential(inst.V0)
    p.set_initial(inst.u0)
    assert np.array_equal(p.read_u(0), inst.u0)
    p.step(0)
    assert p.step_index == 0
    p.close()


def test_status_codes():
    from paper_2001_06113_gb300 import Problem, TdseError
    inst = synth.random_periodic((32,), 2, 1e-3, 3)
    p = Problem(inst.shape, inst.dt, inst.nsteps)
    with pytest.raises(TdseError) as e:
        p.step(1)                       # no V / u0 yet
    assert e.value.status == -6
    p.set_potential(inst.V0)
    p.set_initial(inst.u0)
    p.step(3)
    with pytest.raises(TdseError) as e:
        p.step(1)                       # beyond the tables
    assert e.value.status == -1
    with pytest.raises(TdseError) as e:
        p.set_initial(inst.u0, instance=4)
    assert e.value.status == -1
    p.close()


def test_nonfinite_detected():
    from paper_2001_06113_gb300 import Problem, TdseError
    inst = synth.random_periodic((32,), 2, 1e-3, 3)
    V = inst.V0.copy()
    V[5] = np.nan
    p = Problem(inst.shape, inst.dt, inst.nsteps)
    p.set_potential(V)
    p.set_initial(inst.u0)
    p.step(1)
    with pytest.raises(TdseError) as e:
        p.check_finite()
    assert e.value.status == -5
    p.close()


def test_device_pointers_and_callback_field():
    """Inputs given as CUDA tensors; A(t) given as a Python callback."""
    import torch
    from paper_2001_06113_gb300 import Problem
    inst = synth.random_periodic((64,), 9, 2e-3, 10, pulse=synth.Pulse(2.0, 10.0, 0.02, (1.0,)))
    p = Problem(inst.shape, inst.dt, inst.nsteps)
    p.set_potential(torch.tensor(inst.V0, device="cuda"))
    p.set_vector_potential(lambda t: inst.pulse.A(t))
    p.set_initial(torch.tensor(inst.u0, device="cuda"))
    p.step(10)
    out = torch.empty(64, dtype=torch.complex128, device="cuda")
    p.read_u(0, out=out)
    err = rel_l2(out.cpu().numpy(), oracle_solve(inst))
    p.close()
    assert err <= FP64_TOL, err


@pytest.mark.parametrize("shape", [(128,), (32, 32)])
def test_builtin_pulse_equals_callback(shape):
    """The built-in pulse (phi in closed form on the device) and the same A(t)
    as a callback (8-point Gauss-Legendre per dt/8 on the host) agree to
    rounding: both are phi to ~1e-16."""
    from paper_2001_06113_gb300 import Problem
    d = len(shape)
    pulse = synth.Pulse(30.0, 150.0, 0.05, (1.0, -0.7)[:d])
    inst = synth.random_periodic(shape, 12, 1e-3, 40, pulse=pulse)
    out = []
    for builtin in (True, False):
        p = Problem(inst.shape, inst.dt, inst.nsteps)
        p.set_potential(inst.V0)
        if builtin:
            p.set_pulse(pulse.A0, pulse.omega, pulse.T_pulse, pulse.direction)
        else:
            p.set_vector_potential(lambda t: pulse.A(t))
        p.set_initial(inst.u0)
        p.step(40)
        out.append(p.read_u(0))
        p.close()
    assert rel_l2(out[0], out[1]) < 1e-13


def test_mixed_2d_single_steps_equal_fused_sequence():
    """Mixed 2D: k calls of step(1) (separate end and begin column passes)
    and one step(k) (fused column passes with staged history reads) give the
    same bits."""
    from paper_2001_06113_gb300 import Problem
    inst = synth.periodic_2d_wells(seed=9, M=64, dt=1e-3, nsteps=30)
    out = []
    for chunks in ([1] * 20, [20]):
        pr = Problem((64, 64), inst.dt, inst.nsteps, precision="mixed")
        pr.set_potential(inst.V0)
        p = inst.pulse
        pr.set_pulse(p.A0, p.omega, p.T_pulse, p.direction)
        pr.set_initial(inst.u0)
        for k in chunks:
            pr.step(k)
        out.append(pr.read_u(0))
        pr.close()
    assert np.array_equal(out[0], out[1])
