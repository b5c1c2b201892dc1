"""Uneven 1D batches (one persistent launch per step for contexts of
different n, CUDA-graph replay, autotuned launch shapes) and the n = 16384
mixed-precision 1D instances, through the C ABI on the GPU."""
import numpy as np
import pytest

import synth
from oracle import fields
from oracle.periodic import rel_l2

pytestmark = pytest.mark.gpu

DT, NSTEPS = 1e-3, 40


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def members_data(sizes_counts, seed=0):
    """{N: [Instance, ...]} of seeded uneven-batch members with fixed N."""
    out = {}
    i = 0
    for N, count in sizes_counts:
        out[N] = [synth.periodic_1d_batch_member(seed * 1000 + i + k, dt=DT, nsteps=NSTEPS, sizes=(N,))
                  for k in range(count)]
        i += count
    return out


def make_problem(insts, stream=None, precision="mixed"):
    from paper_2001_06113_gb300 import Problem
    it0 = insts[0]
    pr = Problem(it0.shape, DT, NSTEPS, batch=len(insts), precision=precision, stream=stream)
    load(pr, insts)
    return pr


def load(pr, insts):
    for b, it in enumerate(insts):
        pr.set_potential(it.V0, None, instance=b)
        p = it.pulse
        pr.set_pulse(p.A0, p.omega, p.T_pulse, p.direction, instance=b)
        pr.set_initial(it.u0, instance=b)


def reset(pr, insts):
    for b, it in enumerate(insts):
        pr.set_initial(it.u0, instance=b)


SIZES = [(256, 5), (1024, 3), (4096, 2), (16384, 1), (512, 17)]


def test_batch_members_equal_solo_runs():
    """Each instance of each member after start-up + Adams steps in the fused
    launch equals the same instance run alone, bit for bit."""
    import torch
    from paper_2001_06113_gb300 import Batch
    data = members_data(SIZES)
    stream = torch.cuda.Stream()
    probs = [make_problem(insts, stream) for insts in data.values()]
    batch = Batch(probs, stream=stream)
    batch.step(12)
    stream.synchronize()
    for pr, insts in zip(probs, data.values()):
        ub = pr.read_u()
        for b, it in enumerate(insts):
            solo = make_problem([it])
            solo.step(12)
            assert np.array_equal(solo.read_u(0), ub[b]), (it.shape, b)
            solo.close()


def test_batch_graph_replay_and_tuning_keep_results():
    """A second call from step 0 replays the captured graph; a tuned launch
    shape (other threads per instance, CTA count) gives the same bits."""
    import torch
    from paper_2001_06113_gb300 import Batch
    data = members_data([(256, 9), (2048, 3), (8192, 2)], seed=1)
    stream = torch.cuda.Stream()
    probs = [make_problem(insts, stream) for insts in data.values()]
    batch = Batch(probs, stream=stream)
    batch.step(15)
    stream.synchronize()
    first = [pr.read_u().copy() for pr in probs]
    for pr, insts in zip(probs, data.values()):
        reset(pr, insts)
    batch.step(15)
    stream.synchronize()
    assert batch.describe()["graphs"] == 1
    for pr, u in zip(probs, first):
        assert np.array_equal(pr.read_u(), u)
    batch.tune(3)
    shape = batch.describe()
    assert shape["tuned"] and shape["grid"] >= 1 and shape["mode"] in ("fused", "streams")
    for pr, insts in zip(probs, data.values()):
        reset(pr, insts)
    batch.step(15)
    stream.synchronize()
    for pr, u in zip(probs, first):
        assert np.array_equal(pr.read_u(), u)


def test_batch_mixed_accuracy_against_fp64_path():
    """Members of the fused launch stay within the stated mixed tolerance of
    the FP64 path (itself oracle-checked) after start-up and Adams steps."""
    import torch
    from paper_2001_06113_gb300 import Batch
    data = members_data([(512, 4), (2048, 2)], seed=2)
    stream = torch.cuda.Stream()
    probs = [make_problem(insts, stream) for insts in data.values()]
    Batch(probs, stream=stream).step(NSTEPS)
    stream.synchronize()
    for pr, insts in zip(probs, data.values()):
        ub = pr.read_u()
        for b, it in enumerate(insts):
            ref = make_problem([it], precision="fp64")
            ref.step(NSTEPS)
            assert rel_l2(ub[b], ref.read_u(0)) < 2e-6
            ref.close()


def test_batch_validation():
    import torch
    from paper_2001_06113_gb300 import Batch, Problem, TdseError
    data = members_data([(256, 2), (512, 2)], seed=3)
    a, b = (make_problem(insts) for insts in data.values())
    f64 = make_problem(data[256], precision="fp64")
    with pytest.raises(TdseError):
        Batch([a, f64])                                  # FP64 member: unsupported
    other_dt = Problem((256,), 2 * DT, NSTEPS, precision="mixed")
    with pytest.raises(TdseError):
        Batch([a, other_dt])                             # different dt
    a.step(1)                                            # members at different steps
    batch = Batch([a, b], stream=torch.cuda.Stream())
    with pytest.raises(TdseError):
        batch.step(1)


# ------------------------------------------------------------ n = 16384, mixed
def test_mixed_16384_free_particle_closed_form():
    """V = 0 with a pulse: the scheme is exact, so the mixed-precision
    16384-point instance (FP64 four-step start and read-out, FP32 steps)
    matches e^{-i k^2 t + i k phi(t)} u^_k(0) to the FP32 rounding level."""
    from paper_2001_06113_gb300 import Problem
    M, n = 16384, 40
    pulse = synth.Pulse(3.0, 10.0, n * DT, (1.0,))
    rng = np.random.default_rng(6)
    x = synth.periodic_grid(M)
    ks = np.arange(-60, 61)
    c = (rng.normal(size=ks.size) + 1j * rng.normal(size=ks.size)) * np.exp(-0.001 * ks ** 2)
    u0 = np.exp(1j * np.outer(x, ks)) @ c
    pr = Problem((M,), DT, n, precision="mixed")
    pr.set_potential(np.zeros(M))
    pr.set_pulse(3.0, 10.0, n * DT, (1.0,))
    pr.set_initial(u0)
    assert np.array_equal(pr.read_u(0), u0)
    pr.step(n)
    T = n * DT
    ph = fields.phi_callable(pulse, 1)(T)[0]
    ref = np.exp(1j * np.outer(x, ks)) @ (c * np.exp(-1j * ks ** 2 * T + 1j * ks * ph))
    assert rel_l2(pr.read_u(0), ref) < 1e-6


def test_mixed_16384_against_fp64_8192():
    """V != 0: a well-resolved problem solved at n = 16384 (mixed) and at
    n = 8192 (FP64, oracle-checked path) agrees on the common grid points."""
    from paper_2001_06113_gb300 import Problem
    it16 = synth.periodic_1d_batch_member(3, dt=DT, nsteps=NSTEPS, sizes=(16384,))
    it8 = synth.periodic_1d_batch_member(3, dt=DT, nsteps=NSTEPS, sizes=(8192,))
    assert np.allclose(it16.u0[::2], it8.u0) and np.allclose(it16.V0[::2], it8.V0)
    u16 = make_problem([it16])
    u16.step(NSTEPS)
    ref = Problem((8192,), DT, NSTEPS, precision="fp64")
    load(ref, [it8])
    ref.step(NSTEPS)
    assert rel_l2(u16.read_u(0)[::2], ref.read_u(0)) < 2e-6


@pytest.mark.parametrize("mode", ["fused", "streams"])
def test_batch_modes_give_the_same_bits(mode):
    """Both execution modes of the Adams phase (one fused launch per step;
    each member's own kernel on its own stream, parallel graph branches)
    give the bits of the members run alone."""
    import torch
    from paper_2001_06113_gb300 import Batch
    data = members_data([(512, 6), (4096, 2), (16384, 1)], seed=9)
    stream = torch.cuda.Stream()
    probs = [make_problem(insts, stream) for insts in data.values()]
    batch = Batch(probs, stream=stream)
    batch.set_mode(mode)
    assert batch.describe()["mode"] == mode
    batch.step(NSTEPS - 5)
    stream.synchronize()
    for pr, insts in zip(probs, data.values()):
        ub = pr.read_u()
        for b, it in enumerate(insts):
            solo = make_problem([it])
            solo.step(NSTEPS - 5)
            assert np.array_equal(solo.read_u(0), ub[b]), (mode, it.shape, b)
            solo.close()


@pytest.mark.parametrize("n", [512, 2048, 8192, 16384])
def test_launch_shapes_give_the_same_bits(n):
    """The alternative launch shape of the one-CTA-per-instance kernel (half
    the threads, twice the points per thread of every transform pass) gives
    the bits of the default shape, through the start-up and the Adams steps."""
    data = members_data([(n, 2)], seed=13)
    insts = data[n]
    out = []
    for shape in (0, 1):
        pr = make_problem(insts)
        pr.set_shape_1d(shape)
        assert pr.shape_1d == shape
        pr.step(NSTEPS - 5)
        out.append(pr.read_u())
        pr.close()
    assert np.array_equal(out[0], out[1])


def test_set_initial_batch_equals_per_instance():
    """One copy of all instances' u0 gives the bits of per-instance uploads
    (periodic and free space)."""
    from paper_2001_06113_gb300 import Problem
    data = members_data([(512, 3)], seed=5)[512]
    a, b = make_problem(data), make_problem(data)
    b.set_initial_batch(np.stack([it.u0 for it in data]))
    a.step(12)
    b.step(12)
    assert np.array_equal(a.read_u(), b.read_u())
    insts = [synth.free_bump_gaussians((64,), seed=30 + i, dt=1e-3, nsteps=14) for i in range(2)]
    out = []
    for batched in (False, True):
        pr = Problem((64,), 1e-3, 14, batch=2, bc="free", nu=(512,), H=2.0)
        for i, it in enumerate(insts):
            pr.set_potential(it.V0, instance=i)
            if not batched:
                pr.set_initial(it.u0, instance=i)
        if batched:
            pr.set_initial_batch(np.stack([it.u0 for it in insts]))
        pr.step(10)
        out.append(pr.read_u())
    assert np.array_equal(out[0], out[1])
