"""1D periodic grids beyond one CTA: N = n0 n1 points through the 2D pass
kernels (the four-step transform with the twiddle between the passes, the
grid stored transposed), FP64 from N = 16384 and mixed from N = 32768, up to
2^20 points.

Against the FP64 oracle (Sec. 2): at N = 16384 the stored direct-sum oracle
solution (tests/golden), at larger N the oracle with its DFT pair through
numpy's FFT (pinned against the direct sums in the CPU suite).  FP64 1e-12,
mixed 2e-6; V = 0 against the exact solution.  Such contexts (and any 1D
context created with the four-step layout) join uneven batches.
"""
import os

import numpy as np
import pytest

import synth
from oracle import fields
from oracle.periodic import PeriodicOracle, oracle_for, rel_l2

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def gpu_solve(insts, precision, keep=(), potential="separable", groups=None):
    from paper_2001_06113_gb300 import Problem
    it0 = insts[0]
    prob = Problem(it0.shape, it0.dt, it0.nsteps, precision=precision, batch=len(insts), potential=potential)
    if groups:
        prob.set_step_groups(groups)
    for b, it in enumerate(insts):
        if potential == "separable":
            prob.set_potential(it.V0, it.vfac_table(), instance=b)
        else:
            prob.set_potential_fn(it.Vt, instance=b)
        p = it.pulse
        prob.set_pulse(p.A0, p.omega, p.T_pulse, p.direction, instance=b)
        prob.set_initial(it.u0, instance=b)
    assert np.array_equal(prob.read_u(-1)[0], it0.u0)          # the transposed layout round trip
    out, done = {}, 0
    for n in sorted(set(keep) | {it0.nsteps}):
        prob.step(n - done)
        done = n
        out[n] = prob.read_u(-1)
    prob.close()
    return out


def member(N, i=0, nsteps=12):
    return synth.periodic_1d_batch_member(900 + i, seed=4, nsteps=nsteps, sizes=(N,))


def test_fp64_16384_against_stored_oracle():
    g = np.load(os.path.join(GOLDEN, "periodic_1d_16384.npz"))
    inst = synth.periodic_1d_batch_member(int(g["member"]), seed=int(g["seed"]), nsteps=20)
    got = gpu_solve([inst], "fp64", keep=(10,))
    st = int(g["stride"])
    for n in (10, 20):
        err = rel_l2(got[n][0][::st], g[f"u_{n}"])
        print("FP64 16384 vs oracle", n, err)
        assert err <= 1e-12, (n, err)


@pytest.mark.parametrize("N,precision,tol", [(32768, "fp64", 1e-12), (32768, "mixed", 2e-6),
                                             (65536, "mixed", 2e-6), (262144, "mixed", 2e-6)])
def test_large_1d_against_oracle(N, precision, tol):
    inst = member(N)
    got = gpu_solve([inst], precision, keep=(4,))
    orc = oracle_for(inst, transform="fft")
    ref, kept = orc.solve(inst.u0, inst.nsteps, keep={4})
    for n, r in ((4, kept[4]), (inst.nsteps, ref)):
        err = rel_l2(got[n][0], r)
        print(N, precision, n, err)
        assert err <= tol, (N, precision, n, err)


def test_free_particle_exact_65536():
    inst = member(65536, i=3, nsteps=10)
    inst.V0 = np.zeros_like(inst.V0)
    got = gpu_solve([inst], "fp64")[10][0]
    t = inst.nsteps * inst.dt
    phi = fields.phi_callable(inst.pulse, 1)(t)[0]
    k = np.fft.fftfreq(65536, 1.0 / 65536)
    exact = np.fft.ifft(np.fft.fft(inst.u0) * np.exp(-1j * k * k * t + 1j * k * phi))
    err = rel_l2(got, exact)
    print("free particle 65536", err)
    assert err <= 1e-12, err


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_and_groups_equal_solo_runs(precision):
    insts = [member(32768, i=10 + i, nsteps=10) for i in range(3)]
    batched = gpu_solve(insts, precision)[10]
    grouped = gpu_solve(insts, precision, groups=3)[10]
    assert np.array_equal(batched, grouped)
    for b, it in enumerate(insts):
        assert np.array_equal(batched[b], gpu_solve([it], precision)[10][0]), b


@pytest.mark.parametrize("N", [16384, 32768])
def test_mixed_single_steps_equal_the_fused_chain(N):
    """Mixed runs of Adams steps in the four-step layout (the staged column
    kernel fusing the end of a step with the begin of the next) give the bits
    of the same steps taken one at a time through the generic column passes."""
    from paper_2001_06113_gb300 import Problem
    inst = member(N, i=30, nsteps=16)

    def run(chunks):
        prob = Problem((N,), inst.dt, inst.nsteps, precision="mixed", layout_1d="passes")
        prob.set_potential(inst.V0, inst.vfac_table())
        p = inst.pulse
        prob.set_pulse(p.A0, p.omega, p.T_pulse, p.direction)
        prob.set_initial(inst.u0)
        out = []
        for k in chunks:
            prob.step(k)
            out.append(prob.read_u(0))
        prob.close()
        return out

    fused = run([8, 8])
    single = run([1] * 16)
    assert np.array_equal(fused[0], single[7]) and np.array_equal(fused[1], single[15])


def test_potential_table_32768():
    inst = member(32768, i=20, nsteps=10)
    x = synth.periodic_grid(32768)

    def Vt(t):
        return -20.0 * np.exp(-(np.angle(np.exp(1j * (x - 3.0 * t)))) ** 2 / 0.5)

    inst.Vt = Vt
    got = gpu_solve([inst], "fp64", potential="table")[10][0]
    ref = PeriodicOracle((32768,), inst.dt, Vt, None, fields.phi_callable(inst.pulse, 1),
                         transform="fft").solve(inst.u0, 10)
    err = rel_l2(got, ref)
    print("moving well 32768", err)
    assert err <= 1e-12, err


@pytest.mark.parametrize("mode", ["fused", "streams"])
def test_in_an_uneven_batch(mode):
    """A 32768-point member (four-step layout) in an uneven batch with members
    of one CTA per instance: its pass chain runs on its own stream beside the
    fused launch (or all members on their streams); every member equals the
    same instances run alone, bit for bit, and the large one stays within the
    mixed bound of the oracle.  The FP64 residual check is not built for the
    four-step layout."""
    import torch
    from paper_2001_06113_gb300 import Batch, Problem, TdseError
    big = [member(32768, i, nsteps=12) for i in range(2)]
    small = [synth.periodic_1d_batch_member(40 + i, seed=4, nsteps=12, sizes=(n,)) for i, n in enumerate((512, 2048))]
    stream = torch.cuda.Stream()

    def make(insts):
        it0 = insts[0]
        pr = Problem(it0.shape, it0.dt, it0.nsteps, batch=len(insts), precision="mixed", stream=stream)
        for b, it in enumerate(insts):
            pr.set_potential(it.V0, None, instance=b)
            p = it.pulse
            pr.set_pulse(p.A0, p.omega, p.T_pulse, p.direction, instance=b)
            pr.set_initial(it.u0, instance=b)
        return pr

    groups = [big, [small[0]], [small[1]]]
    probs = [make(g) for g in groups]
    batch = Batch(probs, stream=stream)
    batch.set_mode(mode)
    assert [m["layout"] for m in batch.describe()["members"]] == ["passes", "cta", "cta"]
    batch.step(12)
    stream.synchronize()
    for pr, g in zip(probs, groups):
        solo = make(g)
        solo.step(12)
        stream.synchronize()
        assert np.array_equal(pr.read_u(), solo.read_u()), g[0].shape
        solo.close()
    ref = oracle_for(big[1], transform="fft").solve(big[1].u0, 12)
    e = rel_l2(probs[0].read_u(1), ref)
    assert e <= 2e-6, e
    with pytest.raises(TdseError) as err:
        probs[0].set_residual_check(2, 1e-6)
    assert err.value.status == -7
    batch.close()
    for pr in probs:
        pr.close()
