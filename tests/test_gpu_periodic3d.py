"""GPU parity of the 3D periodic step (Sec. 2 at d = 3) against the FP64 CPU
oracle, which is dimension-generic (its 3D pins: V = 0 exact with
advection, separable V against three 1D references).

The 3D step reuses the 2D pass kernels: the column pass (axis 0) over the
n1 n2 columns of [n0][n1 n2] carries the mode-space work, a transform pass
runs along axis 1, and the row pass (axis 2) over the n0 n1 rows carries the
implicit solve and V u.  Tolerances as in 2D: FP64 1e-12, mixed 2e-6.
"""
import numpy as np
import pytest

import synth
from oracle import fields
from oracle.periodic import PeriodicOracle, oracle_for, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def gpu_solve(insts, precision, order=8, keep=(), potential="separable", groups=None):
    from paper_2001_06113_gb300 import Problem
    it0 = insts[0]
    prob = Problem(it0.shape, it0.dt, it0.nsteps, order=order, precision=precision, batch=len(insts),
                   potential=potential)
    if groups:
        prob.set_step_groups(groups)
    for b, it in enumerate(insts):
        if potential == "separable":
            prob.set_potential(it.V0, it.vfac_table(), instance=b)
        else:
            prob.set_potential_fn(it.Vt, instance=b)
        if it.pulse is not None:
            p = it.pulse
            prob.set_pulse(p.A0, p.omega, p.T_pulse, p.direction, instance=b)
        prob.set_initial(it.u0, instance=b)
    out, done = {}, 0
    for n in sorted(set(keep) | {it0.nsteps}):
        prob.step(n - done)
        done = n
        out[n] = prob.read_u(-1)
    prob.close()
    return out


def _inst(shape, seed, nsteps=12, dt=2e-3, vamp=5.0):
    return synth.random_periodic(shape, seed, dt, nsteps, vamp=vamp, nmodes=2,
                                 pulse=synth.Pulse(1.5, 10.0, nsteps * dt, (1.0, -0.5, 0.7)))


@pytest.mark.parametrize("shape", [(16, 8, 32), (8, 16, 16), (32, 32, 8)])
def test_3d_fp64_matches_oracle(shape):
    inst = _inst(shape, 3)
    got = gpu_solve([inst], "fp64", keep=(3,))
    orc = oracle_for(inst)
    ref, kept = orc.solve(inst.u0, inst.nsteps, keep={3})
    for n, r in ((3, kept[3]), (inst.nsteps, ref)):      # inside the start-up, and after Adams steps
        err = rel_l2(got[n][0], r)
        print(shape, n, err)
        assert err <= 1e-12, (shape, n, err)


def test_3d_free_particle_exact():
    """V = 0 with a pulse: the scheme is exact (eq. uhatkinteq), and so is the GPU path."""
    shape = (16, 8, 16)
    inst = _inst(shape, 5, nsteps=10)
    inst.V0 = np.zeros(shape)
    got = gpu_solve([inst], "fp64")[inst.nsteps][0]
    t = inst.nsteps * inst.dt
    phi = fields.phi_callable(inst.pulse, 3)(t)
    k = np.meshgrid(*[np.fft.fftfreq(m, 1.0 / m) for m in shape], indexing="ij")
    ph = np.exp(-1j * sum(kk * kk for kk in k) * t + 1j * sum(kk * p for kk, p in zip(k, phi)))
    exact = np.fft.ifftn(np.fft.fftn(inst.u0) * ph)
    err = rel_l2(got, exact)
    print("3D free particle", err)
    assert err <= 1e-12, err


@pytest.mark.parametrize("order", [4, 6])
def test_3d_lower_orders(order):
    inst = _inst((16, 8, 16), 7, nsteps=10)
    got = gpu_solve([inst], "fp64", order=order)[inst.nsteps][0]
    ref = oracle_for(inst, order=order).solve(inst.u0, inst.nsteps)
    assert rel_l2(got, ref) <= 1e-12


def test_3d_mixed_within_tolerance():
    inst = _inst((16, 16, 32), 11, nsteps=24, vamp=8.0)
    got = gpu_solve([inst], "mixed")[inst.nsteps][0]
    ref = oracle_for(inst).solve(inst.u0, inst.nsteps)
    err = rel_l2(got, ref)
    print("3D mixed", err)
    assert err <= 2e-6, err


@pytest.mark.parametrize("shape", [(16, 16, 32), (64, 8, 64), (8, 16, 16)])
def test_3d_mixed_single_steps_equal_the_fused_chain(shape):
    """A run of Adams steps (the column pass of one step fused with the next,
    the mode work staged in shared memory) gives the bits of the same steps
    taken one at a time (separate begin / end column passes), for column
    blocks of one column per thread (n0 >= 32) and of several (n0 = 8)."""
    inst = _inst(shape, 31, nsteps=16, vamp=6.0)
    fused = gpu_solve([inst], "mixed", keep=(8,))
    single = gpu_solve([inst], "mixed", keep=tuple(range(1, 17)))
    for n in (8, 16):
        assert np.array_equal(fused[n], single[n]), n


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_3d_batch_members_and_groups_equal_solo_runs(precision):
    insts = [_inst((8, 8, 16), 20 + i, nsteps=11) for i in range(3)]
    batched = gpu_solve(insts, precision)[11]
    grouped = gpu_solve(insts, precision, groups=2)[11]
    assert np.array_equal(batched, grouped)
    for b, it in enumerate(insts):
        alone = gpu_solve([it], precision)[11][0]
        assert np.array_equal(batched[b], alone), b


def test_3d_general_potential_table():
    """A non-separable V(x, t) (a drifting well) through potential tables."""
    shape = (16, 8, 16)
    base = _inst(shape, 13, nsteps=10)
    X = np.meshgrid(*[synth.periodic_grid(m) for m in shape], indexing="ij")

    def Vt(t):
        return -8.0 * np.exp(-((X[0] - 0.3 * t) ** 2 + X[1] ** 2 + (X[2] + 0.5 * t) ** 2) / 0.8)

    base.Vt = Vt
    got = gpu_solve([base], "fp64", potential="table")[10][0]
    ref = PeriodicOracle(shape, base.dt, Vt, None, fields.phi_callable(base.pulse, 3)).solve(base.u0, 10)
    err = rel_l2(got, ref)
    print("3D moving well", err)
    assert err <= 1e-12, err


def test_3d_unsupported_parts():
    from paper_2001_06113_gb300 import Problem, TdseError
    p = Problem((8, 8, 16), 1e-3, 10, precision="mixed")
    with pytest.raises(TdseError) as e:
        p.set_residual_check(2, 1e-6)
    assert e.value.status == -7
    with pytest.raises(TdseError) as e:
        p.set_step_path("cluster")
    assert e.value.status == -7
    p.close()
