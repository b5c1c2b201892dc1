"""FP64 residual check of the mixed-precision implicit step: the residual is
small and reported; a redo in FP64 (forced with tol = 0) keeps the result
within the mixed tolerance of the FP64 path; off-path configurations are
refused."""
import numpy as np
import pytest

import synth
from oracle.periodic import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _problem(inst, precision, every=0, tol=0.0, batch_of=None):
    from paper_2001_06113_gb300 import Problem
    insts = batch_of or [inst]
    pr = Problem(inst.shape, inst.dt, inst.nsteps, precision=precision, batch=len(insts))
    if every:
        pr.set_residual_check(every, tol)
    for b, it in enumerate(insts):
        pr.set_potential(it.V0, it.vfac_table(), instance=b)
        if it.pulse is not None:
            p = it.pulse
            pr.set_pulse(p.A0, p.omega, p.T_pulse, p.direction, instance=b)
        pr.set_initial(it.u0, instance=b)
    return pr


CASES = [
    synth.periodic_2d_wells(seed=3, M=64, dt=1e-3, nsteps=40),
    synth.periodic_1d_cosine(seed=1, M=256, dt=2e-3, nsteps=40),
]


@pytest.mark.parametrize("inst", CASES, ids=["2d_64", "1d_256"])
def test_residual_small_and_reported_without_changing_results(inst):
    plain = _problem(inst, "mixed")
    plain.step(40)
    chk = _problem(inst, "mixed", every=5, tol=1e-3)
    chk.step(40)
    rho, corr, checks = chk.residual_report()
    assert checks == 7                               # steps 10, 15, .., 40 (after the 7 start-up steps)
    assert 0.0 < rho[0] < 1e-6 and corr[0] == 0
    assert np.array_equal(chk.read_u(0), plain.read_u(0))


@pytest.mark.parametrize("inst", CASES, ids=["2d_64", "1d_256"])
def test_forced_fp64_redo_stays_within_tolerance(inst):
    ref = _problem(inst, "fp64")
    ref.step(40)
    u_ref = ref.read_u(0)
    redo = _problem(inst, "mixed", every=1, tol=0.0)
    redo.step(40)
    rho, corr, checks = redo.residual_report()
    assert checks == 33 and corr[0] == 33
    plain = _problem(inst, "mixed")
    plain.step(40)
    e_redo, e_plain = rel_l2(redo.read_u(0), u_ref), rel_l2(plain.read_u(0), u_ref)
    assert e_redo < 2e-6 and e_plain < 2e-6, (e_redo, e_plain)


def test_batch_instances_checked_independently():
    insts = [synth.periodic_2d_wells(seed=10 + i, M=32, dt=1e-3, nsteps=20) for i in range(3)]
    pr = _problem(insts[0], "mixed", every=4, tol=1e-3, batch_of=insts)
    pr.step(20)
    rho, corr, checks = pr.residual_report()
    assert checks == 4 and np.all(rho > 0) and np.all(rho < 1e-6) and not corr.any()
    assert len(set(rho.tolist())) == 3


def test_residual_check_refused_off_path():
    from paper_2001_06113_gb300 import Problem, TdseError
    with pytest.raises(TdseError):
        Problem((64,), 1e-3, 10, precision="fp64").set_residual_check(5, 1e-6)
    with pytest.raises(TdseError):
        Problem((64,), 1e-3, 10, precision="mixed").set_residual_check(-1, 1e-6)
    with pytest.raises(TdseError):   # free space in FP64: nothing to check
        Problem((64,), 1e-3, 10, bc="free", nu=(512,), H=2.0).set_residual_check(5, 1e-6)
    Problem((64,), 1e-3, 10, bc="free", nu=(512,), H=1.0, precision="mixed").set_residual_check(5, 1e-6)
