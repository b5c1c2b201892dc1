"""Checkpoint and resume (tdse_save / tdse_load): a run resumed from a
checkpoint continues bit for bit like the uninterrupted run, for the
periodic mixed 2D path (mid-way through the Adams steps), the periodic FP64
1D path (inside the start-up), the free-space path (2D, and 3D with FP32
transforms), the 3D periodic mixed path and a 1D grid in the four-step
layout."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _make(inst, **kw):
    from paper_2001_06113_gb300 import Problem
    pr = Problem(inst.shape, inst.dt, inst.nsteps, **kw)
    pr.set_potential(inst.V0, inst.vfac_table())
    if inst.pulse is not None:
        p = inst.pulse
        pr.set_pulse(p.A0, p.omega, p.T_pulse, p.direction)
    pr.set_initial(inst.u0)
    return pr


CASES = [
    (synth.periodic_2d_wells(seed=5, M=64, dt=1e-3, nsteps=40), dict(precision="mixed"), 12, 15),
    (synth.periodic_1d_cosine(seed=1, M=128, dt=1e-2, nsteps=40), dict(precision="fp64"), 4, 20),
    (synth.free_bump_gaussians((32, 32), seed=8, dt=1e-3, nsteps=40, A0=20.0, omega=100.0),
     dict(bc="free", nu=(256, 256), H=2.0), 9, 6),
    (synth.free_bump_gaussians((32, 32, 32), seed=8, dt=1e-3, nsteps=40, A0=20.0, omega=100.0,
                               direction=(1.0, -0.5, 0.3)),
     dict(bc="free", nu=(128, 128, 128), H=1.0, precision="mixed"), 9, 5),
    (synth.random_periodic((16, 16, 32), 7, 2e-3, 40, vamp=5.0, nmodes=2,
                           pulse=synth.Pulse(1.5, 10.0, 0.08, (1.0, -0.5, 0.7))), dict(precision="mixed"), 11, 7),
    (synth.periodic_1d_batch_member(77, seed=4, nsteps=40, sizes=(16384,)),
     dict(precision="mixed", layout_1d="passes"), 10, 6),
]


@pytest.mark.parametrize("inst,kw,k1,k2", CASES,
                         ids=["mixed2d", "fp64_1d_in_startup", "free2d", "free3d_mixed", "periodic3d_mixed",
                              "four_step_1d_mixed"])
def test_resume_is_bit_identical(inst, kw, k1, k2):
    from paper_2001_06113_gb300 import TdseError
    a = _make(inst, **kw)
    a.step(k1)
    blob = a.save()
    a.step(k2)
    ua = a.read_u(0)
    b = _make(inst, **kw)                 # fresh context, same configuration
    b.load(blob)
    assert b.step_index == k1
    b.step(k2)
    assert np.array_equal(b.read_u(0), ua)
    from paper_2001_06113_gb300 import Problem
    other = Problem(inst.shape, 2 * inst.dt, inst.nsteps, **kw)
    with pytest.raises(TdseError):
        other.load(blob)
