"""GPU parity against stored FP64 oracle solutions at full size and length.

The stored solutions (tests/golden/*.npz) are written by
tests/golden/make_periodic_goldens.py, which runs only the CPU oracle on the
seeded inputs of synth/; each file keeps those inputs on its subgrid, and the
tests first check that the generator still reproduces them.  Compared on the stored
strided subgrid with the relative L2 norm (eq. l2err):

  * the 2D wells workload, 512^2, all 2000 steps (7 Richardson start-up +
    1993 Adams steps) at steps 10, 500, 1000, 2000: FP64 <= 1e-12, mixed
    <= 1e-6 (the stated mixed tolerance of this workload);
  * the same workload at 1024^2 (start-up + 2 Adams steps): FP64 <= 1e-12,
    mixed <= 1e-6;
  * a 1D instance with N = 16384 and V != 0 (an uneven-batch member, 20
    steps): mixed <= 2e-6 solo, and as a member of an uneven batch stepped
    by the fused persistent launch and by per-member streams, whose small
    members are compared with the oracle computed here.
"""
import math
import os

import numpy as np
import pytest

import synth
from oracle import fields
from oracle.periodic import PeriodicOracle, rel_l2

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _golden(name, inst):
    """The stored solution, after checking that the seeded inputs still match
    the ones it was computed from (to 1e-13: the generator's libm results may
    differ in the last bits between machines)."""
    g = np.load(os.path.join(GOLDEN, name))
    assert str(g["key"]) == inst.name
    st = int(g["stride"])
    sl = tuple(slice(None, None, st) for _ in inst.shape)
    p = inst.pulse
    assert np.allclose(g["params"], [inst.dt, inst.nsteps, p.A0, p.omega, p.T_pulse, *p.direction], rtol=1e-15, atol=0)
    assert np.max(np.abs(inst.u0[sl] - g["u0_sample"])) <= 1e-13 * np.max(np.abs(g["u0_sample"]))
    assert np.max(np.abs(inst.V0[sl] - g["V0_sample"])) <= 1e-13 * np.max(np.abs(g["V0_sample"]))
    return g


def _solve(insts, precision, keep, stream=None, layout_1d="auto"):
    from paper_2001_06113_gb300 import Problem
    it0 = insts[0]
    prob = Problem(it0.shape, it0.dt, it0.nsteps, precision=precision, batch=len(insts), stream=stream,
                   layout_1d=layout_1d)
    for b, it in enumerate(insts):
        prob.set_potential(it.V0, None, instance=b)
        p = it.pulse
        prob.set_pulse(p.A0, p.omega, p.T_pulse, p.direction, instance=b)
        prob.set_initial(it.u0, instance=b)
    out, done = {}, 0
    for n in sorted(keep):
        prob.step(n - done)
        done = n
        out[n] = prob.read_u(0)
    prob.close()
    return out


def _err(u, g, n):
    st = int(g["stride"])
    sl = tuple(slice(None, None, st) for _ in u.shape)
    return rel_l2(u[sl], g[f"u_{n}"])


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_wells_512_full_length(precision, tol):
    inst = synth.periodic_2d_wells(seed=2, M=512, dt=1e-3, nsteps=2000)
    g = _golden("periodic_2d_wells_512.npz", inst)
    steps = [int(n) for n in g["steps"]]
    got = _solve([inst], precision, steps)
    errs = {n: _err(got[n], g, n) for n in steps}
    print(precision, "512^2 vs oracle", errs)
    assert max(errs.values()) <= tol, errs


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_wells_1024(precision, tol):
    inst = synth.periodic_2d_wells(seed=12, M=1024, dt=1e-3, nsteps=9)
    g = _golden("periodic_2d_wells_1024.npz", inst)
    got = _solve([inst], precision, [9])
    err = _err(got[9], g, 9)
    print(precision, "1024^2 vs oracle", err)
    assert err <= tol, err


def _member_16384():
    g = np.load(os.path.join(GOLDEN, "periodic_1d_16384.npz"))
    inst = synth.periodic_1d_batch_member(int(g["member"]), seed=int(g["seed"]), nsteps=20)
    assert inst.shape == (16384,)
    return inst, _golden("periodic_1d_16384.npz", inst)


@pytest.mark.parametrize("layout", ["cta", "passes"])
def test_1d_16384_solo(layout):
    """One CTA per instance, and the four-step form through the 2D passes."""
    inst, g = _member_16384()
    got = _solve([inst], "mixed", [10, 20], layout_1d=layout)
    errs = {n: _err(got[n], g, n) for n in (10, 20)}
    print("1D 16384", layout, "vs oracle", errs)
    assert max(errs.values()) <= 2e-6, errs


@pytest.mark.parametrize("mode,layout", [("fused", "cta"), ("streams", "cta"), ("fused", "passes"),
                                         ("streams", "passes")])
def test_1d_16384_in_uneven_batch(mode, layout):
    """The n = 16384 member in the fused launch or on its own stream (one CTA
    per instance), or in the four-step layout beside the launch / on its
    stream; every member equals the same instance alone, bit for bit."""
    import torch
    from paper_2001_06113_gb300 import Batch, Problem
    big, g = _member_16384()
    small = [synth.periodic_1d_batch_member(700 + k, seed=4, nsteps=20, sizes=(n,)) for k, n in
             enumerate((256, 1024, 4096))]
    stream = torch.cuda.Stream()
    probs = []
    for it in [big] + small:
        pr = Problem(it.shape, it.dt, it.nsteps, precision="mixed", stream=stream,
                     layout_1d=layout if it is big else "auto")
        pr.set_potential(it.V0, None)
        p = it.pulse
        pr.set_pulse(p.A0, p.omega, p.T_pulse, p.direction)
        pr.set_initial(it.u0)
        probs.append(pr)
    batch = Batch(probs, stream=stream)
    batch.set_mode(mode)
    batch.step(20)
    stream.synchronize()
    err = _err(probs[0].read_u(0), g, 20)
    print(mode, layout, "batch member 16384 vs oracle", err)
    assert err <= 2e-6, err
    assert batch.describe()["members"][0]["layout"] == layout
    solo = _solve([big], "mixed", [20], layout_1d=layout)[20]
    assert np.array_equal(probs[0].read_u(0), solo)
    for pr, it in zip(probs[1:], small):
        ref = PeriodicOracle(it.shape, it.dt, it.V0, it.vfac, fields.phi_callable(it.pulse, 1)).solve(it.u0, 20)
        e = rel_l2(pr.read_u(0), ref)
        assert e <= 2e-6, (it.shape, e)
    batch.close()
    for pr in probs:
        pr.close()
