"""The stored oracle solutions (tests/golden/*.npz) still belong to the seeded
inputs that synth/ generates: inputs on the stored subgrid to 1e-13 and the
scalar parameters exactly (the stored solutions themselves come from
tests/golden/make_periodic_goldens.py, which runs only the oracle)."""
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _check(name, inst):
    g = np.load(os.path.join(GOLDEN, name))
    assert str(g["key"]) == inst.name
    st = int(g["stride"])
    sl = tuple(slice(None, None, st) for _ in inst.shape)
    p = inst.pulse
    assert np.array_equal(g["params"], np.array([inst.dt, inst.nsteps, p.A0, p.omega, p.T_pulse, *p.direction]))
    assert np.max(np.abs(inst.u0[sl] - g["u0_sample"])) <= 1e-13 * np.max(np.abs(g["u0_sample"]))
    assert np.max(np.abs(inst.V0[sl] - g["V0_sample"])) <= 1e-13 * np.max(np.abs(g["V0_sample"]))
    for n in g["steps"]:
        u = g[f"u_{int(n)}"]
        assert u.shape == inst.u0[sl].shape and np.all(np.isfinite(u))


def test_wells_512():
    _check("periodic_2d_wells_512.npz", synth.periodic_2d_wells(seed=2, M=512, dt=1e-3, nsteps=2000))


def test_wells_1024():
    _check("periodic_2d_wells_1024.npz", synth.periodic_2d_wells(seed=12, M=1024, dt=1e-3, nsteps=9))


def test_member_16384():
    g = np.load(os.path.join(GOLDEN, "periodic_1d_16384.npz"))
    inst = synth.periodic_1d_batch_member(int(g["member"]), seed=int(g["seed"]), nsteps=20)
    assert inst.shape == (16384,)
    _check("periodic_1d_16384.npz", inst)
