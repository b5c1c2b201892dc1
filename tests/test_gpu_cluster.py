"""The 2D mixed Adams step over CTA clusters (512 x 512) against the pass
kernels, and the pass kernels' instance groups on parallel streams.

The cluster kernel keeps the transform intermediates in distributed shared
memory and streams the state, history and V by TMA; it does the same
arithmetic, operation for operation, as the row and column pass kernels, so
the two paths must agree bit for bit on every run: several runs of different
lengths (each launch begins and ends a run), batches that do not fill the
resident clusters evenly, lower Adams orders, potential tables (shared and
per instance), and the FP64 residual check.  Its oracle parity follows
from these bitwise comparisons and the pass kernels' own oracle parity
(test_gpu_periodic, the full-length golden test, potential tables, orders,
residual check).  The pass kernels are the default; the cluster path runs
when selected.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

M = 512


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _problem(insts, path, order=8, potential="separable", res_every=0):
    from paper_2001_06113_gb300 import Problem
    it0 = insts[0]
    prob = Problem(it0.shape, it0.dt, it0.nsteps, order=order, precision="mixed", batch=len(insts),
                   potential=potential)
    prob.set_step_path(path)
    for b, it in enumerate(insts):
        if potential == "separable":
            prob.set_potential(it.V0, it.vfac_table(), instance=b)
        elif potential == "table":
            prob.set_potential_fn(it.Vt, instance=b)
        p = it.pulse
        prob.set_pulse(p.A0, p.omega, p.T_pulse, p.direction, instance=b)
        prob.set_initial(it.u0, instance=b)
    if potential == "shared_table":
        prob.set_potential_fn(it0.Vt, instance=-1)
    if res_every:
        prob.set_residual_check(res_every, 1e-6)
    return prob


def _runs(prob, runs):
    out = []
    for k in runs:
        prob.step(k)
        out.append(prob.read_u(-1).copy())
    return out


def _both(insts, runs, **kw):
    a = _problem(insts, "passes", **kw)
    b = _problem(insts, "cluster", **kw)
    assert a.step_path == "passes" and b.step_path == "cluster"
    ra, rb = _runs(a, runs), _runs(b, runs)
    a.close()
    b.close()
    return ra, rb


def test_cluster_path_selectable_at_512():
    from paper_2001_06113_gb300 import Problem, TdseError
    inst = synth.periodic_2d_wells(seed=2, M=M, dt=1e-3, nsteps=20)
    p = Problem(inst.shape, inst.dt, inst.nsteps, precision="mixed")
    assert p.step_path == "passes"                 # default
    p.set_step_path("cluster")
    assert p.step_path == "cluster"
    shape = p.describe_steps()
    assert shape["path"] == "cluster" and shape["clusters"] >= 1 and shape["ctas_per_cluster"] == 16
    p.close()
    p = Problem(inst.shape, inst.dt, inst.nsteps, precision="fp64")
    with pytest.raises(TdseError) as e:
        p.set_step_path("cluster")
    assert e.value.status == -7
    assert p.step_path == "passes"
    p.close()


def test_cluster_equals_passes_bitwise():
    """Runs of 10 (start-up + 3 Adams steps), 1 and 9 steps; 3 instances."""
    insts = [synth.periodic_2d_wells(seed=2 + i, M=M, dt=1e-3, nsteps=20) for i in range(3)]
    ra, rb = _both(insts, [10, 1, 9])
    for k, (x, y) in enumerate(zip(ra, rb)):
        assert np.array_equal(x, y), k


def test_cluster_uneven_batch_bitwise():
    """More instances than resident clusters (some clusters take two)."""
    from paper_2001_06113_gb300 import Problem
    insts = [synth.periodic_2d_wells(seed=30 + i, M=M, dt=1e-3, nsteps=12) for i in range(9)]
    ra, rb = _both(insts, [12])
    assert np.array_equal(ra[0], rb[0])


@pytest.mark.parametrize("order", [4, 6])
def test_cluster_lower_orders_bitwise(order):
    insts = [synth.periodic_2d_wells(seed=40 + order, M=M, dt=1e-3, nsteps=16)]
    ra, rb = _both(insts, [9, 7], order=order)
    for x, y in zip(ra, rb):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("potential", ["table", "shared_table"])
def test_cluster_potential_tables_bitwise(potential):
    insts = [synth.moving_wells_2d(seed=6 + i, M=M, dt=1e-3, nsteps=14) for i in range(2)]
    ra, rb = _both(insts, [10, 4], potential=potential)
    for x, y in zip(ra, rb):
        assert np.array_equal(x, y)


def test_cluster_residual_check_bitwise():
    insts = [synth.periodic_2d_wells(seed=50, M=M, dt=1e-3, nsteps=20)]
    ra, rb = _both(insts, [20], res_every=4)
    assert np.array_equal(ra[0], rb[0])


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_step_groups_bitwise(precision):
    """Instance groups on parallel streams give the same bits as one chain."""
    from paper_2001_06113_gb300 import Problem
    insts = [synth.random_periodic((64, 32), 60 + i, 2e-3, 16, vamp=6.0,
                                   pulse=synth.Pulse(1.5, 10.0, 0.032, (1.0, 0.4))) for i in range(5)]
    out = {}
    for G in (1, 2, 4, 5, 8):
        prob = Problem((64, 32), 2e-3, 16, precision=precision, batch=len(insts))
        prob.set_step_groups(G)
        for b, it in enumerate(insts):
            prob.set_potential(it.V0, None, instance=b)
            p = it.pulse
            prob.set_pulse(p.A0, p.omega, p.T_pulse, p.direction, instance=b)
            prob.set_initial(it.u0, instance=b)
        prob.step(11)
        prob.step(5)
        out[G] = prob.read_u(-1)
        assert prob.describe_steps()["groups"] == min(G, len(insts))
        prob.close()
    for G in (2, 4, 5, 8):
        assert np.array_equal(out[G], out[1]), G

