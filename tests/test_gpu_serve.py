"""The request loop on the GPU: a seeded trace of 1D periodic, 2D periodic
and 2D free-space solves admitted by HBM budget and overlapped on the
device; every result equals the same solve run alone, and the mixed
periodic results stay within the stated tolerance of the FP64 path."""
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


def _trace():
    return synth.serve_requests(seed=7, rate=60.0, duration=0.4, T_range=(0.01, 0.03), sizes_1d=(1024, 4096),
                                sizes_2d=(128, 256), sizes_free=(64,))


def test_results_equal_alone_and_in_the_mix():
    import torch
    from paper_2001_06113_gb300.serve import Server, TorchBackend, requests_from_trace
    reqs = requests_from_trace(_trace())
    assert len({r.bc for r in reqs}) == 2 and len(reqs) >= 10
    be = TorchBackend()
    srv = Server(be, hbm_budget=4 << 30, max_active=32)
    st = srv.run(reqs)
    assert st["requests"] == len(reqs) and st["peak_active"] > 1
    for r in reqs:
        alone = TorchBackend()
        h = alone.prepare(r)
        alone.start(h)
        torch.cuda.synchronize()
        assert np.array_equal(alone.finish(h), r.result), (r.rid, r.bc, r.inst.shape)


def test_mixed_results_within_tolerance_of_fp64():
    from paper_2001_06113_gb300.serve import Request, Server, TorchBackend
    trace = [(t, k, inst) for t, k, inst in _trace() if k != "free"][:6]
    reqs = [Request(i, t, inst, precision="mixed") for i, (t, k, inst) in enumerate(trace)]
    refs = [Request(i, 0.0, inst, precision="fp64") for i, (t, k, inst) in enumerate(trace)]
    Server(TorchBackend(), hbm_budget=4 << 30).run(reqs)
    Server(TorchBackend(), hbm_budget=4 << 30).run(refs)
    for r, f in zip(reqs, refs):
        assert rel_l2(r.result, f.result) < 1e-6, (r.inst.shape, r.nsteps)


def test_free_space_fp32_requests_within_tolerance():
    """Free-space requests routed to the FP32-transform variant (contour for
    eps = 1e-4 with FP32 sums) stay within the mixed bar of FP64 solves on
    the eps = 1e-10 contour, and equal the same solves run alone."""
    import torch
    from paper_2001_06113_gb300.serve import (Request, Server, TorchBackend, free_contour_params,
                                              requests_from_trace)
    trace = synth.serve_requests(seed=8, rate=60.0, duration=0.5, T_range=(0.01, 0.03), sizes_1d=(1024,),
                                 sizes_2d=(128,), sizes_free=(64, 128))
    reqs = requests_from_trace(trace, free_precision="mixed")
    free = [r for r in reqs if r.bc == "free"]
    assert free and all(r.precision == "mixed" for r in free)
    Server(TorchBackend(), hbm_budget=4 << 30, max_active=16).run(reqs)
    for r in free:
        ref = Request(r.rid, 0.0, r.inst, bc="free", precision="fp64", free=free_contour_params(r.inst, 1e-10))
        be = TorchBackend()
        h = be.prepare(ref)
        be.start(h)
        torch.cuda.synchronize()
        assert rel_l2(r.result, be.finish(h)) < 2e-6, (r.inst.shape, r.nsteps)
        alone = TorchBackend()
        h = alone.prepare(r)
        alone.start(h)
        torch.cuda.synchronize()
        assert np.array_equal(alone.finish(h), r.result)


def test_budget_limits_concurrency():
    from paper_2001_06113_gb300 import Problem
    from paper_2001_06113_gb300.serve import Request, Server, TorchBackend
    insts = [synth.periodic_2d_wells(seed=40 + i, M=256, dt=1e-3, nsteps=30) for i in range(6)]
    need = Problem.workspace_bytes_for((256, 256), 1e-3, 30, precision="mixed")
    reqs = [Request(i, 0.0, inst) for i, inst in enumerate(insts)]
    srv = Server(TorchBackend(), hbm_budget=2 * need + need // 2)
    srv.run(reqs)
    assert srv.peak_active == 2 and srv.peak_bytes <= 2 * need + need // 2


def test_bad_requests_fail_alone():
    """A request with a NaN in V (non-finite result) and an invalid one (grid
    not a power of two) fail with their own errors; the rest of the stream is
    served and equals the same solves alone."""
    import copy
    import torch
    from paper_2001_06113_gb300.serve import Request, Server, TorchBackend
    insts = [synth.periodic_2d_wells(seed=60 + i, M=64, dt=1e-3, nsteps=20) for i in range(4)]
    bad = copy.deepcopy(insts[1])
    bad.V0 = bad.V0.copy()
    bad.V0[3, 5] = np.nan
    odd = synth.random_periodic((48,), 3, 1e-3, 12)
    reqs = [Request(0, 0.0, insts[0]), Request(1, 0.0, bad), Request(2, 0.0, insts[2]), Request(3, 0.0, odd),
            Request(4, 0.0, insts[3])]
    st = Server(TorchBackend(), hbm_budget=2 << 30).run(reqs)
    assert st["completed"] == 3 and st["failed"] == 2
    assert reqs[1].error.startswith("finish") and "NONFINITE" in reqs[1].error
    assert reqs[3].error.startswith("prepare")
    for r in (reqs[0], reqs[2], reqs[4]):
        be = TorchBackend()
        h = be.prepare(r)
        be.start(h)
        torch.cuda.synchronize()
        assert np.array_equal(be.finish(h), r.result)


def test_stated_stream_sample_against_the_oracle():
    """The request stream at its stated sizes and lengths (1D N 2^10..2^16,
    2D periodic 2^7..2^10, free space 2^6..2^9 with nu = 8n and FP32
    transforms on the eps = 1e-4 contour, T ~ U[0.5, 2]): the two cheapest
    requests of each class (points x steps) of the first second of arrivals,
    served together, against the FP64 oracle (periodic: <= 1e-6 as stated for
    the stream; free space: <= 2e-6 against the oracle on the same contour)."""
    from oracle import fields, gamma
    from oracle.freespace import FreeSpaceOracle
    from oracle.periodic import oracle_for
    from paper_2001_06113_gb300.serve import Server, TorchBackend, requests_from_trace
    trace = synth.serve_requests(seed=5, rate=200.0, duration=1.0, T_range=(0.5, 2.0),
                                 sizes_1d=tuple(2 ** p for p in range(10, 17)),
                                 sizes_free=tuple(2 ** p for p in range(6, 10)))
    picked = []
    for kind in ("1d", "2d", "free"):
        cls = sorted((x for x in trace if x[1] == kind), key=lambda x: np.prod(x[2].shape) * x[2].nsteps)
        picked += cls[:2]
    reqs = requests_from_trace(picked, free_precision="mixed", free_R=8)
    Server(TorchBackend(), hbm_budget=8 << 30, max_active=8).run(reqs)
    for r, (t, kind, inst) in zip(reqs, picked):
        assert r.error is None, r.error
        if kind == "free":
            fp = r.free
            rules = [gamma.GammaRule.for_nu(M, nu, fp["H"], q=fp["gauss_q"], n_r=fp["n_r"])
                     for M, nu in zip(inst.shape, fp["nu"])]
            ref = FreeSpaceOracle(rules, inst.dt, inst.V0, inst.vfac,
                                  fields.phi_callable(inst.pulse, inst.dim)).solve(inst.u0, inst.nsteps)
            tol = 2e-6
        else:
            ref = oracle_for(inst).solve(inst.u0, inst.nsteps)
            tol = 1e-6
        err = rel_l2(r.result, ref)
        print(kind, inst.shape, inst.nsteps, err)
        assert err <= tol, (kind, inst.shape, err)
