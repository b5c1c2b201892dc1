"""The accuracy-adaptive free-space selector on the GPU: a looser target
chooses a configuration that is not slower, and every choice is within its
bound of the high-accuracy reference."""
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


@pytest.mark.parametrize("shape", [(128,), (64, 64)])
def test_looser_target_is_not_slower_and_within_bound(shape):
    from paper_2001_06113_gb300.select import select_free
    inst = synth.free_bump_gaussians(shape, seed=5, dt=5e-4, nsteps=30)
    tight = select_free(inst, 1e-10, probe_steps=24)
    loose = select_free(inst, 1e-4, probe_steps=24)
    for r, eps in ((tight, 1e-10), (loose, 1e-4)):
        c = r["choice"]
        assert c.err <= 0.1 * eps, (eps, c)
        assert all(x.err is not None for x in r["candidates"])
    assert loose["choice"].ms_per_step <= 1.05 * tight["choice"].ms_per_step
    # the looser target admits the FP32-transform candidates
    assert any(x.precision == "mixed" for x in loose["candidates"])
    assert not any(x.precision == "mixed" for x in tight["candidates"])
