"""Failure detection without a GPU fault: a bounded device wait that runs out
is reported as DAGS_E_TIMEOUT through the status word, and the context stays
usable afterwards."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dags():
    from paper_2602_21644_gb300 import build
    build.build()
    from paper_2602_21644_gb300 import dags as d
    d.load()
    return d


@pytest.mark.parametrize("spins", [0, 1, 1000])
def test_wait_timeout_is_reported_and_context_survives(dags, spins):
    from paper_2602_21644_gb300 import synth
    sc = synth.tiny_scene(0)
    cam = dags.Camera(*sc.camera.as_tuple())
    ctx = dags.Context(sc.records.shape[0], cam.width, cam.height, 1)
    ctx.selftest_timeout(spins)
    with pytest.raises(dags.DagsError) as e:
        ctx.check()
    assert e.value.code == -4                     # DAGS_E_TIMEOUT
    ctx.check()                                   # the status word was cleared
    gauss = torch.from_numpy(sc.records).cuda()
    poses = torch.from_numpy(np.ascontiguousarray(sc.poses)).cuda()
    targets = torch.from_numpy(sc.targets).cuda()
    image, last, loss = ctx.forward(gauss, cam, poses, targets)
    torch.cuda.synchronize()
    ctx.check()
    assert np.isfinite(loss.item()) and loss.item() > 0
    ctx.close()


def test_selftest_rejects_bad_limits(dags):
    ctx = dags.Context(16, 16, 16, 1)
    for spins in (-1, 1 << 25):
        with pytest.raises(dags.DagsError) as e:
            ctx.selftest_timeout(spins)
        assert e.value.code == -1                 # DAGS_E_INVAL
    ctx.close()
