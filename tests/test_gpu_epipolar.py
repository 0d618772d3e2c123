"""GPU epipolar verification and static recovery (epipolar_verify, C ABI)
against the FP64 oracle (oracle/epipolar.py, Sec. IV-C, Eqs. (18), (19)) on
synthetic matches of two tracking frames, plus the edge cases."""
import numpy as np
import pytest

from oracle import epipolar as oepi
from paper_2602_21644_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dags():
    from paper_2602_21644_gb300 import build
    build.build()
    from paper_2602_21644_gb300 import dags as d
    d.load()
    return d


def run(dags, d, eps=1.0):
    n = d["records"].shape[0]
    cam = dags.Camera(*d["camera"].as_tuple())
    ctx = dags.Context(n, cam.width, cam.height, 1)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    g = t(d["records"])
    lab = t(d["labels"])
    dist, dbar = ctx.epipolar_verify(cam, t(d["pose_1"].ravel()), t(d["pose_2"].ravel()), t(d["p1"]), t(d["p2"]),
                                     t(d["gid"]), g, lab, eps=eps)
    torch.cuda.synchronize()
    status = None
    try:
        ctx.check()
    except dags.DagsError as e:
        status = e.code
    out = dict(d=dist.cpu().numpy(), dbar=dbar.cpu().numpy(), labels=lab.cpu().numpy(),
               mp=g[:, 11].cpu().numpy(), status=status)
    ctx.close()
    valid = (d["gid"] >= 0) & (d["gid"] < n)
    ref = oepi.verify(d["camera"].as_tuple(), d["pose_1"], d["pose_2"], d["p1"][valid], d["p2"][valid],
                      d["gid"][valid], n, d["records"][:, 11], d["labels"], eps=eps)
    return out, ref


@pytest.mark.parametrize("frames,n_sample", [((11, 16), 20_000), ((11, 12), 3_000)])
def test_matches_oracle(dags, frames, n_sample):
    d = synth.epipolar_matches(frames=frames, n_sample=n_sample)
    out, ref = run(dags, d)
    assert out["status"] is None
    np.testing.assert_allclose(out["d"], ref["d"], rtol=2e-7, atol=1e-9)
    has = ref["count"] > 0
    assert np.all(np.isnan(out["dbar"][~has]))
    np.testing.assert_allclose(out["dbar"][has], ref["dbar"][has], rtol=2e-7, atol=1e-9)
    near = np.abs(ref["dbar"] - 1.0) <= 1e-5
    ok = ~near
    np.testing.assert_array_equal(out["labels"][ok], ref["labels"][ok])
    np.testing.assert_array_equal(out["mp"][ok], ref["mp"][ok].astype(np.float32))
    restored = (d["labels"] == 1) & (out["labels"] == 0)
    print(f"\nframes {frames}: {len(d['gid'])} matches, restored {int(restored.sum())}, "
          f"moving restored {int((restored & d['moving']).sum())}")
    assert restored.sum() > 0


def test_out_of_range_ids_are_reported_and_skipped(dags):
    d = synth.epipolar_matches(n=50_000, n_sample=2_000)
    gid = d["gid"].copy()
    gid[::97] = 50_000 + 5           # beyond n
    gid[1::211] = -3
    d2 = dict(d, gid=gid)
    out, ref = run(dags, d2)          # the oracle sees the valid matches only
    assert out["status"] == -7        # DAGS_E_BOUNDS
    has = ref["count"] > 0
    np.testing.assert_allclose(out["dbar"][has], ref["dbar"][has], rtol=2e-7, atol=1e-9)


def test_no_matches_changes_nothing(dags):
    d = synth.epipolar_matches(n=20_000, n_sample=10)
    d2 = dict(d, p1=d["p1"][:0], p2=d["p2"][:0], gid=d["gid"][:0])
    out, _ = run(dags, d2)
    assert out["d"].size == 0 and np.all(np.isnan(out["dbar"]))
    np.testing.assert_array_equal(out["labels"], d["labels"])
    np.testing.assert_array_equal(out["mp"], d["records"][:, 11])
