"""GPU semantic-on-demand trigger (semantic_trigger, C ABI) against the FP64
oracle (oracle/schedule.py, Sec. IV-B, Eqs. (13)-(16)).

1. A 200-frame sequence of seeded statistics (U_bar and the background
   residual mean, the two inputs of the trigger) driven through the kernel
   frame by frame, each frame's refresh taken from the previous decision:
   the refreshed frames must be identical, R and S equal to FP64 rounding.
2. The whole chain on one ray-cast frame: mp_update then semantic_trigger
   against oracle.mp.mp_update then oracle.schedule.step."""
import dataclasses

import numpy as np
import pytest

from oracle import schedule as osch

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dags():
    from paper_2602_21644_gb300 import build
    build.build()
    from paper_2602_21644_gb300 import dags as d
    d.load()
    return d


def drive(dags, ctx, U, e, counts, cfg):
    """Run the kernel over the sequence; returns refreshed frames and (e_bar, R, S) per frame."""
    stats = torch.zeros((len(U), dags.MP_STATS_HEAD + 4), dtype=torch.float64)
    stats[:, 1] = torch.from_numpy(U)
    stats[:, dags.MP_STATS_HEAD] = torch.from_numpy(counts)
    stats[:, dags.MP_STATS_HEAD + 1] = torch.from_numpy(e)
    stats = stats.cuda()
    state = torch.zeros(2, dtype=torch.int32, device="cuda")
    scores = torch.zeros((len(U), 3), dtype=torch.float64, device="cuda")
    frames, nxt = [], True
    for t in range(len(U)):
        if nxt:
            frames.append(t)
        ctx.semantic_trigger(stats[t], state, nxt, cfg=cfg, score=scores[t])
        nxt = bool(state[1].item())
    return frames, scores.cpu().numpy()


@pytest.mark.parametrize("kw", [dict(), dict(theta=1.0), dict(w_u=0.8, w_r=0.2, theta=0.3, n_max=4),
                                dict(w_u=0.0, w_r=1.0, theta=0.5, e_ref=0.02)])
def test_sequence_matches_oracle(dags, kw):
    rng = np.random.default_rng(7)
    T = 200
    U = rng.beta(2.0, 5.0, T)                       # mostly below theta, sometimes above
    e = rng.gamma(2.0, 0.012, T)                    # metres, around e_ref / 2
    counts = np.where(rng.random(T) < 0.05, 0.0, 1000.0)   # an empty background now and then
    ctx = dags.Context(16, 8, 8, 1)
    cfg = dags.default_sched_cfg(**kw)
    frames, sc = drive(dags, ctx, U, e, counts, cfg)
    ocfg = dataclasses.replace(osch.ScheduleConfig(), **kw)
    e_used = np.where(counts > 0, e, 0.0)
    ref_frames, rs = osch.run(U, e_used, ocfg)
    S = np.array([s for _, s in rs])
    R = np.array([r for r, _ in rs])
    # no score within FP64 rounding of theta: the decisions are exact
    assert np.min(np.abs(S - ocfg.theta)) > 1e-12
    assert frames == ref_frames
    np.testing.assert_array_equal(sc[:, 0], e_used)
    np.testing.assert_allclose(sc[:, 1], R, rtol=1e-15, atol=0)
    np.testing.assert_allclose(sc[:, 2], S, rtol=1e-15, atol=1e-16)
    if kw.get("theta") == 1.0:
        assert frames == list(range(0, T, ocfg.n_max))
    ctx.close()


def test_invalid_config_rejected(dags):
    ctx = dags.Context(16, 8, 8, 1)
    stats = torch.zeros(dags.MP_STATS_HEAD + 4, dtype=torch.float64, device="cuda")
    state = torch.zeros(2, dtype=torch.int32, device="cuda")
    for kw in (dict(w_u=0.6, w_r=0.6), dict(w_u=-0.1, w_r=1.1), dict(e_ref=0.0), dict(n_max=0)):
        with pytest.raises(dags.DagsError):
            ctx.semantic_trigger(stats, state, True, cfg=dags.default_sched_cfg(**kw))
    ctx.close()


def test_after_mp_update_matches_oracle(dags):
    from test_gpu_mp import mp_scene, run_both
    d = mp_scene(20_000, frame=30, width=160, height=120)
    gpu, ref = run_both(dags, d, seg_refreshed=False)
    ctx = dags.Context(16, 8, 8, 1)
    stats = torch.from_numpy(gpu["stats"]).cuda()
    state = torch.tensor([4, 0], dtype=torch.int32, device="cuda")
    score = torch.zeros(3, dtype=torch.float64, device="cuda")
    ctx.semantic_trigger(stats, state, False, score=score)
    sc = score.cpu().numpy()
    st = state.cpu().numpy()
    e_bar = osch.residual_mean(ref["pixel"]["e"], d["inst"])
    since, R, S, nxt = osch.step(ref["U_bar"], e_bar, 4, False)
    # FP32 residuals and U_tilde on the GPU against FP64: 1e-5 as for the MP update
    assert abs(sc[0] - e_bar) <= 1e-5 * max(1.0, e_bar)
    assert abs(sc[1] - R) <= 1e-5 / 0.05
    assert abs(sc[2] - S) <= 1e-4
    assert st[0] == since == 5
    if abs(S - 0.35) > 1e-4:
        assert bool(st[1]) == nxt
    ctx.close()
