"""What the learned MP proposal gains over the method without it: the
experiment of paper_2602_21644_gb300.mp_eval (train on one synthetic
sequence, evaluate fresh prior / stale prior / learned proposal on a held-out one)
and its assertions."""
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


@pytest.fixture(scope="module")
def experiment(dags):
    from paper_2602_21644_gb300 import mp_eval
    return mp_eval.experiment(dags)


@pytest.fixture(scope="module")
def result(experiment):
    from paper_2602_21644_gb300 import mp_eval
    m = mp_eval.metrics(experiment)
    print("\n" + ", ".join(f"{k} {v:.4f}" for k, v in m.items()))
    return m


def test_scheduled_refreshes(experiment):
    # the trigger refreshes at frame 0 and at least every N_max = 10 frames;
    # the frames it refreshes are those its previous frame decided
    from paper_2602_21644_gb300 import mp_eval
    sm = mp_eval.schedule_metrics(experiment)
    print("\n" + repr(sm))
    T = len(experiment["fresh"])
    for name in ("scheduled", "scheduled_learned", "calibrated", "calibrated_learned"):
        h = experiment[name]
        ref = [f for f, r in enumerate(h) if r["refreshed"]]
        assert ref[0] == 0 and all(b - a <= 10 for a, b in zip(ref, ref[1:] + [T]))
        assert sm[name]["calls"] == len(ref) <= T
    assert sm["stale"]["calls"] == (T + 9) // 10


def test_calibrated_trigger(experiment):
    # The default e_ref (5 cm) lies below the background residual of these
    # sequences, so R = 1 every frame and the trigger fires on every frame.
    # Fitted on the training sequence (e_ref = twice the largest mean
    # background residual at any prior age, theta halfway between the scores
    # of fresh and nine-frame-old priors), R stays below 1/2 and the trigger
    # skips frames on the held-out sequence
    from paper_2602_21644_gb300 import mp_eval
    cal = experiment["calibration"]
    sm = mp_eval.schedule_metrics(experiment)
    print("\n" + repr(cal) + "\n" + repr({k: sm[k] for k in ("calibrated", "calibrated_learned")}))
    T = len(experiment["fresh"])
    assert cal["e_ref"] > 0 and np.isfinite(cal["theta"])
    assert min(cal["S_fresh"], cal["S_stale"]) <= cal["theta"] <= max(cal["S_fresh"], cal["S_stale"])
    R = [r["score"][1].item() for r in experiment["calibrated"]]
    assert np.mean(np.array(R) < 1.0) > 0.9, R
    assert sm["calibrated"]["calls"] < T, sm


def test_training_converges(result):
    assert result["loss_last"] < 0.9 * result["loss_first"], result


def test_learned_map_closer_to_fresh_prior_than_stale_prior(result):
    # per-pixel MP between refreshes against the fresh-prior arm's map: the
    # dynamic region (M > 0.5) is recovered far better (0.74 against 0.59
    # IoU). The mean absolute error is reported but varies between trainings
    # (0.084-0.110 against 0.096 for the stale prior): the background's fused
    # M_p takes the dispersion of a radius-2 disk of residuals, which the
    # network's 3x3 receptive field cannot form exactly
    assert result["iou_l"] > result["iou_s"] + 0.05, result
    assert result["mae_l"] < result["mae_s"] + 0.03, result


def test_label_agreement_does_not_drop(result):
    # static/dynamic labels of the Gaussians: agreement with the fresh-prior arm's
    # labels between refreshes. The labels integrate the map over frames
    # through Eq. (9) and the median threshold, so the per-pixel gain shows
    # only weakly here: it must not lose agreement (training is not
    # bit-reproducible: FP32 atomics in the gradient reductions)
    assert result["agree_l"] >= result["agree_s"] - 0.02, result
    assert np.isfinite(result["gt_l"]) and np.isfinite(result["gt_s"])


def test_training_on_rendered_frames_generalises(dags):
    # 2,000 frames the plain method generates on the mapping room at 640x480
    # (observations rendered by the library), then the held-out ray-cast
    # sequence at 640x480: the learned map beats the stale prior
    from paper_2602_21644_gb300 import mp_eval
    ex = mp_eval.experiment_rendered(dags, n_frames=2000, steps=2500, eval_frames=30)
    m = mp_eval.metrics(ex)
    print("\n" + ", ".join(f"{k} {v:.4f}" for k, v in m.items()))
    assert m["loss_last"] < 0.9 * m["loss_first"], m
    assert m["mae_l"] < m["mae_s"] and m["iou_l"] > m["iou_s"], m


def test_gain_against_ground_truth_when_the_map_follows_the_objects(dags):
    # The map keeps its moving objects at their current positions (as mapping
    # would), so residuals no longer flag the background the objects left or
    # now cover. Between semantic refreshes the stale prior misses the parts
    # of each object that moved out of its old mask; the learned proposal,
    # trained on the fresh-prior maps of another sequence, recovers them:
    # dynamic-label IoU against the ground-truth moving Gaussians rises.
    from paper_2602_21644_gb300 import mp_eval
    ex = mp_eval.experiment(dags, follow=True)
    m = mp_eval.metrics(ex)
    print("\n" + ", ".join(f"{k} {v:.4f}" for k, v in m.items()))
    sm = mp_eval.schedule_metrics(ex)
    print(repr(sm))
    # with the default constants every arm separates the moving Gaussians
    # only weakly within 40 frames (the fresh prior reaches 0.22 IoU: the
    # labels need M^t above max(median, 0.5), and M^t rises from its
    # uninformed 0.2 at the rates of Eq. (11) scaled by rho between
    # refreshes); the learned proposal still recovers part of what the stale
    # prior misses (measured 0.183 against 0.175)
    assert m["gt_j"] > m["gt_s"], m
    assert m["gt_l"] > m["gt_s"], m
