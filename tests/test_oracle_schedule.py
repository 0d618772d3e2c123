"""Pins of the semantic-on-demand trigger oracle (Sec. IV-B, Eqs. (13)-(16)):
closed forms and special cases that fix each term (no GPU)."""
import numpy as np

from oracle import mp as M
from oracle import schedule as S


def test_residual_term_closed_form():
    cfg = S.ScheduleConfig(w_u=0.0, w_r=1.0)
    assert S.score(0.7, 0.0, cfg) == (0.0, 0.0)
    assert S.score(0.7, 0.0125, cfg) == (0.25, 0.25)          # e_ref / 4
    assert S.score(0.7, 0.05, cfg) == (1.0, 1.0)              # e_bar = e_ref
    assert S.score(0.7, 0.2, cfg) == (1.0, 1.0)               # clipped at 1


def test_uncertainty_term_alone():
    cfg = S.ScheduleConfig(w_u=1.0, w_r=0.0)
    for u in (0.0, 0.125, 0.5, 1.0):
        assert S.score(u, 0.3, cfg)[1] == u


def test_weighted_sum():
    cfg = S.ScheduleConfig(w_u=0.25, w_r=0.75, e_ref=0.1)
    R, s = S.score(0.5, 0.05, cfg)
    assert R == 0.5 and s == 0.25 * 0.5 + 0.75 * 0.5


def test_threshold_is_strict():
    cfg = S.ScheduleConfig(w_u=1.0, w_r=0.0, theta=0.5, n_max=100)
    assert S.step(0.5, 0.0, 3, False, cfg)[3] is False
    assert S.step(0.5 + 2 ** -20, 0.0, 3, False, cfg)[3] is True


def test_fixed_cadence_when_scores_never_exceed_theta():
    # S <= w_u + w_r = 1, so theta = 1 leaves only the skip-interval rule:
    # a refresh every N_max frames starting at frame 0
    rng = np.random.default_rng(0)
    U, e = rng.random(47), rng.random(47)
    for n_max in (1, 3, 10):
        cfg = S.ScheduleConfig(theta=1.0, n_max=n_max)
        frames, _ = S.run(U, e, cfg)
        assert frames == list(range(0, 47, n_max))


def test_trigger_restarts_the_interval():
    # the scores of frames 3 and 4 exceed theta: frames 4 and 5 are refreshed;
    # the forced cadence restarts from frame 5 (next forced refresh at 15)
    U = np.zeros(30)
    U[[3, 4]] = 0.9
    cfg = S.ScheduleConfig(w_u=1.0, w_r=0.0, theta=0.35, n_max=10)
    frames, rs = S.run(U, np.zeros(30), cfg)
    assert frames == [0, 4, 5, 15, 25]
    assert [s for _, s in rs][3] == 0.9


def test_residual_mean_is_the_background_region_mean():
    # constant depth residual 0.03 m on the background, 0.2 m inside an
    # instance: the verified-set mean is 0.03; it is also the MP oracle's
    # region-0 mean of e(p), Eq. (4)
    W, H = 16, 12
    inst = np.zeros(W * H, np.uint8)
    inst[40:70] = 1
    d_rend = np.full(W * H, 2.0)
    d_obs = d_rend + np.where(inst == 0, 0.03, 0.2)
    c = np.full((W * H, 3), 0.5)
    px = M.pixel_mp(inst, d_obs, c, d_rend, c.copy(), np.array([[0.1, 0.05], [0.9, 0.8]]), M.MPConfig(), (W, H))
    e_bar = S.residual_mean(px["e"], inst)
    assert abs(e_bar - 0.03) < 1e-12
    assert abs(e_bar - px["mean"][0]) < 1e-12
    assert S.residual_mean(px["e"], np.ones(W * H, np.uint8)) == 0.0   # empty background
