"""The collision-outcome classifier of the friction map (Sec. VI B/C) on
synthetic shell samples (host logic, no GPU)."""
import numpy as np

from paper_2505_10171_gb300 import validation as V

AIR = -np.ones(96)


def _touch(frac_inside=0.2, level=0.8):
    s = AIR.copy()
    s[: int(96 * frac_inside)] = level
    return s


def test_push_pull_captured_without_entering():
    seq = [AIR, AIR, _touch(0.1), _touch(0.3), _touch(0.2), _touch(0.25)]
    assert V.classify_outcome(seq) == V.PUSH_PULL


def test_enter_exit_inside_then_detached():
    inside = np.full(96, 0.95)
    seq = [AIR, _touch(0.3), inside, inside, _touch(0.4), AIR, AIR]
    assert V.classify_outcome(seq) == V.ENTER_EXIT


def test_captured_after_entering_and_left_behind_and_no_contact():
    inside = np.full(96, 0.95)
    assert V.classify_outcome([AIR, inside, _touch(0.3)]) == V.CAPTURED_AFTER_ENTERING
    assert V.classify_outcome([AIR, _touch(0.3), AIR]) == V.LEFT_BEHIND
    assert V.classify_outcome([AIR, AIR, AIR]) == V.NO_CONTACT


def test_mostly_wetted_shell_is_not_inside():
    # half the shell in the drop (mean phi 0) is contact, not immersion
    half = np.concatenate([np.full(48, 1.0), np.full(48, -1.0)])
    assert V.classify_outcome([AIR, half, half]) == V.PUSH_PULL


def test_capture_case_matches_the_paper_shapes():
    from paper_2505_10171_gb300 import workloads as W
    w = W.capture_case(1.0, 0.5, scale=1.0)
    p = w["params"]
    assert (p["nx"], p["ny"], p["nz"]) == (400, 181, 71)
    R_p, R_d = w["particles"][0]["R"], w["R_d"]
    assert R_p == 10.0 and R_d == 50.0
    assert abs(p["body_force_a"][0] * R_d ** 2 / p["sigma"] - 1.25) < 1e-12     # Bo = f_x R_d^2 / sigma
    g_d = p["body_force_a"][0] * 2.0 / 3.0 * np.pi * R_d ** 3
    assert 0.26 <= g_d <= 1.57                                                  # Table I, total force on the drop
    assert abs(1.0 * -p["g_particle"][2] / (p["sigma"] * R_p) - 5.23) < 1e-12    # mu g_p/(sigma R_p) at mu = 1
    assert 0.52 <= -p["g_particle"][2] <= 5.23                                  # Table I, particle weight
    # the rest overlap g_p/k_n stays below delta_R: a fluid node separates
    # sphere and substrate (full scale and the half scale of the map)
    for scale in (1.0, 0.5):
        w = W.capture_case(1.0, 0.5, scale=scale)
        assert w["particles"][0]["x"][2] - w["particles"][0]["R"] > 0.5
