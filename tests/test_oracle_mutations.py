"""Planted mistakes: each test compiles a copy of the oracle with one plausible error (a flipped
sign, a dropped term, a swapped bound) and checks that a pin of tests/test_oracle_pins.py
rejects it.  This shows the pins constrain every part of the oracle they are meant to.

One plausible slip in the restart bookkeeping is deliberately absent: also setting r_prev = r on
a restart step.  It cannot change any result, because the step after a restart has k = 0,
which never restarts and always sets r_prev = r before the next test reads it (Section 3's
r(z^{n,k-1}) at k = 1 is r(z^{n,0})); no test can tell it apart from the oracle."""
import os

import numpy as np
import pytest

import oracle
from tests import test_oracle_pins as pins

MUTATIONS = {
    # r(z)^2: cross term of the metric P with the wrong sign (Section 2.2)
    "p_norm_cross_sign": ("return (omega / eta) * sx + 2.0 * cross + sy / (eta * omega);",
                          "return (omega / eta) * sx - 2.0 * cross + sy / (eta * omega);",
                          ["pd"]),
    # dual step: projection residual with the wrong sign (Section 2.2)
    "dual_step_sign": ("yp[i] = sigma * (clampd(s, lc[i], uc[i]) - s);",
                       "yp[i] = sigma * (s - clampd(s, lc[i], uc[i]));",
                       ["step", "firm"]),
    # primal step: gradient sign (Section 2.2)
    "primal_step_sign": ("xp[j] = clampd(x[j] - tau * (c[j] - aty[j]), lv[j], uv[j]);",
                         "xp[j] = clampd(x[j] - tau * (c[j] + aty[j]), lv[j], uv[j]);",
                         ["step", "firm"]),
    # Halpern: anchor term dropped (Section 3)
    "halpern_anchor_dropped": ("x[j] = a * ((1.0 + g) * xh[j] - g * x[j]) + b * x0[j];",
                               "x[j] = a * ((1.0 + g) * xh[j] - g * x[j]);",
                               ["solve"]),
    # reflection with the wrong sign (Section 3)
    "reflection_sign": ("y[i] = a * ((1.0 + g) * yh[i] - g * y[i]) + b * y0[i];",
                        "y[i] = a * ((1.0 + g) * yh[i] + g * y[i]) + b * y0[i];",
                        ["rate"]),
    # dual objective: lower and upper bound swapped (Section 4)
    "kkt_dobj_bounds": ("if (y[i] > 0.0) dobj += lc[i] * y[i];",
                        "if (y[i] > 0.0) dobj += uc[i] * y[i];",
                        ["kkt"]),
    # primal residual against the wrong interval (Section 4)
    "kkt_pres_interval": ("double p = ax[i] - clampd(ax[i], lc[i], uc[i]);",
                          "double p = ax[i] - clampd(ax[i], lc[i], lc[i]);",
                          ["kkt"]),
    # PID: controller output added instead of subtracted (Section 3)
    "pid_sign": ("double lw = log(omega) - (kp * e + ki * state[0] + kd * de);",
                 "double lw = log(omega) + (kp * e + ki * state[0] + kd * de);",
                 ["pid"]),
    # PID: derivative term uses the previous error with the wrong sign (Section 3)
    "pid_derivative": ("double de = state[2] != 0.0 ? e - state[1] : 0.0;",
                       "double de = state[2] != 0.0 ? e + state[1] : 0.0;",
                       ["pid"]),
    # restart condition 2: "no local progress" inverted (Section 3)
    "restart_progress": ("if (r <= beta_n * r0 && r > r_prev) return 1;",
                         "if (r <= beta_n * r0 && r < r_prev) return 1;",
                         ["restart"]),
    # restart condition 3 against k instead of the total count (Section 3)
    "restart_artificial": ("if ((double)k >= beta_a * (double)(t + 1)) return 1;",
                           "if ((double)k >= beta_a * (double)(k + 1)) return 1;",
                           ["restart"]),
    # restart point: the anchor set to the pre-step iterate z instead of the PDHG output z^
    # (Section 3, "restart ... at the current solution", read as z^ = T(z))
    "restart_anchor_at_z": ("for (int32_t j = 0; j < n; ++j) x[j] = x0[j] = xh[j];",
                            "for (int32_t j = 0; j < n; ++j) { x0[j] = x[j]; x[j] = xh[j]; }",
                            ["restart_trace"]),
    # r0 never refreshed after the first epoch (Section 3: r0 = r(z^{n,0}) of the current epoch)
    "restart_r0_first_epoch_only": ("if (k == 0) r0 = r;", "if (t == 0) r0 = r;",
                                    ["restart_epochs"]),
    # r0 taken from the step that decided the restart instead of the new epoch's first step
    "restart_r0_at_restart_step": ([("if (k == 0) r0 = r;", "if (t == 0) r0 = r;"),
                                    ("      k = 0;\n      if (trace && t < trace_cap) trace[4 * t + 2] = 1.0;",
                                     "      k = 0;\n      r0 = r;\n      if (trace && t < trace_cap) trace[4 * t + 2] = 1.0;")],
                                   ["restart_epochs"]),
    # Ruiz: factor 1/max instead of 1/sqrt(max)
    "ruiz_sqrt": ("for (int32_t i = 0; i < m; ++i) fr[i] = fr[i] > 0.0 ? 1.0 / sqrt(fr[i]) : 1.0;",
                  "for (int32_t i = 0; i < m; ++i) fr[i] = fr[i] > 0.0 ? 1.0 / fr[i] : 1.0;",
                  ["scale"]),
}

CHECKS = {
    "pd": lambda: pins.test_P_positive_definite_iff_eta_norm_below_one(),
    "firm": lambda: [pins.test_T_firmly_nonexpansive_in_P(s) for s in range(3)],
    "rate": lambda: [pins.test_halpern_rate_bound(g, "small") for g in (0.5, 1.0)],
    "step": lambda: (pins.test_pdhg_step_hand_worked(), [pins.test_step_lands_in_X_and_Y(s) for s in range(3)]),
    "kkt": lambda: (pins.test_kkt_hand_worked(), pins.test_kkt_zero_at_planted_optimum(lambda: pins.gen.free_and_boxed_mix(2, 60, 80))),
    "pid": lambda: (pins.test_pid_three_restarts_hand_worked(), pins.test_pid_proportional_only_is_pdlp_smoothing()),
    "restart": lambda: pins.test_restart_decisions_hand_labelled(),
    "solve": lambda: ([pins.test_solve_reaches_planted_optimum(s) for s in range(2)],
                      [pins.test_solve_matches_vertex_enumeration(s) for s in range(3)]),
    "scale": lambda: (pins.test_ruiz_equilibrates_rows_and_columns(), pins.test_pock_chambolle_pass()),
    "restart_trace": lambda: pins.test_restart_trace_hand_worked(),
    "restart_epochs": lambda: [pins.test_restart_decisions_follow_the_epoch_definitions(s) for s in range(3)],
}


def test_unmutated_oracle_passes_every_check():
    for name, fn in CHECKS.items():
        fn()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    sites, checks = MUTATIONS[name][:-1], MUTATIONS[name][-1]
    pairs = sites[0] if len(sites) == 1 else [sites]
    src = oracle.source()
    for old, new in pairs:
        assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
        src = src.replace(old, new)
    path = oracle.compile_variant(src, os.path.join(tmp_path, f"lib_{name}.so"))
    with oracle.using_library(path):
        for chk in checks:
            with pytest.raises(AssertionError):
                CHECKS[chk]()
