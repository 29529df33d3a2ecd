"""Learned warm start end to end (small): train the network on steady solves of the
batched solver, seed held-out problems with its prediction, and check what it gains:
fewer steps and less wall time to R < 1e-7 than from the rest state (retired
instances leave the launched tiles), and the same steady profiles."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_warm_start_saves_steps_and_reaches_the_same_state():
    from paper_1702_01335_gb300.warmstart import evaluate
    r = evaluate(W.warm_start_draws(384, 11), W.warm_start_draws(48, 12), n_plain=2, epochs=300)
    print("\\n[warm start] median steps cold %.0f -> warm %.0f; mean %.0f -> %.0f; converged %s; "
          "max warm/cold profile difference %.2e" % (
              r["steps_median"]["cold"], r["steps_median"]["warm"], r["steps_mean"]["cold"],
              r["steps_mean"]["warm"], r["converged"], r["warm_vs_cold_final_profile_max_rel_diff"]))
    print("[warm start] wall s: cold %.3f, warm %.3f (inference and seeding %.3f)" % (
        r["wall_s"]["batched_cold"], r["wall_s"]["batched_warm"], r["wall_s"]["warm_inference_and_seeding"]))
    assert r["steps_median"]["warm"] < r["steps_median"]["cold"]
    assert r["steps_mean"]["warm"] < r["steps_mean"]["cold"]
    assert r["converged"]["warm"] >= r["converged"]["cold"] - 1
    assert r["warm_vs_cold_final_profile_max_rel_diff"] < 1e-3
