"""Learned warm start: what the trained network gains over the plain
optimiser, assessed by the exact engine (dose evaluations to reach the plain
optimiser's best objective of 100 evaluations from an open-field start)."""
import os

import numpy as np
import pytest

from paper_2512_18863_gb300 import warmstart as W

pytestmark = pytest.mark.gpu


def test_bad_proposal_falls_back_to_the_assessed_open_field_start():
    """A network with zero weights proposes closed leaves and minimum MU; the
    engine rates it worse than the assessed open field, the warm arm falls
    back to the control arm's start and then needs exactly the control's
    evaluations plus the proposal's assessment."""
    p = {k: np.zeros(shp) for k, shp in W.param_layout()}
    net = W.WarmStartNet(batch_max=64, params=p)
    row = W.evaluate(net, [777], n_iter=30)[0]
    net.close()
    assert row["fallback"]
    assert row["j_proposal"] > row["j_open_scaled"]
    assert row["reached"] and row["control_reached"]
    assert row["warm_evals"] == row["control_evals"] + 1


@pytest.mark.skipif(not os.path.exists(W.default_weights_path()), reason="no trained weights")
def test_trained_network_needs_fewer_dose_evaluations_on_held_out_phantoms():
    """Spec bar: on held-out phantoms the warm start reaches the plain
    optimiser's final objective in at most half its dose evaluations (median);
    against the control (the open field with the same MU assessment) the
    network must still save evaluations."""
    d = np.load(W.default_weights_path())
    seeds = [int(s) for s in d["test_seeds"][-8:]]
    assert not set(seeds) & set(int(s) for s in d["train_seeds"])
    net = W.load_net()
    rows = W.evaluate(net, seeds)
    assert net.status() == 0
    net.close()
    s = W.summarise(rows)
    print(s)
    assert s["reached"] == len(rows)
    assert s["median_eval_ratio"] <= 0.5, s
    assert s["median_warm_over_control"] < 1.0, s
    assert s["median_proposal_over_open"] < 1.0, s
