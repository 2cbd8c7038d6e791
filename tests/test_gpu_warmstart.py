"""Learned warm start: what the trained network gains over the plain
optimiser, assessed by the exact engine (dose evaluations to reach the plain
optimiser's best objective of 100 evaluations from an open-field start)."""
import os

import numpy as np
import pytest

from paper_2512_18863_gb300 import warmstart as W

pytestmark = pytest.mark.gpu


def test_bad_proposal_falls_back_to_the_open_field_start():
    """A network with zero weights proposes closed leaves and minimum MU; the
    engine rates it worse than the open field, the optimiser falls back and
    then needs exactly the plain optimiser's evaluations (plus the judging one)."""
    p = {k: np.zeros(shp) for k, shp in W.param_layout()}
    net = W.WarmStartNet(batch_max=64, params=p)
    row = W.evaluate(net, [777], n_iter=30)[0]
    net.close()
    assert row["fallback"]
    assert row["j_proposal"] > row["j_open"]
    assert row["reached"]
    assert row["warm_evals"] == row["plain_evals"] + 1


@pytest.mark.skipif(not os.path.exists(W.default_weights_path()), reason="no trained weights")
def test_trained_network_needs_fewer_dose_evaluations_on_held_out_phantoms():
    d = np.load(W.default_weights_path())
    seeds = [int(s) for s in d["test_seeds"][-4:]]
    assert not set(seeds) & set(int(s) for s in d["train_seeds"])
    net = W.load_net()
    rows = W.evaluate(net, seeds)
    assert net.status() == 0
    net.close()
    s = W.summarise(rows)
    assert s["reached"] == len(rows)
    assert s["median_eval_ratio"] <= 0.75, s
    assert s["median_proposal_over_open"] < 1.0, s
