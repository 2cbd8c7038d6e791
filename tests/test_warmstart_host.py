"""Host-side pieces of the learned warm start (no GPU)."""
import os

import numpy as np
import pytest

from oracle import cnn_oracle as N
from paper_2512_18863_gb300 import synth as S
from paper_2512_18863_gb300 import warmstart as W


def test_plan_encoding_round_trips():
    m = S.machine_model(1004, r_px=4)
    rng = np.random.default_rng(0)
    lv = np.sort(rng.uniform(-60, 60, (5, 60, 2)), axis=-1)
    mu = rng.uniform(0.5, 2.0, 5)
    y = W.encode_plan(lv, mu)
    assert y.shape == (5, W.N_OUT)
    l2, m2 = W.decode_plan(y, m)
    np.testing.assert_allclose(l2, lv, rtol=1e-12)
    np.testing.assert_allclose(m2, mu, rtol=1e-12)
    y[:, 0], y[:, 1] = 0.5, -0.5                 # crossed pair: decoded in order
    l3, _ = W.decode_plan(y, m)
    assert np.all(l3[:, 0, 0] <= l3[:, 0, 1])


def test_parameter_layout_matches_the_oracle():
    p = N.init_params(1)
    v = W.flatten_params(p)
    assert v.size == 236601
    q = W.unflatten_params(v)
    for k, shp in W.param_layout():
        np.testing.assert_array_equal(q[k], p[k])


def test_warmstart_cases_are_seeded_and_varied():
    a, b = S.warmstart_case(11), S.warmstart_case(11)
    np.testing.assert_array_equal(a.phantom.masks["ptv"], b.phantom.masks["ptv"])
    c = S.warmstart_case(12)
    assert not np.array_equal(a.phantom.masks["ptv"], c.phantom.masks["ptv"])
    for w in (a, c):
        assert w.phantom.masks["ptv"].sum() > 50
        assert w.plan.n_cp == 36


@pytest.mark.skipif(not os.path.exists(W.default_weights_path()), reason="no trained weights")
def test_committed_weights_are_finite_and_complete():
    d = np.load(W.default_weights_path())
    assert d["params"].shape == (236601,)
    assert np.all(np.isfinite(d["params"]))
    assert len(d["train_seeds"]) >= 1000 and len(d["test_seeds"]) >= 50
    assert d["loss"][-1] < d["loss"][0]


def test_best_mu_scale_finds_the_closed_form_optimum():
    """With no organ above its threshold the objective is 100 mean((a D - p)^2),
    minimised at a = p mean(D) / mean(D^2); with an overdosed organ the optimum
    moves down and the search still finds the minimum of a fine grid."""
    import torch
    from types import SimpleNamespace
    rng = np.random.default_rng(4)
    n = (6, 7, 8)
    ptv = rng.random(n) < 0.3
    blad = (~ptv) & (rng.random(n) < 0.3)
    D = torch.tensor(rng.uniform(0.5, 1.5, n))
    case = SimpleNamespace(masks={"ptv": ptv, "bladder": blad, "rectum": np.zeros(n, bool)}, presc=2.0)
    Dn = D.clone()
    Dn[torch.as_tensor(blad)] = 0.0                   # organ dose zero: PTV term only
    a, j = W.best_mu_scale(case, Dn)
    d = Dn[torch.as_tensor(ptv)].numpy()
    a_ref = 2.0 * d.mean() / (d * d).mean()
    assert a == pytest.approx(a_ref, rel=1e-6)
    a2, j2 = W.best_mu_scale(case, D)                 # bladder pushes the scale down
    grid = np.linspace(0.25, 4.0, 20001)
    sel = {k: D[torch.as_tensor(v)] for k, v in case.masks.items()}
    vals = [float(W.objective_quadratic_sel(sel, g, 2.0)) for g in grid]
    assert j2 <= min(vals) + 1e-9
    assert a2 < a_ref
