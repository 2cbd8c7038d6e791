"""Host-side pieces of the gradient optimiser, on CPU: the paper's L1
objective (Sec. 3.3) and the quadratic dose-volume variant on hand-worked
values, the benchmark's analytic dose gradient against torch autograd of the
quadratic objective, the start plans, and the deliverable-plan projection
against the hand-worked projections of Sec. 2.2.1."""
import os

import numpy as np
import pytest
import torch

import bench
from paper_2512_18863_gb300 import optimize as OPT
from paper_2512_18863_gb300 import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _toy():
    D = torch.tensor([1.0, 2.0, 3.0, 0.5, 4.0, 1.5], dtype=torch.float64)
    masks = {"ptv": torch.tensor([1, 1, 1, 0, 0, 0], dtype=torch.bool),
             "bladder": torch.tensor([0, 0, 0, 1, 1, 0], dtype=torch.bool),
             "rectum": torch.tensor([0, 0, 0, 0, 1, 1], dtype=torch.bool)}
    return D, masks


def test_l1_objective_hand_values():
    D, m = _toy()
    # PTV: 100 (|1-2| + |2-2| + |3-2|) = 200; bladder: 1 (0.5 + 4) = 4.5;
    # rectum: 10 (4 + 1.5) = 55
    L = OPT.objective_l1(D, m, 2.0, weights={"ptv": 100.0, "bladder": 1.0, "rectum": 10.0})
    assert float(L) == pytest.approx(259.5, abs=1e-12)
    # structures absent from the masks are skipped; a zero weight drops a term
    L2 = OPT.objective_l1(D, m, 2.0, weights={"ptv": 100.0, "bladder": 0.0, "femur": 5.0})
    assert float(L2) == pytest.approx(200.0, abs=1e-12)


def test_quadratic_objective_hand_values():
    D, m = _toy()
    # PTV: 100 mean((-1)^2, 0, 1) = 200/3; OAR threshold 0.5 x 2 = 1:
    # bladder mean(0, 3^2) = 4.5; rectum 10 mean(3^2, 0.5^2) = 46.25
    L = OPT.objective_quadratic(D, m, 2.0)
    assert float(L) == pytest.approx(200.0 / 3.0 + 4.5 + 46.25, abs=1e-12)


def test_bench_dose_gradient_is_the_quadratic_objectives_gradient():
    rng = np.random.default_rng(3)
    D = torch.tensor(rng.uniform(0.0, 3.0, (6, 7, 8)), dtype=torch.float64, requires_grad=True)
    masks = {k: torch.tensor(rng.random((6, 7, 8)) < p) for k, p in
             (("ptv", 0.3), ("bladder", 0.2), ("rectum", 0.2))}
    dp = 0.9 * float(D.detach()[masks["ptv"]].median())
    L = OPT.objective_quadratic(D, masks, dp)
    L.backward()
    g = bench._objective_grad(D.detach(), masks, torch)
    torch.testing.assert_close(g, D.grad, rtol=1e-12, atol=1e-15)


def test_start_plans():
    w = S.small_pelvis(n=(8, 12, 12), n_cp=3, r_px=1)
    lv, jw, mu = OPT.open_field_start(w.plan, w.machine, margin=5.0)
    np.testing.assert_array_equal(lv[:, :, 0], np.repeat(w.plan.jaws[:, :1] - 5.0, lv.shape[1], 1))
    np.testing.assert_array_equal(lv[:, :, 1], np.repeat(w.plan.jaws[:, 1:2] + 5.0, lv.shape[1], 1))
    assert np.all(mu == 1.0) and np.array_equal(jw, w.plan.jaws)
    lv, jw, mu = OPT.closed_start(w.plan, w.machine)
    centre = 0.5 * (w.plan.jaws[:, 0] + w.plan.jaws[:, 1])
    assert np.all(lv == centre[:, None, None]) and np.all(mu == 0.0)


def test_deliverable_projection_matches_hand_worked_values():
    rows = np.loadtxt(os.path.join(GOLDEN, "projection_eq.txt"), comments="#")
    for a, b, wmin, F, ea, eb in rows:
        m = S.Machine(**{**S.machine_model(1, r_px=1).__dict__, "wmin_leaf": wmin, "f_leaf": F,
                         "wmin_jaw": wmin, "f_jaw": F, "eps_mu": 0.01})
        lv = np.array([[[a, b]]])
        jw = np.array([[a, b, a, b]])
        lp, jp, mp = OPT.project_plan(lv, jw, np.array([0.004]), m)
        assert tuple(lp[0, 0]) == pytest.approx((ea, eb), abs=1e-12)
        assert tuple(jp[0]) == pytest.approx((ea, eb, ea, eb), abs=1e-12)
        assert mp[0] == 0.01
