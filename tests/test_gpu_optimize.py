"""Gradient-based plan optimisation through the engine (Sec. 2.5.4, Sec. 3.3)."""
import numpy as np
import pytest
import torch

from paper_2512_18863_gb300 import optimize as opt
from paper_2512_18863_gb300 import synth as S
from paper_2512_18863_gb300.engine import DoseEngine

pytestmark = pytest.mark.gpu


def _case():
    w = S.small_pelvis(seed=41, n=(24, 40, 40), spacing=3.0, n_cp=12, r_px=5,
                       ptv_radii=(18.0, 15.0, 18.0))
    eng = DoseEngine(w.phantom, w.machine, w.plan.gantry_deg, w.plan.iso)
    masks = {k: w.phantom.masks[k] for k in ("ptv", "bladder", "rectum")}
    return w, eng, masks


def test_quadratic_objective_decreases_from_open_field():
    w, eng, masks = _case()
    init = opt.open_field_start(w.plan, w.machine)
    D0 = eng.forward(*init)
    presc = float(D0[torch.as_tensor(masks["ptv"], device=eng.device)].mean())
    res = opt.optimise(eng, masks, presc, init, n_iter=40, lr=0.5, lr_mu=0.05,
                       objective="quadratic")
    assert res.history[-1] < 0.5 * res.history[0]
    la, ja, ma = opt.project_plan(res.leaves, res.jaws, res.mu, w.machine)
    assert np.all(la[..., 1] - la[..., 0] >= w.machine.wmin_leaf - 1e-4)
    assert np.all(ma >= w.machine.eps_mu)
    eng.close()


def test_l1_objective_from_closed_zero_mu_start():
    """The paper's start (closed apertures, zero MU) receives gradient through
    the straight-through projection and the objective falls."""
    w, eng, masks = _case()
    init = opt.closed_start(w.plan, w.machine)
    res = opt.optimise(eng, masks, 2.0, init, n_iter=30, lr=1.0, lr_mu=0.2, objective="l1",
                       weights={"ptv": 100.0, "bladder": 1.0, "rectum": 10.0})
    assert res.history[-1] < 0.8 * res.history[0]
    assert res.mu.max() > 0.05
    eng.close()
