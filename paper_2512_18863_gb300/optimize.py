"""Gradient-based VMAT plan optimisation through the dose engine.

The paper optimises leaf positions, jaws and MUs directly with a
gradient-based optimiser (Adam), starting from closed apertures with zero MU,
for 100 iterations (Sec. 2.5.4, Sec. 3.3), with the objective

    L = l_PTV || D_PTV - D_p ||_1 + sum_s l_s || D_s ||_1          (Eq. L)

over the PTV and the organs at risk.  Delivered parameters are the projected
ones (Sec. 2.2.1); the projection is applied inside the engine on every
forward, and the straight-through reading of the backward pass lets the
closed / zero-MU start receive gradient.

The dose and its adjoint run in the CUDA library (engine.DoseFn); the
objective is a handful of elementwise torch ops on the dose grid.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from .engine import DoseEngine

# weights the paper's grid search selected (Sec. 3.3): PTV 100, bladder 1,
# rectum 10, femoral heads 0.1, external 10
PAPER_WEIGHTS = {"ptv": 100.0, "bladder": 1.0, "rectum": 10.0, "femur": 0.1, "body": 10.0}


def objective_l1(D, masks, prescription, weights=PAPER_WEIGHTS):
    """Eq. L of the paper (sums of absolute values over each structure)."""
    L = weights["ptv"] * (D[masks["ptv"]] - prescription).abs().sum()
    for name, lam in weights.items():
        if name == "ptv" or name not in masks or lam == 0.0:
            continue
        L = L + lam * D[masks[name]].abs().sum()
    return L


def objective_quadratic(D, masks, prescription, weights=None, oar_fraction=0.5):
    """Quadratic dose-volume variant: l_PTV mean_PTV (D - D_p)^2 +
    sum_s l_s mean_s max(D - f D_p, 0)^2."""
    weights = weights or {"ptv": 100.0, "bladder": 1.0, "rectum": 10.0}
    L = weights["ptv"] * ((D[masks["ptv"]] - prescription) ** 2).mean()
    for name, lam in weights.items():
        if name == "ptv" or name not in masks or lam == 0.0:
            continue
        ex = torch.clamp(D[masks[name]] - oar_fraction * prescription, min=0.0)
        L = L + lam * (ex ** 2).mean()
    return L


def open_field_start(plan, machine, margin=5.0):
    """Every leaf pair open to the CP's jaw opening (plus margin), MU 1."""
    leaves = np.zeros_like(plan.leaves)
    leaves[:, :, 0] = plan.jaws[:, None, 0] - margin
    leaves[:, :, 1] = plan.jaws[:, None, 1] + margin
    return leaves, plan.jaws.copy(), np.ones_like(plan.mu)


def closed_start(plan, machine):
    """The paper's start: closed apertures at the field centre and zero MU."""
    centre = 0.5 * (plan.jaws[:, 0] + plan.jaws[:, 1])
    leaves = np.repeat(centre[:, None, None], plan.leaves.shape[1], 1).repeat(2, 2)
    return leaves, plan.jaws.copy(), np.zeros_like(plan.mu)


@dataclass
class OptResult:
    leaves: np.ndarray
    jaws: np.ndarray
    mu: np.ndarray
    history: list = field(default_factory=list)
    dose_evals: int = 0


def optimise(engine: DoseEngine, masks: dict, prescription: float, init, n_iter=100, lr=0.5,
             lr_mu=0.05, objective="l1", weights=None, target=None, optimise_jaws=True,
             callback=None) -> OptResult:
    """Adam over (leaves, jaws, MU).  init = (leaves, jaws, mu) arrays.
    Stops early when the objective reaches `target` (dose-evaluation count is
    reported; one evaluation = one forward + one adjoint)."""
    dev = engine.device
    leaves = torch.tensor(init[0], dtype=torch.float32, device=dev, requires_grad=True)
    jaws = torch.tensor(init[1], dtype=torch.float32, device=dev, requires_grad=optimise_jaws)
    mu = torch.tensor(init[2], dtype=torch.float32, device=dev, requires_grad=True)
    m = {k: torch.as_tensor(v, device=dev) for k, v in masks.items()}
    groups = [{"params": [leaves], "lr": lr}, {"params": [mu], "lr": lr_mu}]
    if optimise_jaws:
        groups.append({"params": [jaws], "lr": lr})
    opt = torch.optim.Adam(groups)
    fn = objective_l1 if objective == "l1" else objective_quadratic
    hist = []
    evals = 0
    for it in range(n_iter):
        opt.zero_grad(set_to_none=True)
        D = engine(leaves, jaws, mu)
        L = fn(D, m, prescription, weights) if weights is not None else fn(D, m, prescription)
        L.backward()
        evals += 1
        val = float(L.detach())
        hist.append(val)
        if callback is not None:
            callback(it, val)
        if target is not None and val <= target:
            break
        opt.step()
    return OptResult(leaves.detach().cpu().numpy(), jaws.detach().cpu().numpy(),
                     mu.detach().cpu().numpy(), hist, evals)


def project_plan(leaves, jaws, mu, machine):
    """The deliverable plan: the hardware projection of Sec. 2.2.1 applied to
    raw parameters (what the engine doses)."""
    def pair(a, b, wmin, F):
        c = 0.5 * (a + b)
        w = np.maximum(b - a, wmin)
        c = np.clip(c, -F, F)
        return c - 0.5 * w, c + 0.5 * w

    la, lb = pair(leaves[..., 0], leaves[..., 1], machine.wmin_leaf, machine.f_leaf)
    jx0, jx1 = pair(jaws[:, 0], jaws[:, 1], machine.wmin_jaw, machine.f_jaw)
    jy0, jy1 = pair(jaws[:, 2], jaws[:, 3], machine.wmin_jaw, machine.f_jaw)
    return (np.stack([la, lb], -1), np.stack([jx0, jx1, jy0, jy1], -1),
            np.maximum(mu, machine.eps_mu))
