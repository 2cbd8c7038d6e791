"""Learned warm start for the plan optimiser.

The paper's Discussion ("Future directions") proposes a network that learns
delivery parameters from target and organ-at-risk masks, with the dose
engine as the arbiter.  Here a 5-layer BF16 CNN (include/pdrt_cnn.h) maps the
beam's-eye-view projection of the PTV, bladder and rectum masks of each
control point to its 60 leaf pairs and MU; it is trained on plans that the
engine's own gradient optimiser (optimize.optimise) produced on seeded
synthetic pelvis phantoms.  The optimiser then starts from the proposal; the
plain open-field start stays the fallback, and the engine decides between
them by objective value.

Everything numeric runs in the CUDA library: the projection
(pdrt_bev_project), the network forward, backward and Adam update
(pdrt_cnn_*) and the dose engine.  This module marshals arguments, encodes
plans as network targets and drives data generation, training and the
warm-versus-plain evaluation.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from . import synth as S
from .engine import DoseEngine
from .optimize import objective_quadratic, open_field_start, optimise

SIDE = _lib.CNN_SIDE
N_OUT = _lib.CNN_OUT
BEV_PITCH_MM = 2.5          # 64 x 2.5 mm = 16 cm field at the isocentre plane
LEAF_SCALE_MM = 50.0        # network units: leaf position / 50 mm
MU_SCALE = 2.0              # MU / 2
STRUCTURES = ("ptv", "bladder", "rectum")


def _stream():
    return torch.cuda.current_stream().cuda_stream


def param_layout():
    """(name, shape) of the FP32 parameter vector, in order."""
    out = []
    cin = 3
    for l in range(1, 5):
        out += [(f"W{l}", (64, 3, 3, cin)), (f"b{l}", (64,))]
        cin = 64
    out += [("W5", (N_OUT, 1024)), ("b5", (N_OUT,))]
    return out


def flatten_params(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], np.float64).reshape(-1) for k, _ in param_layout()])


def unflatten_params(v) -> dict:
    v = np.asarray(v)
    out, o = {}, 0
    for k, shp in param_layout():
        n = int(np.prod(shp))
        out[k] = v[o:o + n].reshape(shp)
        o += n
    assert o == v.size
    return out


def init_params(seed: int) -> dict:
    """He-style initial weights, zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for k, shp in param_layout():
        if k.startswith("b"):
            p[k] = np.zeros(shp)
        else:
            fan = int(np.prod(shp[1:]))
            gain = 2.0 if k != "W5" else 1.0
            p[k] = rng.normal(0.0, math.sqrt(gain / fan), size=shp)
    return p


class WarmStartNet:
    """Handle of the CUDA network (weights, Adam state and buffers on the GPU)."""

    def __init__(self, batch_max: int = 256, params: dict | None = None, seed: int = 0,
                 device=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        self.batch_max = int(batch_max)
        with torch.cuda.device(self.device):
            self._h = _lib.pdrt_cnn_create(self.batch_max, _stream())
        self.n_params = _lib.pdrt_cnn_param_count()
        self.set_params(params if params is not None else init_params(seed))

    def close(self):
        if getattr(self, "_h", None):
            _lib.pdrt_cnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        v = flatten_params(p) if isinstance(p, dict) else np.asarray(p, np.float64)
        t = torch.tensor(v, dtype=torch.float32, device=self.device)
        assert t.numel() == self.n_params
        _lib.pdrt_cnn_set_params(self._h, t.data_ptr(), _stream())
        torch.cuda.current_stream().synchronize()

    def get_params(self) -> np.ndarray:
        t = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        _lib.pdrt_cnn_get_params(self._h, t.data_ptr(), _stream())
        return t.cpu().numpy()

    @staticmethod
    def _x(x):
        if x.dtype != torch.bfloat16 or not x.is_contiguous():
            x = x.to(torch.bfloat16).contiguous()
        assert x.shape[1:] == (SIDE, SIDE, 3)
        return x

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        """x: [n][64][64][3] (BF16 or convertible) on the device -> [n][121] FP32."""
        x = self._x(x)
        n = x.shape[0]
        y = torch.empty((n, N_OUT), dtype=torch.float32, device=self.device)
        for i in range(0, n, self.batch_max):
            j = min(n, i + self.batch_max)
            _lib.pdrt_cnn_forward(self._h, x[i:j].data_ptr(), j - i, y[i:j].data_ptr(), _stream())
        return y

    def backward(self, dy: torch.Tensor) -> torch.Tensor:
        """Parameter gradient of the last forward (n <= batch_max) for dy [n][121]."""
        dy = dy.to(torch.float32).contiguous()
        g = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        _lib.pdrt_cnn_backward(self._h, dy.shape[0], dy.data_ptr(), g.data_ptr(), _stream())
        return g

    def train_step(self, x: torch.Tensor, target: torch.Tensor, lr: float, loss_out=None):
        x = self._x(x)
        target = target.to(torch.float32).contiguous()
        ptr = loss_out.data_ptr() if loss_out is not None else None
        _lib.pdrt_cnn_train_step(self._h, x.data_ptr(), target.data_ptr(), x.shape[0], lr, ptr,
                                 _stream())

    def activation(self, layer: int, n: int) -> torch.Tensor:
        """Copy of activation h_layer (0..4, BF16 NHWC) of the last forward of n samples."""
        side = SIDE >> layer
        ch = 3 if layer == 0 else 64
        out = torch.empty((n, side, side, ch), dtype=torch.bfloat16, device=self.device)
        _lib.pdrt_cnn_read_activation(self._h, layer, n, out.data_ptr(), _stream())
        return out

    def status(self) -> int:
        return _lib.pdrt_cnn_status(self._h, _stream())


# ---------------------------------------------------------------------------
# beam's-eye-view inputs
# ---------------------------------------------------------------------------
def mask_bits(phantom) -> np.ndarray:
    """uint8 [nz][ny][nx]: bit s set where the voxel is in STRUCTURES[s]."""
    bits = np.zeros(phantom.shape, np.uint8)
    for s, name in enumerate(STRUCTURES):
        if name in phantom.masks:
            bits |= (np.asarray(phantom.masks[name], bool).astype(np.uint8) << s)
    return bits


def bev_inputs(phantom, gantry_deg, iso, sid=1000.0, pitch=BEV_PITCH_MM, device=None) -> torch.Tensor:
    """Network inputs of every control point: BF16 [n_cp][64][64][3]."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    bits = torch.tensor(mask_bits(phantom), device=dev)
    nz, ny, nx = phantom.shape
    reach = 0.5 * math.sqrt((nx * phantom.spacing[0]) ** 2 + (ny * phantom.spacing[1]) ** 2)
    step = 0.5 * min(phantom.spacing)
    out = torch.empty((len(gantry_deg), SIDE, SIDE, 3), dtype=torch.bfloat16, device=dev)
    _lib.pdrt_bev_project(bits.data_ptr(), nx, ny, nz, phantom.spacing, phantom.origin, iso, sid,
                          list(gantry_deg), SIDE, pitch, reach, step, out.data_ptr(), _stream())
    return out


# ---------------------------------------------------------------------------
# plan <-> network units
# ---------------------------------------------------------------------------
def encode_plan(leaves, mu) -> np.ndarray:
    """[n_cp][121]: leaves (left, right per pair) / 50 mm, then MU / 2."""
    n = leaves.shape[0]
    out = np.empty((n, N_OUT))
    out[:, :120] = leaves.reshape(n, 120) / LEAF_SCALE_MM
    out[:, 120] = mu / MU_SCALE
    return out


def decode_plan(y, machine) -> tuple:
    """Network output [n_cp][121] -> (leaves, mu) in machine units; left and
    right are ordered, MU kept at or above the machine's minimum."""
    y = np.asarray(y, np.float64)
    n = y.shape[0]
    lv = y[:, :120].reshape(n, 60, 2) * LEAF_SCALE_MM
    lv = np.stack([lv.min(-1), lv.max(-1)], -1)
    mu = np.maximum(y[:, 120] * MU_SCALE, machine.eps_mu)
    return lv, mu


# ---------------------------------------------------------------------------
# plans from the engine's optimiser, training, evaluation
# ---------------------------------------------------------------------------
N_ITER = 100                 # the paper's iteration count for gradient optimisation
OPT_LR, OPT_LR_MU = 0.5, 0.05


@dataclass
class Case:
    work: object
    engine: DoseEngine
    masks: dict
    presc: float
    open_init: tuple


def make_case(seed: int) -> Case:
    """Phantom, engine and open-field start; the prescription is the mean PTV
    dose of the open-field start (sets the dose scale of the objective)."""
    w = S.warmstart_case(seed)
    eng = DoseEngine(w.phantom, w.machine, w.plan.gantry_deg, w.plan.iso)
    masks = {k: w.phantom.masks[k] for k in STRUCTURES}
    init = open_field_start(w.plan, w.machine)
    D0 = eng.forward(*init)
    presc = float(D0[torch.as_tensor(masks["ptv"], device=eng.device)].mean())
    return Case(w, eng, masks, presc, init)


def objective_of(case: Case, leaves, jaws, mu) -> float:
    """The exact engine's objective value of a parameter set (one forward)."""
    D = case.engine.forward(leaves, jaws, mu)
    m = {k: torch.as_tensor(v, device=case.engine.device) for k, v in case.masks.items()}
    return float(objective_quadratic(D, m, case.presc))


def plain_optimise(case: Case, n_iter=N_ITER, target=None):
    return optimise(case.engine, case.masks, case.presc, case.open_init, n_iter=n_iter, lr=OPT_LR,
                    lr_mu=OPT_LR_MU, objective="quadratic", target=target)


def generate(seeds, n_iter=N_ITER, log=None):
    """Training pairs from the plain optimiser: inputs BF16 [N][64][64][3] and
    targets FP32 [N][121] on the device, one row per control point."""
    xs, ts = [], []
    t0 = time.time()
    for i, sd in enumerate(seeds):
        c = make_case(int(sd))
        res = plain_optimise(c, n_iter)
        from .optimize import project_plan
        lv, _, mu = project_plan(res.leaves, res.jaws, res.mu, c.work.machine)
        xs.append(bev_inputs(c.work.phantom, c.work.plan.gantry_deg, c.work.plan.iso))
        ts.append(torch.tensor(encode_plan(lv, mu), dtype=torch.float32, device=xs[-1].device))
        c.engine.close()
        if log and (i + 1) % 100 == 0:
            log(f"generated {i + 1}/{len(seeds)} plans in {time.time() - t0:.1f} s")
    return torch.cat(xs), torch.cat(ts)


def train(net: WarmStartNet, X, T, epochs=30, batch=256, lr=1e-3, seed=0, log=None):
    """Mini-batch Adam on the MSE (pdrt_cnn_train_step); lr decays by cosine."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = X.shape[0]
    steps = epochs * max(1, n // batch)
    loss = torch.zeros(1, device=X.device)
    hist = []
    k = 0
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(X.device)
        acc, cnt = 0.0, 0
        for i in range(0, n - batch + 1, batch):
            idx = perm[i:i + batch]
            rate = 0.5 * lr * (1.0 + math.cos(math.pi * k / steps))
            net.train_step(X[idx], T[idx], rate, loss)
            k += 1
            if i % (16 * batch) == 0:
                acc += float(loss)
                cnt += 1
        hist.append(acc / max(cnt, 1))
        if log:
            log(f"epoch {ep + 1}/{epochs}: loss {hist[-1]:.5f}")
    return hist


def propose(net: WarmStartNet, case: Case):
    """The network's (leaves, jaws, MU) for a case; jaws are the plan's."""
    x = bev_inputs(case.work.phantom, case.work.plan.gantry_deg, case.work.plan.iso)
    y = net.forward(x).cpu().numpy()
    lv, mu = decode_plan(y, case.work.machine)
    return lv, case.open_init[1].copy(), mu


def best_mu_scale(case: Case, D: torch.Tensor, lo=0.25, hi=4.0):
    """(alpha, J(alpha D)): the global MU factor that minimises the objective
    of a dose D.  The dose is linear in the MU (Eq. D_total), so alpha D is
    the dose of the plan with every MU scaled by alpha and no further dose
    evaluation is needed; J is convex in alpha (a sum of squares of affine and
    rectified affine functions): a grid then golden-section search."""
    dev = D.device
    sel = {k: D[torch.as_tensor(v, device=dev)] for k, v in case.masks.items()}

    def J(a):
        return float(objective_quadratic_sel(sel, a, case.presc))

    grid = np.geomspace(lo, hi, 61)
    vals = [J(a) for a in grid]
    k = int(np.argmin(vals))
    a0, a1 = grid[max(k - 1, 0)], grid[min(k + 1, len(grid) - 1)]
    g = (math.sqrt(5.0) - 1.0) / 2.0
    x1, x2 = a1 - g * (a1 - a0), a0 + g * (a1 - a0)
    f1, f2 = J(x1), J(x2)
    for _ in range(40):
        if f1 <= f2:
            a1, x2, f2 = x2, x1, f1
            x1 = a1 - g * (a1 - a0)
            f1 = J(x1)
        else:
            a0, x1, f1 = x1, x2, f2
            x2 = a0 + g * (a1 - a0)
            f2 = J(x2)
    a = 0.5 * (a0 + a1)
    return a, J(a)


def objective_quadratic_sel(sel: dict, alpha: float, presc: float, weights=None, oar_fraction=0.5):
    """objective_quadratic of the dose alpha D, given the voxels of D inside
    each structure (sel[name] = D[mask])."""
    weights = weights or {"ptv": 100.0, "bladder": 1.0, "rectum": 10.0}
    L = weights["ptv"] * ((alpha * sel["ptv"] - presc) ** 2).mean()
    for name, lam in weights.items():
        if name == "ptv" or name not in sel or lam == 0.0 or sel[name].numel() == 0:
            continue
        ex = torch.clamp(alpha * sel[name] - oar_fraction * presc, min=0.0)
        L = L + lam * (ex ** 2).mean()
    return L


def assess(case: Case, prop):
    """The exact engine's assessment of a proposal (one dose evaluation): the
    proposal with its MU rescaled by best_mu_scale, and its objective."""
    D = case.engine.forward(*prop)
    alpha, j = best_mu_scale(case, D)
    return (prop[0], prop[1], prop[2] * alpha), j, alpha


def evaluate(net: WarmStartNet, seeds, n_iter=N_ITER):
    """Warm versus plain on held-out phantoms, with a control that isolates
    what the network adds.  Three arms per phantom:
      plain    the plain optimiser, n_iter evaluations from the open-field
               start; its best objective J* is the target and plain_evals
               the evaluations it took to reach it;
      control  the open-field start through the same one-evaluation MU
               assessment as the proposal (assess: best global MU scale),
               then the optimiser until J <= J*;
      warm     the network's proposal through the assessment; the engine
               keeps the better of it and the assessed open-field start (so
               the warm arm pays two assessments), then optimises until
               J <= J* (at most n_iter more evaluations).
    warm / plain is the spec comparison; warm / control is the
    network's own gain (same line search, other start)."""
    rows = []
    for sd in seeds:
        c = make_case(int(sd))
        plain = plain_optimise(c, n_iter)
        j_star = min(plain.history)
        plain_evals = int(np.argmin(plain.history)) + 1
        j_open = plain.history[0]
        open_s, j_open_s, alpha_open = assess(c, c.open_init)
        ctrl = optimise(c.engine, c.masks, c.presc, open_s, n_iter=n_iter, lr=OPT_LR, lr_mu=OPT_LR_MU,
                        objective="quadratic", target=j_star)
        prop, j_prop, alpha = assess(c, propose(net, c))
        fallback = j_prop > j_open_s
        start = open_s if fallback else prop
        warm = optimise(c.engine, c.masks, c.presc, start, n_iter=n_iter, lr=OPT_LR, lr_mu=OPT_LR_MU,
                        objective="quadratic", target=j_star)
        D_p = c.engine.forward(plain.leaves, plain.jaws, plain.mu)
        D_w = c.engine.forward(warm.leaves, warm.jaws, warm.mu)
        rows.append({
            "seed": int(sd), "j_open": j_open, "j_open_scaled": j_open_s, "j_proposal": j_prop,
            "j_star": j_star, "mu_scale": float(alpha), "mu_scale_open": float(alpha_open),
            "fallback": bool(fallback), "plain_evals": plain_evals,
            "control_evals": 1 + ctrl.dose_evals, "control_reached": bool(min(ctrl.history) <= j_star),
            "warm_evals": 2 + warm.dose_evals, "reached": bool(min(warm.history) <= j_star),
            "dose_diff_rel": float((D_w - D_p).abs().max() / D_p.max()),
        })
        c.engine.close()
    return rows


def summarise(rows) -> dict:
    r = np.array([x["warm_evals"] / x["plain_evals"] for x in rows])
    rc = np.array([x["warm_evals"] / x["control_evals"] for x in rows])
    cp = np.array([x["control_evals"] / x["plain_evals"] for x in rows])
    return {"cases": len(rows), "median_eval_ratio": float(np.median(r)),
            "mean_eval_ratio": float(np.mean(r)),
            "frac_at_most_half": float(np.mean(r <= 0.5)),
            "median_warm_over_control": float(np.median(rc)),
            "mean_warm_over_control": float(np.mean(rc)),
            "median_control_over_plain": float(np.median(cp)),
            "reached": int(sum(x["reached"] for x in rows)),
            "control_reached": int(sum(x["control_reached"] for x in rows)),
            "fallbacks": int(sum(x["fallback"] for x in rows)),
            "median_plain_evals": float(np.median([x["plain_evals"] for x in rows])),
            "median_control_evals": float(np.median([x["control_evals"] for x in rows])),
            "median_warm_evals": float(np.median([x["warm_evals"] for x in rows])),
            "median_proposal_over_open": float(np.median([x["j_proposal"] / x["j_open"] for x in rows])),
            "median_proposal_over_scaled_open": float(np.median([x["j_proposal"] / x["j_open_scaled"]
                                                                 for x in rows])),
            "median_dose_diff_rel": float(np.median([x["dose_diff_rel"] for x in rows]))}


WEIGHTS_FILE = "warmstart_weights.npz"


def default_weights_path() -> str:
    import os
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", WEIGHTS_FILE)


def load_net(path=None, batch_max=256) -> WarmStartNet:
    d = np.load(path or default_weights_path())
    return WarmStartNet(batch_max=batch_max, params=d["params"].astype(np.float64))


def main(argv=None):
    """Generate plans with the engine's optimiser, train the network on the
    GPU, evaluate warm versus plain on held-out phantoms, save the weights."""
    import argparse
    import json
    import os
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=100)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--iters", type=int, default=N_ITER)
    ap.add_argument("--out", default=os.path.dirname(default_weights_path()))
    ap.add_argument("--seed", type=int, default=5000)
    ap.add_argument("--eval-only", default=None,
                    help="evaluate the weights in this .npz on its held-out seeds (no training)")
    a = ap.parse_args(argv)
    os.makedirs(a.out, exist_ok=True)
    log = lambda s: print(s, flush=True)   # noqa: E731
    if a.eval_only:
        d = np.load(a.eval_only)
        net = load_net(a.eval_only)
        rows = evaluate(net, d["test_seeds"][:a.test], a.iters)
        summ = summarise(rows)
        with open(os.path.join(a.out, "warmstart_eval.json"), "w") as f:
            json.dump({"summary": summ, "cases": rows}, f, indent=1)
        log(json.dumps(summ))
        net.close()
        return
    t0 = time.time()
    train_seeds = a.seed + np.arange(a.train)
    test_seeds = a.seed + 100000 + np.arange(a.test)
    X, T = generate(train_seeds, a.iters, log)
    t_gen = time.time() - t0
    net = WarmStartNet(batch_max=a.batch, seed=a.seed)
    t1 = time.time()
    hist = train(net, X, T, a.epochs, a.batch, a.lr, a.seed, log)
    torch.cuda.synchronize()
    t_train = time.time() - t1
    if net.status() != 0:
        raise RuntimeError("a tensor-core wait expired during training")
    params = net.get_params()
    np.savez(os.path.join(a.out, WEIGHTS_FILE), params=params.astype(np.float32),
             loss=np.array(hist), train_seeds=train_seeds, test_seeds=test_seeds)
    rows = evaluate(net, test_seeds, a.iters)
    summ = summarise(rows)
    summ.update({"train_plans": int(a.train), "samples": int(X.shape[0]), "epochs": a.epochs,
                 "final_loss": hist[-1], "generate_s": t_gen, "train_s": t_train})
    with open(os.path.join(a.out, "warmstart_eval.json"), "w") as f:
        json.dump({"summary": summ, "cases": rows}, f, indent=1)
    log(json.dumps(summ))
    net.close()


if __name__ == "__main__":
    main()
