"""Pins of the oracle's adjoint and cross-checks with the PyTorch restatement.

* dot-product tests <A x, y> = <x, A^T y> per linear stage (1e-12),
* central finite differences of the FP64 forward (step 0.01 mm / 0.01 MU)
  against the analytic gradient, away from pixel-boundary kinks and clamps
  (the overlap of Sec. 2.2.2 is piecewise linear, so the FD is exact there),
* exact projection Jacobian (ste = 0) through active clamps (Sec. 2.2.1),
* the independent torch FP64 restatement: forward and autograd gradients.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle import torch_ref
from paper_2512_18863_gb300 import synth as S


def _small(seed=7, n=(12, 20, 20), spacing=4.0, n_cp=3, r_px=3, ste=1):
    w = S.small_pelvis(seed=seed, n=n, spacing=spacing, n_cp=n_cp, r_px=r_px,
                       ptv_radii=(14.0, 12.0, 14.0))
    w.machine.ste = ste
    return w


def _rel(a, b):
    return abs(a - b) / max(abs(a), abs(b), 1e-300)


def test_dot_product_gather():
    w = _small()
    mod = O.Model(w.phantom, w.machine, w.plan)
    rng = np.random.default_rng(1)
    for b in range(w.plan.n_cp):
        x = rng.standard_normal(mod.vol_shape())
        y = rng.standard_normal(w.phantom.shape)
        assert _rel(np.vdot(mod.gather(b, x), y), np.vdot(x, mod.gather_T(b, y))) < 1e-12


def test_dot_product_conv():
    w = _small()
    mod = O.Model(w.phantom, w.machine, w.plan)
    rng = np.random.default_rng(2)
    z = mod.wepl(1)
    x = rng.standard_normal(mod.vol_shape())
    y = rng.standard_normal(mod.vol_shape())
    assert _rel(np.vdot(mod.conv(z, x), y), np.vdot(x, mod.conv_T(z, y))) < 1e-12


def test_dot_product_magnify():
    w = _small()
    mod = O.Model(w.phantom, w.machine, w.plan)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((mod.lat.nv, mod.lat.nu))
    y = rng.standard_normal(mod.vol_shape())
    assert _rel(np.vdot(mod.magnify(x), y), np.vdot(x, mod.magnify_T(y))) < 1e-12


def _far_from_kinks(x, d, off):
    """True if edge x is > 0.06 mm from every pixel boundary (off + (k+1/2) d)."""
    t = (x - off) / d - 0.5
    return min(t - np.floor(t), np.ceil(t) - t) * d > 0.06


def _pick_params(w, mod, rng, count):
    """Random differentiable parameters: open leaf edges inside the jaws,
    jaw edges, MUs; all away from kinks and clamps."""
    lat = mod.lattice
    picks = []
    pl = w.plan
    for b in range(pl.n_cp):
        jx0, jx1, jy0, jy1 = pl.jaws[b]
        lb = w.machine.leaf_bounds
        for i in range(w.machine.n_pairs):
            l, r = pl.leaves[b, i]
            if r - l < 2.0 or lb[i + 1] <= jy0 or lb[i] >= jy1:
                continue
            for s, x in ((0, l), (1, r)):
                if jx0 + 0.5 < x < jx1 - 0.5 and _far_from_kinks(x, lat["du"], 0.0):
                    picks.append(("leaves", (b, i, s)))
        for s in range(4):
            d, off = (lat["du"], 0.0) if s < 2 else (lat["dv"], -lat["cv"] * lat["dv"] + round(lat["cv"]) * lat["dv"])
            if _far_from_kinks(pl.jaws[b, s], d, off):
                picks.append(("jaws", (b, s)))
        picks.append(("mu", (b,)))
    idx = rng.choice(len(picks), size=min(count, len(picks)), replace=False)
    return [picks[i] for i in idx]


@pytest.mark.parametrize("ste", [1, 0])
def test_gradient_vs_central_fd(ste):
    """T9: central FD of L = <g, D> on the FP64 forward vs orc_dose_grad."""
    w = _small(ste=ste)
    mod = O.Model(w.phantom, w.machine, w.plan)
    rng = np.random.default_rng(11)
    g = rng.standard_normal(w.phantom.shape)
    dl, dj, dm = mod.dose_grad(g)
    grads = {"leaves": dl, "jaws": dj, "mu": dm}
    picks = _pick_params(w, mod, rng, 40)
    assert len(picks) >= 20
    base = {"leaves": w.plan.leaves.copy(), "jaws": w.plan.jaws.copy(), "mu": w.plan.mu.copy()}
    scale = {k: np.abs(v).max() for k, v in grads.items()}
    for name, ix in picks:
        h = 0.01
        vals = []
        for sgn in (+1, -1):
            p = {k: v.copy() for k, v in base.items()}
            p[name][ix] += sgn * h
            vals.append(np.vdot(g, mod.dose(p["leaves"], p["jaws"], p["mu"])))
        fd = (vals[0] - vals[1]) / (2 * h)
        an = grads[name][ix]
        assert abs(fd - an) <= 1e-6 * scale[name] + 1e-9 * abs(an), (name, ix, fd, an)


def test_projection_jacobian_through_clamps():
    """Sec. 2.2.1 with ste = 0: the gradient of a raw parameter passes through
    the projection's exact Jacobian.  A leaf pair narrower than w_min moves as
    a rigid gap (each raw edge moves both projected edges by 1/2); an aperture
    centre beyond the travel range F has zero gradient in the centre
    direction.  FD through the clamp is exact (piecewise linear)."""
    w = _small(ste=0, n_cp=1)
    m = w.machine
    m.wmin_leaf = 3.0
    mod = O.Model(w.phantom, m, w.plan)
    lat = mod.lattice
    pl = w.plan
    jy0, jy1 = pl.jaws[0, 2], pl.jaws[0, 3]
    lb = m.leaf_bounds
    rows = [i for i in range(m.n_pairs) if lb[i] >= jy0 and lb[i + 1] <= jy1]
    i = rows[len(rows) // 2]
    pl.leaves[0, i] = (1.13, 2.37)                       # width 1.24 < w_min = 3
    rng = np.random.default_rng(4)
    g = rng.standard_normal(w.phantom.shape)
    dl, _, _ = mod.dose_grad(g)
    for s in (0, 1):
        vals = []
        for sgn in (+1, -1):
            lv = pl.leaves.copy()
            lv[0, i, s] += sgn * 0.01
            vals.append(np.vdot(g, mod.dose(lv, pl.jaws, pl.mu)))
        fd = (vals[0] - vals[1]) / 0.02
        assert abs(fd - dl[0, i, s]) <= 1e-7 * np.abs(dl).max(), (s, fd, dl[0, i, s])
    assert abs(dl[0, i, 0] - dl[0, i, 1]) <= 1e-12 * np.abs(dl).max()
    del lat


def test_fluence_vjp_vs_fd_on_fluence():
    """VJP of the fluence layer alone (Sec. 2.2.1-2.2.2) against FD of F."""
    w = _small(ste=0, n_cp=2)
    mod = O.Model(w.phantom, w.machine, w.plan)
    rng = np.random.default_rng(8)
    dF = rng.standard_normal((mod.lat.nv, mod.lat.nu))
    pl = w.plan

    def F_of(lv_raw, jw_raw):
        lv_p, jw_p, _ = mod.project(0, lv_raw[None], jw_raw[None], np.ones(1))
        return mod.fluence(lv_p, jw_p)

    dl, dj = mod.fluence_vjp(0, dF)
    for s in range(4):
        vals = []
        for sgn in (+1, -1):
            jw = pl.jaws[0].copy()
            jw[s] += sgn * 0.01
            vals.append(np.vdot(dF, F_of(pl.leaves[0], jw)))
        assert (vals[0] - vals[1]) / 0.02 == pytest.approx(dj[s], rel=1e-7, abs=1e-9)


def _torch_model(w):
    return torch_ref.TorchDose(w.phantom, w.machine, w.plan.gantry_deg, w.plan.iso)


@pytest.mark.parametrize("ste", [1, 0])
def test_torch_restatement_forward_and_autograd(ste):
    """The independent torch FP64 transcription agrees with the C oracle on
    the dose (1e-12 of max) and its autograd gradients agree with the C
    analytic adjoint (1e-9 relative, away from kinks)."""
    w = _small(ste=ste)
    mod = O.Model(w.phantom, w.machine, w.plan)
    D = mod.dose()
    tm = _torch_model(w)
    leaves = torch.tensor(w.plan.leaves, dtype=torch.float64, requires_grad=True)
    jaws = torch.tensor(w.plan.jaws, dtype=torch.float64, requires_grad=True)
    mu = torch.tensor(w.plan.mu, dtype=torch.float64, requires_grad=True)
    Dt = tm.dose(leaves, jaws, mu)
    np.testing.assert_allclose(Dt.detach().numpy(), D, rtol=0, atol=1e-12 * D.max())
    rng = np.random.default_rng(12)
    g = rng.standard_normal(w.phantom.shape)
    (Dt * torch.from_numpy(g)).sum().backward()
    dl, dj, dm = mod.dose_grad(g)
    for a, b in ((leaves.grad.numpy(), dl), (jaws.grad.numpy(), dj), (mu.grad.numpy(), dm)):
        assert np.abs(a - b).max() <= 1e-9 * np.abs(b).max()
