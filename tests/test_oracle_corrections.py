"""Pins of the fluence corrections of Sec. 2.2.2 beyond transmission (source
penumbra, off-axis profile, collimator rotation) in the oracle, and of their
adjoint."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle import torch_ref
from paper_2512_18863_gb300 import synth as S


def _model(pen_u=4.0, pen_v=6.0, oap=(1.0, 0.0, 0.0), n=(41, 9, 41), ste=1, coll=0.0, sz=2.5):
    nz, ny, nx = n
    ph = S.Phantom(hu=np.zeros(n, np.float32), spacing=(2.0, 2.0, sz),
                   origin=(-(nx // 2) * 2.0, -(ny // 2) * 2.0, -(nz // 2) * sz))
    m = S.machine_model(61, r_px=3)
    m.pen_fwhm_u, m.pen_fwhm_v, m.off_axis, m.ste = pen_u, pen_v, oap, ste
    m.collimator_deg = coll
    return O.Model(ph, m, S.static_field(m)), m


def test_penumbra_of_a_single_pixel_is_the_normalised_gaussian():
    """A one-pixel fluence blurred along u then v is the outer product of two
    discrete Gaussians exp(-(t pitch)^2 / (2 sigma^2)), sigma = FWHM / 2.3548,
    each of unit sum (the blur keeps the total fluence)."""
    mod, m = _model(pen_u=5.0, pen_v=7.5)
    L = mod.lattice
    F = np.zeros((L["nv"], L["nu"]))
    a0, c0 = int(L["cu"]), int(round(L["cv"]))
    F[c0, a0] = 1.0
    G = mod.fluence_correct(F)
    assert G.sum() == pytest.approx(1.0, rel=1e-13)
    su, sv = 5.0 / (2 * math.sqrt(2 * math.log(2))), 7.5 / (2 * math.sqrt(2 * math.log(2)))
    for t in range(-4, 5):
        assert G[c0, a0 + t] / G[c0, a0] == pytest.approx(math.exp(-(t * 2.0) ** 2 / (2 * su * su)), rel=1e-12)
        assert G[c0 + t, a0] / G[c0, a0] == pytest.approx(math.exp(-(t * 2.5) ** 2 / (2 * sv * sv)), rel=1e-12)
    assert G[c0 + 2, a0 + 3] == pytest.approx(G[c0 + 2, a0] * G[c0, a0 + 3] / G[c0, a0], rel=1e-12)
    ru = math.ceil(3 * su / 2.0)
    assert G[c0, a0 + ru] > 0 and G[c0, a0 + ru + 1] == 0.0


def test_off_axis_profile_multiplies_by_c0_c1r_c2r2():
    oap = (0.98, 2.5e-4, -1.5e-6)
    mod, _ = _model(pen_u=0.0, pen_v=0.0, oap=oap)
    L = mod.lattice
    F = np.ones((L["nv"], L["nu"]))
    G = mod.fluence_correct(F)
    u = (np.arange(L["nu"]) - L["cu"]) * L["du"]
    v = (np.arange(L["nv"]) - L["cv"]) * L["dv"]
    r = np.sqrt(u[None, :] ** 2 + v[:, None] ** 2)
    np.testing.assert_allclose(G, oap[0] + oap[1] * r + oap[2] * r * r, rtol=1e-14)


def test_corrections_dot_product():
    mod, _ = _model(oap=(1.0, 2e-4, 1e-6))
    L = mod.lattice
    rng = np.random.default_rng(3)
    x = rng.standard_normal((L["nv"], L["nu"]))
    y = rng.standard_normal((L["nv"], L["nu"]))
    a, b = np.vdot(mod.fluence_correct(x), y), np.vdot(x, mod.fluence_correct_T(y))
    assert abs(a - b) <= 1e-12 * abs(a)


def test_collimator_rotation_zero_is_identity():
    mod, _ = _model(pen_u=0.0, pen_v=0.0, coll=0.0, sz=2.0)
    F = np.random.default_rng(5).random((mod.lattice["nv"], mod.lattice["nu"]))
    np.testing.assert_array_equal(mod.rotate(F), F)


@pytest.mark.parametrize("coll", [90.0, 180.0, -90.0])
def test_collimator_quarter_turns_permute_pixels(coll):
    """With square pixels and the isocentre on a pixel centre, quarter turns
    move pixels onto pixels: a feature at (u, v) lands at R(coll) (u, v); for
    +90 deg an opening on the +u side appears on the +v side."""
    mod, _ = _model(pen_u=0.0, pen_v=0.0, coll=coll, sz=2.0)
    L = mod.lattice
    assert L["du"] == L["dv"] and float(L["cu"]).is_integer() and float(L["cv"]).is_integer()
    nu, nv, cu, cv = L["nu"], L["nv"], int(L["cu"]), int(L["cv"])
    F = np.zeros((nv, nu))
    rng = np.random.default_rng(7)
    F[cv - 6:cv + 7, cu - 6:cu + 7] = rng.random((13, 13))   # asymmetric, well inside
    G = mod.rotate(F)
    q = int(round(coll / 90.0)) % 4
    for c in range(cv - 8, cv + 9):
        for a in range(cu - 8, cu + 9):
            du_, dv_ = a - cu, c - cv
            # source pixel R(-coll) (du_, dv_)
            src = {0: (du_, dv_), 1: (dv_, -du_), 2: (-du_, -dv_), 3: (-dv_, du_)}[q]
            assert G[c, a] == pytest.approx(F[cv + src[1], cu + src[0]], abs=1e-12)
    if q == 1:
        P = np.zeros((nv, nu)); P[cv, cu + 5] = 1.0
        assert mod.rotate(P)[cv + 5, cu] == pytest.approx(1.0, abs=1e-12)


def test_collimator_rotation_of_a_radial_map_within_interpolation_bound():
    """A map that depends on r only is unchanged by a turn up to the bilinear
    interpolation error, |err| <= (h^2 / 8) (|f_aa| + |f_cc|) with h = 1 pixel."""
    mod, _ = _model(pen_u=0.0, pen_v=0.0, coll=37.0, sz=2.0)
    L = mod.lattice
    a = np.arange(L["nu"]) - L["cu"]
    c = np.arange(L["nv"]) - L["cv"]
    s = 6.0   # pixels
    F = np.exp(-(a[None, :] ** 2 + c[:, None] ** 2) / (2 * s * s))
    G = mod.rotate(F)
    bound = 2.0 / 8.0 / (s * s)          # |f''| <= 1/s^2 per axis for a unit Gaussian
    inner = (np.abs(a[None, :]) < L["cu"] - 3) & (np.abs(c[:, None]) < L["cv"] - 3)
    assert np.abs(G - F)[inner].max() <= bound
    assert np.abs(G - F)[inner].max() > 0.0


@pytest.mark.parametrize("coll", [23.0, -61.0, 145.0])
def test_collimator_rotation_is_bilinear_resampling(coll):
    """A feature at s appears at R(coll) s, so pixel x reads the corrected map
    at R(coll)^-1 x, in mm (pixels 2 x 2.5 mm here), bilinearly, zero
    outside the lattice; scipy.ndimage.map_coordinates (order 1, zero
    outside) resamples the same points independently."""
    from scipy.ndimage import map_coordinates
    mod, _ = _model(pen_u=0.0, pen_v=0.0, coll=coll, sz=2.5)
    L = mod.lattice
    assert L["du"] != L["dv"]
    F = np.random.default_rng(9).random((L["nv"], L["nu"]))
    G = mod.rotate(F)
    t = math.radians(coll)
    Rinv = np.linalg.inv(np.array([[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]]))
    c, a = np.meshgrid(np.arange(L["nv"]), np.arange(L["nu"]), indexing="ij")
    uv = np.stack([(a - L["cu"]) * L["du"], (c - L["cv"]) * L["dv"]]).reshape(2, -1)
    us, vs = Rinv @ uv
    coords = np.stack([vs / L["dv"] + L["cv"], us / L["du"] + L["cu"]])
    exp = map_coordinates(F, coords, order=1, mode="grid-constant", cval=0.0).reshape(F.shape)
    np.testing.assert_allclose(G, exp, rtol=1e-12, atol=1e-14)


def test_collimator_rotation_dot_product():
    mod, _ = _model(coll=23.0)
    L = mod.lattice
    rng = np.random.default_rng(11)
    x = rng.standard_normal((L["nv"], L["nu"]))
    y = rng.standard_normal((L["nv"], L["nu"]))
    a, b = np.vdot(mod.rotate(x), y), np.vdot(x, mod.rotate_T(y))
    assert abs(a - b) <= 1e-12 * abs(a)
    a, b = np.vdot(mod.fluence_correct(x), y), np.vdot(x, mod.fluence_correct_T(y))
    assert abs(a - b) <= 1e-12 * abs(a)


def _corrected_case(ste, coll=0.0):
    w = S.small_pelvis(seed=63, n=(12, 20, 20), spacing=4.0, n_cp=3, r_px=3,
                       ptv_radii=(14.0, 12.0, 14.0))
    S.with_corrections(w.machine, 5, collimator_deg=coll)
    w.machine.ste = ste
    return w


@pytest.mark.parametrize("ste,coll", [(1, 0.0), (0, 0.0), (1, 17.0)])
def test_gradient_with_corrections_vs_central_fd(ste, coll):
    from tests.test_oracle_adjoint import _pick_params
    w = _corrected_case(ste, coll)
    mod = O.Model(w.phantom, w.machine, w.plan)
    rng = np.random.default_rng(17)
    g = rng.standard_normal(w.phantom.shape)
    dl, dj, dm = mod.dose_grad(g)
    grads = {"leaves": dl, "jaws": dj, "mu": dm}
    scale = {k: np.abs(v).max() for k, v in grads.items()}
    base = {"leaves": w.plan.leaves.copy(), "jaws": w.plan.jaws.copy(), "mu": w.plan.mu.copy()}
    picks = _pick_params(w, mod, rng, 30)
    assert len(picks) >= 15
    for name, ix in picks:
        vals = []
        for sgn in (+1, -1):
            p = {k: v.copy() for k, v in base.items()}
            p[name][ix] += sgn * 0.01
            vals.append(np.vdot(g, mod.dose(p["leaves"], p["jaws"], p["mu"])))
        fd = (vals[0] - vals[1]) / 0.02
        assert abs(fd - grads[name][ix]) <= 1e-6 * scale[name] + 1e-9 * abs(grads[name][ix])


@pytest.mark.parametrize("coll", [0.0, 17.0])
def test_torch_restatement_with_corrections(coll):
    w = _corrected_case(1, coll)
    mod = O.Model(w.phantom, w.machine, w.plan)
    D = mod.dose()
    tm = torch_ref.TorchDose(w.phantom, w.machine, w.plan.gantry_deg, w.plan.iso)
    leaves = torch.tensor(w.plan.leaves, dtype=torch.float64, requires_grad=True)
    jaws = torch.tensor(w.plan.jaws, dtype=torch.float64, requires_grad=True)
    mu = torch.tensor(w.plan.mu, dtype=torch.float64, requires_grad=True)
    Dt = tm.dose(leaves, jaws, mu)
    np.testing.assert_allclose(Dt.detach().numpy(), D, rtol=0, atol=1e-12 * D.max())
    g = np.random.default_rng(19).standard_normal(w.phantom.shape)
    (Dt * torch.from_numpy(g)).sum().backward()
    dl, dj, dm = mod.dose_grad(g)
    for a, b in ((leaves.grad.numpy(), dl), (jaws.grad.numpy(), dj), (mu.grad.numpy(), dm)):
        assert np.abs(a - b).max() <= 1e-9 * np.abs(b).max()
