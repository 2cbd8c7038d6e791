"""Pins of the warm-start network oracle (oracle/cnn_oracle.py) against
library routines and finite differences."""
import numpy as np
import pytest
import torch
from scipy.signal import correlate2d

from oracle import cnn_oracle as N


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-6, 6, 5000),
                        1.0 + np.arange(-64, 64) * 2.0 ** -9])          # exact ties included
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(N.bf16(x), ref)
    assert N.bf16(1.0 + 2.0 ** -8) == 1.0                # tie to even
    assert N.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6


def test_conv_is_strided_same_correlation():
    """z[b,y,x,o] = b_o + sum_c correlate2d(x[b,:,:,c], W[o,:,:,c], 'same')[2y, 2x]."""
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 12, 10, 3))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    z = N.conv_forward(x, W, b)
    assert z.shape == (2, 6, 5, 4)
    for bb in range(2):
        for o in range(4):
            ref = sum(correlate2d(x[bb, :, :, c], W[o, :, :, c], mode="same") for c in range(3))
            np.testing.assert_allclose(z[bb, :, :, o], ref[::2, ::2] + b[o], rtol=1e-12, atol=1e-12)


def test_first_layer_is_equivariant_to_two_pixel_shifts():
    p = N.init_params(3)
    rng = np.random.default_rng(2)
    x = (rng.random((1, 64, 64, 3)) < 0.3).astype(np.float64)
    xs = np.zeros_like(x)
    xs[:, 2:, 4:, :] = x[:, :-2, :-4, :]
    z = N.conv_forward(x, p["W1"], p["b1"])
    zs = N.conv_forward(xs, p["W1"], p["b1"])
    np.testing.assert_allclose(zs[:, 2:-1, 3:-1, :], z[:, 1:-2, 1:-3, :], rtol=1e-12, atol=1e-12)


def test_network_gradients_vs_central_differences():
    """Plain FP64 network (no rounding): every parameter class against central
    finite differences of L = sum(out * R)."""
    p = N.init_params(4)
    for l in range(1, 6):
        p[f"b{l}"] = np.random.default_rng(l).normal(0, 0.1, p[f"b{l}"].shape)
    rng = np.random.default_rng(5)
    x = (rng.random((2, 64, 64, 3)) < 0.4).astype(np.float64)
    R = rng.standard_normal((2, N.N_OUT))
    acts = N.forward(p, x, bf=False)
    g = N.backward(p, acts, R, bf=False)

    def L(q):
        a = N.forward(q, x, bf=False)
        pattern = np.concatenate([(a[f"z{l}"] > 0).ravel() for l in range(1, 5)])
        return float(np.sum(a["out"] * R)), pattern

    h = 1e-7
    checked = 0
    for name in ("W1", "b1", "W2", "b2", "W3", "W4", "b4", "W5", "b5"):
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, 4, replace=False):
            q = {k: v.copy() for k, v in p.items()}
            q[name].reshape(-1)[idx] += h
            lp, pp = L(q)
            q[name].reshape(-1)[idx] -= 2 * h
            lm, pm = L(q)
            if not np.array_equal(pp, pm):
                continue          # a ReLU kink lies inside [-h, h]: no derivative there
            checked += 1
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, idx, fd, an)
    assert checked >= 30


def test_bf16_network_stays_close_to_fp64_network():
    """The rounding points change outputs by BF16-sized relative amounts only."""
    p = N.init_params(6)
    x = (np.random.default_rng(7).random((2, 64, 64, 3)) < 0.4).astype(np.float64)
    a = N.forward(p, x, bf=True)["out"]
    b = N.forward(p, x, bf=False)["out"]
    assert np.abs(a - b).max() <= 0.05 * np.abs(b).max()
    assert np.abs(a - b).max() > 0


def test_mse_and_adam_match_torch():
    rng = np.random.default_rng(8)
    out, t = rng.standard_normal((3, 121)), rng.standard_normal((3, 121))
    L, d = N.mse_loss(out, t)
    to = torch.tensor(out, requires_grad=True)
    Lt = torch.nn.functional.mse_loss(to, torch.tensor(t))
    Lt.backward()
    assert L == pytest.approx(float(Lt.detach()), rel=1e-14)
    np.testing.assert_allclose(d, to.grad.numpy(), rtol=1e-14)
    p0 = rng.standard_normal(50)
    tp = torch.tensor(p0.copy(), requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-3)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for t_ in range(1, 4):
        g = rng.standard_normal(50)
        tp.grad = torch.tensor(g)
        opt.step()
        p, m, v = N.adam_step(p, g, m, v, t_, 1e-3)
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-15)


def _ball_bits(center, r, n=(40, 40, 40), sp=(4.0, 4.0, 4.0), bit=0):
    nz, ny, nx = n
    origin = (-(nx - 1) / 2 * sp[0], -(ny - 1) / 2 * sp[1], -(nz - 1) / 2 * sp[2])
    z, y, x = np.meshgrid(*[origin[d] + np.arange(n[2 - d]) * sp[d] for d in (2, 1, 0)], indexing="ij")
    inside = (x - center[0]) ** 2 + (y - center[1]) ** 2 + (z - center[2]) ** 2 <= r * r
    bits = np.zeros(n, np.uint8)
    bits[inside] = 1 << bit
    return bits, sp, origin


def test_bev_projection_of_a_ball_at_the_isocentre_is_a_disc():
    """A ball of radius r at the isocentre projects to a disc of radius
    r / sqrt(1 - (r/sid)^2) at the isocentre plane, up to one voxel of
    voxelisation, at every gantry angle."""
    r, sid = 40.0, 1000.0
    bits, sp, origin = _ball_bits((0.0, 0.0, 0.0), r)
    out = N.bev_project(bits, sp, origin, (0.0, 0.0, 0.0), sid, [0.0, 37.0, 90.0], 64, 2.5, 100.0, 1.0)
    pu = (np.arange(64) - 31.5) * 2.5
    rr = np.hypot(*np.meshgrid(pu, pu))
    R = r / np.sqrt(1 - (r / sid) ** 2)
    for b in range(3):
        m = out[b, :, :, 0]
        assert np.all(m[rr < R - 4.0] == 1) and np.all(m[rr > R + 4.0] == 0)
        assert np.all(out[b, :, :, 1:] == 0)


def test_bev_projection_axes_and_gantry_rotation():
    """e_u = (cos g, -sin g, 0), e_v = +z: a ball at +x lands at +u for gantry
    0; a ball at -y lands at +u for gantry 90; a ball at +z lands at +v."""
    pu = (np.arange(64) - 31.5) * 2.5
    for center, g, axis in (((40.0, 0.0, 0.0), 0.0, "u"), ((0.0, -40.0, 0.0), 90.0, "u"),
                            ((0.0, 0.0, 40.0), 0.0, "v")):
        bits, sp, origin = _ball_bits(center, 15.0, bit=2)
        m = N.bev_project(bits, sp, origin, (0.0, 0.0, 0.0), 1000.0, [g], 64, 2.5, 100.0, 1.0)[0, :, :, 2]
        assert m.sum() > 20
        py, px = np.nonzero(m)
        cu, cv = pu[px].mean(), pu[py].mean()
        if axis == "u":
            assert 30.0 < cu < 50.0 and abs(cv) < 3.0
        else:
            assert 30.0 < cv < 50.0 and abs(cu) < 3.0
