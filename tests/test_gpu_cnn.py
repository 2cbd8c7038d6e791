"""Warm-start network kernels (tcgen05 BF16 GEMMs, FP32 accumulation) and
the beam's-eye-view projection against the FP64 oracle (oracle/cnn_oracle.py).

Bars.  Layer by layer, with the GPU's own BF16 input activations fed to the
oracle, a stored activation may differ from the oracle's only where the FP32
and FP64 sums round to neighbouring BF16 values: |dh| <= 2^-7 |h| + 2^-20 and
at most 1 % of the elements differ at all.  The FP32 output of the dense head
and the parameter gradients (the oracle's backward run on the GPU's
activations) agree to 2e-3 of each tensor's largest entry.  End to end, from
the raw input, each output element stays within the bound propagated from one
BF16 step per stored activation.  The beam's-eye-view projection (bytes) is
bit-exact.
"""
import numpy as np
import pytest
import torch

from oracle import cnn_oracle as N
from paper_2512_18863_gb300 import warmstart as W

pytestmark = pytest.mark.gpu


def _f64(t):
    return t.float().cpu().numpy().astype(np.float64)


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    x = np.zeros((n, 64, 64, 3))
    for b in range(n):                     # blobs like projected structures
        for c in range(3):
            cy, cx = rng.uniform(10, 54, 2)
            ry, rx = rng.uniform(4, 16, 2)
            yy, xx = np.mgrid[0:64, 0:64]
            x[b, :, :, c] = (((yy - cy) / ry) ** 2 + ((xx - cx) / rx) ** 2 <= 1.0)
    return x


def _params(seed):
    p = W.init_params(seed)
    rng = np.random.default_rng(seed + 1)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.normal(0.0, 0.05, p[k].shape)
    return p


@pytest.fixture(scope="module")
def net_and_forward():
    n = 70                                   # not a multiple of the 128-row tiles
    p = _params(3)
    x = _inputs(n, 4)
    net = W.WarmStartNet(batch_max=96, params=p)
    xt = torch.tensor(x, dtype=torch.bfloat16, device=net.device)
    y = net.forward(xt)
    h = [net.activation(l, n) for l in range(5)]
    torch.cuda.synchronize()
    yield net, p, x, _f64(y), [_f64(t) for t in h]
    net.close()


def test_conv_layers_match_oracle_layer_by_layer(net_and_forward):
    net, p, x, y, h = net_and_forward
    np.testing.assert_array_equal(h[0], x)
    for l in range(1, 5):
        z = N.conv_forward(h[l - 1], N.bf16(p[f"W{l}"]), p[f"b{l}"])
        ref = N.bf16(np.maximum(z, 0.0))
        d = np.abs(h[l] - ref)
        assert np.all(d <= 2.0 ** -7 * np.abs(ref) + 2.0 ** -20), f"layer {l}: {d.max():.3e}"
        assert (d > 0).mean() <= 0.01, f"layer {l}: {(d > 0).mean():.4f} of the values differ"
        assert ref.max() > 0


def test_dense_head_matches_oracle(net_and_forward):
    net, p, x, y, h = net_and_forward
    ref = h[4].reshape(len(x), -1) @ N.bf16(p["W5"]).T + p["b5"]
    assert np.abs(y - ref).max() <= 2e-3 * np.abs(ref).max()


def _forward_with_flips(p, x, rng, frac):
    """The oracle's forward with the discrepancy the layer test allows: one
    BF16 step (2^-8 |h|, the typical spacing) up or down at a random fraction
    `frac` of every layer's stored activations."""
    h = N.bf16(x)
    for l in range(1, 5):
        h = N.bf16(np.maximum(N.conv_forward(h, N.bf16(p[f"W{l}"]), p[f"b{l}"]), 0.0))
        flip = (rng.random(h.shape) < frac) * rng.choice([-1.0, 1.0], h.shape)
        h = h + flip * np.abs(h) * 2.0 ** -8
    return h.reshape(h.shape[0], -1) @ N.bf16(p["W5"]).T + p["b5"]


def test_end_to_end_forward_close_to_oracle(net_and_forward):
    """Raw input to output, no GPU activations fed to the oracle.  The
    tolerance is derived from the stored activations' BF16 rounding: the GPU
    and the oracle round each stored activation from sums taken in FP32 and
    FP64, so they may differ by one BF16 step at up to 1 % of the values
    (the layer test's bar).  Propagating such flips through the oracle's
    network (8 random draws) gives the output spread they cause; the GPU must
    stay within 3x its largest value, element by element."""
    net, p, x, y, h = net_and_forward
    ref = N.forward(p, x)["out"]
    spread = np.max([np.abs(_forward_with_flips(p, x, np.random.default_rng(100 + k), 0.01) - ref)
                     for k in range(8)], axis=0)
    tol = 3.0 * spread.max()
    err = np.abs(y - ref).max()
    assert err <= tol, f"end-to-end error {err:.3e} vs derived tolerance {tol:.3e}"
    assert tol <= 2e-2 * np.abs(ref).max()


def test_backward_matches_oracle(net_and_forward):
    net, p, x, y, h = net_and_forward
    n = len(x)
    dy = np.random.default_rng(9).standard_normal((n, W.N_OUT)) / n
    g = net.backward(torch.tensor(dy, dtype=torch.float32, device=net.device))
    gpu = W.unflatten_params(g.cpu().numpy().astype(np.float64))
    acts = {f"h{l}": h[l] for l in range(5)}
    ref = N.backward(p, acts, dy)
    for k, _ in W.param_layout():
        scale = np.abs(ref[k]).max()
        assert scale > 0, k
        err = np.abs(gpu[k] - ref[k]).max()
        assert err <= 2e-3 * scale, f"{k}: {err:.3e} vs {scale:.3e}"


def test_first_adam_step_moves_every_weight_by_lr_against_its_gradient():
    """Adam's first step from zero moments is -lr * g / (|g| + eps): each
    parameter moves by lr against the sign of its gradient."""
    n = 16
    p = _params(11)
    x = torch.tensor(_inputs(n, 12), dtype=torch.bfloat16, device="cuda")
    t = torch.tensor(np.random.default_rng(13).normal(0, 0.5, (n, W.N_OUT)), dtype=torch.float32,
                     device="cuda")
    net = W.WarmStartNet(batch_max=n, params=p)
    y = net.forward(x)
    dy = 2.0 * (y - t) / y.numel()
    g = net.backward(dy).cpu().numpy()
    p0 = net.get_params()
    loss = torch.zeros(1, device="cuda")
    net.train_step(x, t, 1e-3, loss)
    p1 = net.get_params()
    torch.cuda.synchronize()
    assert float(loss) == pytest.approx(float(((y - t) ** 2).mean()), rel=1e-5)
    big = np.abs(g) > 1e-4
    assert big.sum() > 1000
    np.testing.assert_allclose((p1 - p0)[big], -1e-3 * np.sign(g[big]), rtol=2e-3, atol=1e-7)
    assert net.status() == 0
    net.close()


def test_training_fits_a_small_batch():
    n = 32
    x = torch.tensor(_inputs(n, 21), dtype=torch.bfloat16, device="cuda")
    t = torch.tensor(np.random.default_rng(22).normal(0, 0.5, (n, W.N_OUT)), dtype=torch.float32,
                     device="cuda")
    net = W.WarmStartNet(batch_max=n, seed=5)
    loss = torch.zeros(1, device="cuda")
    hist = []
    for it in range(300):
        net.train_step(x, t, 2e-3, loss)
        if it % 50 == 0 or it == 299:
            hist.append(float(loss))
    assert hist[-1] < 0.1 * hist[0], hist
    assert net.status() == 0
    net.close()


def test_bev_projection_matches_oracle():
    from paper_2512_18863_gb300 import synth as S
    ph = S.pelvis_phantom(n=(40, 64, 96), spacing=(4.0, 4.0, 4.0), seed=3,
                          ptv_radii=(30.0, 25.0, 35.0), ptv_offset=(10.0, -5.0, 8.0))
    g = [0.0, 33.0, 90.0, 211.0]
    got = _f64(W.bev_inputs(ph, g, (0.0, 0.0, 0.0)))
    nz, ny, nx = ph.shape
    reach = 0.5 * np.sqrt((nx * 4.0) ** 2 + (ny * 4.0) ** 2)
    ref = N.bev_project(W.mask_bits(ph), ph.spacing, ph.origin, (0.0, 0.0, 0.0), 1000.0, g, 64,
                        W.BEV_PITCH_MM, reach, 2.0)
    assert ref[..., 0].sum() > 100 and ref[..., 1].sum() > 50 and ref[..., 2].sum() > 50
    # byte-valued output: bit-exact (both sides take the nearest-voxel
    # decisions in FP32 with the same rounded operations)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("seed,side_deg", [(5, 0.0), (6, 17.3), (7, 255.5)])
def test_bev_projection_bit_exact_on_ragged_grids(seed, side_deg):
    """Odd, anisotropic grids with an off-centre isocentre and angles that put
    sample points near voxel boundaries: still bit-exact."""
    from paper_2512_18863_gb300 import _lib
    from paper_2512_18863_gb300 import synth as S
    rng = np.random.default_rng(seed)
    ph = S.pelvis_phantom(n=(23, 41, 57), spacing=(3.5, 3.5, 2.5), seed=seed,
                          ptv_radii=(25.0, 20.0, 22.0), ptv_offset=(4.0, -3.0, 2.0))
    iso = (float(rng.uniform(-6, 6)), float(rng.uniform(-6, 6)), float(rng.uniform(-4, 4)))
    g = [side_deg + 37.0 * k for k in range(5)]
    bits = W.mask_bits(ph)
    dev = torch.device("cuda", torch.cuda.current_device())
    bt = torch.tensor(bits, device=dev)
    out = torch.empty((len(g), 64, 64, 3), dtype=torch.bfloat16, device=dev)
    nz, ny, nx = ph.shape
    reach, step = 110.0, 1.25
    _lib.pdrt_bev_project(bt.data_ptr(), nx, ny, nz, ph.spacing, ph.origin, iso, 1000.0, g, 64,
                          W.BEV_PITCH_MM, reach, step, out.data_ptr(),
                          torch.cuda.current_stream().cuda_stream)
    ref = N.bev_project(bits, ph.spacing, ph.origin, iso, 1000.0, g, 64, W.BEV_PITCH_MM, reach, step)
    assert ref.sum() > 100
    np.testing.assert_array_equal(_f64(out), ref)
