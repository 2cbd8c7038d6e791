"""FP64 oracle of the warm-start network (test infrastructure only).

The paper names a network that learns delivery parameters from target and
organ-at-risk masks as a future direction (Discussion, "Future directions")
without fixing its form; this module is the definition the CUDA kernels are
checked against:

  input   x    [B][64][64][3]  beam's-eye-view projections of PTV, bladder,
                                rectum (0/1), NHWC, BF16 (exact for 0/1)
  conv l  z_l  = b_l + sum_{ky,kx,ci} W_l[co][ky][kx][ci] h_{l-1}[2y+ky-1][2x+kx-1][ci]
               (3x3, stride 2, zero padding 1; l = 1..4, 64 output channels,
                spatial 64 -> 32 -> 16 -> 8 -> 4)
          h_l  = bf16(relu(z_l))            (stored activations are BF16)
  dense   out  = b_5 + W_5 h_4              (h_4 flattened in (y, x, c) order,
                                             1024 -> 121, FP32 output)

Weights enter every product rounded to BF16; sums are exact here (FP64) and
FP32 on the GPU.  Backward of an upstream gradient dout [B][121]:

  g_5  = bf16(dout)
  dW_5 = g_5^T h_4,  db_5 = sum_b g_5,  dh_4 = g_5 W_5
  g_l  = bf16(dh_l * [h_l > 0])                         (l = 4..1)
  dW_l = sum_pixels g_l (x) im2col(h_{l-1}),  db_l = sum_pixels g_l
  dh_{l-1} = col2im(g_l W_l)                             (l >= 2)

bf16() is round-to-nearest-even of the FP32 value.  With bf16=False every
rounding is skipped (a plain FP64 network, used for finite-difference pins).

Only tests/ and the benchmark's baseline leg may import this module.
"""
from __future__ import annotations

import math

import numpy as np

N_OUT = 121          # 60 leaf pairs x (left, right) + MU
CH = 64
IN_CH = 3
SIDE = 64


def bf16(x) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    u = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed: int) -> dict:
    """He-style initialisation (FP64 master values)."""
    rng = np.random.default_rng(seed)
    p = {}
    cin = IN_CH
    for l in range(1, 5):
        fan = 9 * cin
        p[f"W{l}"] = rng.normal(0.0, np.sqrt(2.0 / fan), size=(CH, 3, 3, cin))
        p[f"b{l}"] = np.zeros(CH)
        cin = CH
    p["W5"] = rng.normal(0.0, np.sqrt(1.0 / 1024), size=(N_OUT, 4 * 4 * CH))
    p["b5"] = np.zeros(N_OUT)
    return p


def _patches(xp, ky, kx, ho, wo):
    return xp[:, ky:ky + 2 * ho:2, kx:kx + 2 * wo:2, :]


def conv_forward(x, W, b):
    """z[b][y][x][o] = b[o] + sum W[o][ky][kx][c] x[b][2y+ky-1][2x+kx-1][c]."""
    B, H, Wd, C = x.shape
    ho, wo = H // 2, Wd // 2
    xp = np.zeros((B, H + 2, Wd + 2, C))
    xp[:, 1:-1, 1:-1, :] = x
    z = np.zeros((B, ho, wo, W.shape[0])) + b
    for ky in range(3):
        for kx in range(3):
            z += np.einsum("bhwc,oc->bhwo", _patches(xp, ky, kx, ho, wo), W[:, ky, kx, :])
    return z


def conv_backward(x, W, g):
    """Weight, bias and input gradients of conv_forward for upstream g."""
    B, H, Wd, C = x.shape
    ho, wo = H // 2, Wd // 2
    xp = np.zeros((B, H + 2, Wd + 2, C))
    xp[:, 1:-1, 1:-1, :] = x
    dW = np.zeros_like(W)
    dxp = np.zeros_like(xp)
    for ky in range(3):
        for kx in range(3):
            dW[:, ky, kx, :] = np.einsum("bhwo,bhwc->oc", g, _patches(xp, ky, kx, ho, wo))
            dxp[:, ky:ky + 2 * ho:2, kx:kx + 2 * wo:2, :] += np.einsum("bhwo,oc->bhwc", g,
                                                                       W[:, ky, kx, :])
    return dW, g.sum(axis=(0, 1, 2)), dxp[:, 1:-1, 1:-1, :]


def forward(params: dict, x, bf=True) -> dict:
    """Activations of the whole network (see the module docstring)."""
    r = bf16 if bf else (lambda a: np.asarray(a, dtype=np.float64))
    acts = {"h0": r(x)}
    h = acts["h0"]
    for l in range(1, 5):
        z = conv_forward(h, r(params[f"W{l}"]), params[f"b{l}"])
        h = r(np.maximum(z, 0.0))
        acts[f"z{l}"] = z
        acts[f"h{l}"] = h
    flat = h.reshape(h.shape[0], -1)
    acts["out"] = flat @ r(params["W5"]).T + params["b5"]
    return acts


def backward(params: dict, acts: dict, dout, bf=True) -> dict:
    """Parameter gradients for upstream dout [B][121] (see the docstring)."""
    r = bf16 if bf else (lambda a: np.asarray(a, dtype=np.float64))
    grads = {}
    g = r(dout)
    h4 = acts["h4"]
    flat = h4.reshape(h4.shape[0], -1)
    grads["W5"] = g.T @ flat
    grads["b5"] = g.sum(axis=0)
    dh = (g @ r(params["W5"])).reshape(h4.shape)
    for l in range(4, 0, -1):
        gl = r(dh * (acts[f"h{l}"] > 0))
        dW, db, dx = conv_backward(acts[f"h{l - 1}"], r(params[f"W{l}"]), gl)
        grads[f"W{l}"] = dW
        grads[f"b{l}"] = db
        dh = dx
    return grads


def mse_loss(out, target):
    """L = mean over all entries of (out - target)^2 and dL/dout."""
    d = out - target
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, Algorithm 1) on arrays p, g, m, v at
    step t >= 1; returns the new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def bev_project(bits, spacing, origin, iso, sid, gantry_deg, side, pitch, reach, step):
    """Beam's-eye-view projection of a uint8 bit-mask volume bits [nz][ny][nx]
    (the network input): for each gantry angle g and BEV pixel (py, px), the
    ray from the source S = iso - sid e_w through P = iso + u e_u + v e_v, with
    e_w = (sin g, cos g, 0), e_u = (cos g, -sin g, 0), e_v = (0, 0, 1),
    u = (px - (side-1)/2) pitch, v = (py - (side-1)/2) pitch, is sampled at
    depths w = -reach, -reach + step, ... (n = floor(2 reach / step) + 1
    samples) beyond the isocentre plane, i.e. at X = S + t (P - S) with
    t = (sid + w) / sid; channel s is 1 where a sample's nearest voxel
    round((X - origin) / spacing) has bit s.  Returns float64
    [n_cp][side][side][3].

    The nearest-voxel index is an integer decided by floating point, so it is
    taken in the kernel's precision: FP32, each operation rounded to nearest
    (numpy float32 arithmetic is IEEE single precision), in this order:
    S = (iso_x - sid sn, iso_y - sid cs, iso_z); P - S = (u cs + sid sn,
    -(u sn) + sid cs, v); X = S + t (P - S) per axis; index = rint((X - o) / s)
    with ties to even.  cs and sn are cos and sin of (g pi / 180) in double,
    then rounded to FP32."""
    f = np.float32
    nz, ny, nx = bits.shape
    out = np.zeros((len(gantry_deg), side, side, 3))
    half = f(0.5) * f(side - 1)
    idx_pix = np.arange(side, dtype=np.float32)
    pu = (idx_pix - half) * f(pitch)                    # float32 ops, rounded per step
    U, V = np.meshgrid(pu, pu)                          # [py][px]
    n_steps = int(np.floor(2.0 * reach / step)) + 1
    sid32, reach32, step32 = f(sid), f(reach), f(step)
    o32 = [f(origin[d]) for d in range(3)]
    s32 = [f(spacing[d]) for d in range(3)]
    iso32 = [f(iso[d]) for d in range(3)]
    for b, g in enumerate(gantry_deg):
        ang = float(g) * math.pi / 180.0
        cs, sn = f(math.cos(ang)), f(math.sin(ang))
        S = (iso32[0] - sid32 * sn, iso32[1] - sid32 * cs, iso32[2])
        Dv = (U * cs + sid32 * sn, -(U * sn) + sid32 * cs, V)
        acc = np.zeros((side, side), dtype=np.uint8)
        for q in range(n_steps):
            w = -reach32 + f(q) * step32
            t = (sid32 + w) / sid32
            idx = [np.rint((S[d] + t * Dv[d] - o32[d]) / s32[d]).astype(np.int64) for d in range(3)]
            ok = ((idx[0] >= 0) & (idx[0] < nx) & (idx[1] >= 0) & (idx[1] < ny)
                  & (idx[2] >= 0) & (idx[2] < nz))
            vals = np.zeros((side, side), dtype=np.uint8)
            vals[ok] = bits[idx[2][ok], idx[1][ok], idx[0][ok]]
            acc |= vals
        for s in range(3):
            out[b, :, :, s] = (acc >> s) & 1
    return out
