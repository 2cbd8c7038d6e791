"""Learned warm start for the plan optimiser.

The paper's Discussion ("Future directions") proposes a network that learns
delivery parameters from target and organ-at-risk masks, with the dose
engine as the judge.  Here a 5-layer BF16 CNN (include/pdrt_cnn.h) maps the
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
