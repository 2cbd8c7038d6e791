"""DoseEngine: PyTorch-facing wrapper of the sm_103a dose library.

PyTorch provides device memory and the stream; every step of the dose
computation runs in the library's CUDA kernels (via the C ABI in
include/pdrt.h).  DoseFn makes the engine a differentiable layer: its
backward calls the hand-written adjoint (pdrt_dose_backward) and returns
gradients for leaves, jaws and MUs (Sec. 2.1: gradient-carrying layers),
nothing for the fixed geometry.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib


def _stream_ptr():
    return torch.cuda.current_stream().cuda_stream


def _f32(x, device):
    t = torch.as_tensor(x, dtype=torch.float32, device=device)
    return t.contiguous()


def calibrate(machine, sxy, sz, ref_mu=None, ref_gy=None) -> float:
    """Output calibration of Sec. 2.4 by the library (pdrt_calibrate): the
    factor that makes ref_mu MU of the 10 x 10 cm reference field give ref_gy
    Gy at 10 cm depth in water on a grid of pitch (sxy, sxy, sz).  Defaults:
    the machine's cal_ref_mu / cal_ref_gy, else 100 MU -> 1 Gy."""
    if not torch.cuda.is_available():
        raise RuntimeError("calibrate needs a CUDA device (GB300, sm_103a); no CPU path exists")
    ref_mu = float(getattr(machine, "cal_ref_mu", 100.0) if ref_mu is None else ref_mu)
    ref_gy = float(getattr(machine, "cal_ref_gy", 1.0) if ref_gy is None else ref_gy)
    return _lib.pdrt_calibrate(_lib.machine_struct(machine, cal=1.0), sxy, sz, ref_mu, ref_gy,
                               _stream_ptr())


class DoseEngine:
    """One CT grid + one VMAT geometry (gantry angles, isocentre, beam model).

    phantom: object with hu (nz, ny, nx), spacing (sx, sy, sz), origin,
             hu_to_red (n, 2)
    machine: beam model (synth.Machine or any object with the same fields)
    """

    def __init__(self, phantom, machine, gantry_deg, iso, scratch_budget_bytes=0, device=None,
                 tensor_cores=None, conv=None, fft_pmax=None):
        if not torch.cuda.is_available():
            raise RuntimeError("DoseEngine needs a CUDA device (GB300, sm_103a); no CPU path exists")
        _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.shape = tuple(int(s) for s in phantom.hu.shape)
        nz, ny, nx = self.shape
        self.n_cp = len(gantry_deg)
        self.n_pairs = len(machine.leaf_bounds) - 1
        self._grid = None
        self._plan = None
        with torch.cuda.device(self.device):
            hu = _f32(phantom.hu, self.device)
            sx, sy, sz = (float(s) for s in phantom.spacing)
            self._grid = _lib.pdrt_grid_create(hu.data_ptr(), nx, ny, nz, sx, sy, sz,
                                               list(phantom.origin), np.asarray(phantom.hu_to_red),
                                               _stream_ptr())
            # output factor: the machine's, or the calibration of Sec. 2.4
            # on this grid's pitch when the machine leaves it open (None)
            self.cal = machine.cal
            if self.cal is None:
                self.cal = calibrate(machine, sx, sz)
            self._machine = _lib.machine_struct(machine, cal=self.cal)
            self._plan = _lib.pdrt_plan_upload(self._grid, list(np.asarray(gantry_deg, float)),
                                               list(np.asarray(iso, float)), self._machine,
                                               scratch_budget_bytes, _stream_ptr())
            torch.cuda.current_stream().synchronize()   # hu is read by the grid kernel
        if tensor_cores is not None:
            _lib.pdrt_plan_set_tensor_cores(self._plan, tensor_cores)
        self.info = _lib.pdrt_plan_get_info(self._plan)
        self._fft_default = self.info["fft_pmax"]
        if conv is not None or fft_pmax is not None:
            self.set_conv(conv or "fft", fft_pmax)

    def set_conv(self, path: str, fft_pmax=None):
        """Convolution path: "fft" (FFT for slices up to fft_pmax, default the
        upload's choice, tensor cores for the rest), "tc" (tensor cores for
        every slice) or "simt" (FP32 SIMT kernel)."""
        if path == "fft":
            _lib.pdrt_plan_set_tensor_cores(self._plan, True)
            _lib.pdrt_plan_set_fft(self._plan, self._fft_default if fft_pmax is None else fft_pmax)
        elif path == "tc":
            _lib.pdrt_plan_set_tensor_cores(self._plan, True)
            _lib.pdrt_plan_set_fft(self._plan, 0)
        elif path == "simt":
            _lib.pdrt_plan_set_tensor_cores(self._plan, False)
        else:
            raise ValueError(f"unknown convolution path {path!r}")
        self.info = _lib.pdrt_plan_get_info(self._plan)

    # -- raw entry points (tensors on self.device, float32, contiguous) -----
    def forward(self, leaves, jaws, mu, out=None):
        leaves, jaws, mu = self._params(leaves, jaws, mu)
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        _lib.pdrt_dose_forward(self._grid, self._plan, leaves.data_ptr(), jaws.data_ptr(),
                               mu.data_ptr(), out.data_ptr(), _stream_ptr())
        return out

    def backward(self, leaves, jaws, mu, dose_grad):
        leaves, jaws, mu = self._params(leaves, jaws, mu)
        g = _f32(dose_grad, self.device)
        if tuple(g.shape) != self.shape:
            raise ValueError(f"dose gradient shape {tuple(g.shape)} != grid {self.shape}")
        dl = torch.empty_like(leaves)
        dj = torch.empty_like(jaws)
        dm = torch.empty_like(mu)
        _lib.pdrt_dose_backward(self._grid, self._plan, leaves.data_ptr(), jaws.data_ptr(),
                                mu.data_ptr(), g.data_ptr(), dl.data_ptr(), dj.data_ptr(),
                                dm.data_ptr(), _stream_ptr())
        return dl, dj, dm

    def __call__(self, leaves, jaws, mu):
        """Differentiable dose (autograd through the hand-written adjoint)."""
        return DoseFn.apply(leaves, jaws, mu, self)

    # -- diagnostics -----------------------------------------------------------
    def set_tensor_cores(self, enable: bool):
        """Route the convolution to the tensor cores (True; the FFT path, if on,
        keeps the slices within its size limit) or the FP32 SIMT kernel."""
        _lib.pdrt_plan_set_tensor_cores(self._plan, enable)
        self.info = _lib.pdrt_plan_get_info(self._plan)

    def set_spectrum_memo(self, enable: bool):
        """Kernel-spectrum memo of the FFT convolution on (allocated for the
        current FFT size limit) or off (freed); results do not depend on it."""
        _lib.pdrt_plan_set_spectrum_memo(self._plan, enable)
        self.info = _lib.pdrt_plan_get_info(self._plan)

    def reset_spectrum_memo(self):
        """Forget every memoised spectrum (stream-ordered on the current stream)."""
        _lib.pdrt_plan_reset_spectrum_memo(self._plan, _stream_ptr())

    def set_chunk(self, chunk_cp: int):
        """Control points per pass (1 .. the count the scratch was sized for)."""
        _lib.pdrt_plan_set_chunk(self._plan, chunk_cp)
        self.info = _lib.pdrt_plan_get_info(self._plan)

    def autotune(self, leaves, jaws, mu, dose_grad=None):
        """Time the candidate schedules (tensor cores or SIMT, control points
        per pass) on these inputs and keep the fastest on the plan."""
        leaves, jaws, mu = self._params(leaves, jaws, mu)
        out = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        gptr = dl = dj = dm = None
        if dose_grad is not None:
            g = _f32(dose_grad, self.device)
            dl, dj, dm = torch.empty_like(leaves), torch.empty_like(jaws), torch.empty_like(mu)
            gptr = g.data_ptr()
        r = _lib.pdrt_plan_autotune(self._grid, self._plan, leaves.data_ptr(), jaws.data_ptr(),
                                    mu.data_ptr(), out.data_ptr(), gptr,
                                    None if dl is None else dl.data_ptr(),
                                    None if dj is None else dj.data_ptr(),
                                    None if dm is None else dm.data_ptr(), _stream_ptr())
        self.info = _lib.pdrt_plan_get_info(self._plan)
        return r

    def status_flags(self):
        return _lib.pdrt_plan_status(self._plan, _stream_ptr())

    def work(self):
        return _lib.pdrt_plan_work(self._plan, _stream_ptr())

    def profile(self, enable=True):
        _lib.pdrt_profile_enable(self._plan, enable)

    def profile_read(self):
        return _lib.pdrt_profile_read(self._plan, _stream_ptr())

    def close(self):
        if self._plan is not None:
            _lib.pdrt_plan_destroy(self._plan)
            self._plan = None
        if self._grid is not None:
            _lib.pdrt_grid_destroy(self._grid)
            self._grid = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _params(self, leaves, jaws, mu):
        leaves = _f32(leaves, self.device)
        jaws = _f32(jaws, self.device)
        mu = _f32(mu, self.device)
        if tuple(leaves.shape) != (self.n_cp, self.n_pairs, 2):
            raise ValueError(f"leaves must be ({self.n_cp}, {self.n_pairs}, 2), got {tuple(leaves.shape)}")
        if tuple(jaws.shape) != (self.n_cp, 4):
            raise ValueError(f"jaws must be ({self.n_cp}, 4), got {tuple(jaws.shape)}")
        if tuple(mu.shape) != (self.n_cp,):
            raise ValueError(f"mu must be ({self.n_cp},), got {tuple(mu.shape)}")
        return leaves, jaws, mu


class DoseFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, leaves, jaws, mu, engine):
        ctx.engine = engine
        ctx.save_for_backward(leaves, jaws, mu)
        return engine.forward(leaves.detach(), jaws.detach(), mu.detach())

    @staticmethod
    def backward(ctx, g):
        leaves, jaws, mu = ctx.saved_tensors
        dl, dj, dm = ctx.engine.backward(leaves.detach(), jaws.detach(), mu.detach(), g.contiguous())
        return dl.to(leaves.dtype), dj.to(jaws.dtype), dm.to(mu.dtype), None
