"""Many independent plans in one CUDA-graph launch (pdrt_batch_*).

The beam sequence of the paper is organised for batched operation (Sec. 2.2);
here whole plans -- each a DoseEngine with its own grid and arc -- are
recorded once into a single CUDA graph with parallel branches and replayed
with one graph launch.  The batch owns the device buffers the graph reads and
writes: set inputs with copy_() into `leaves[i]`, `jaws[i]`, `mu[i]`,
`dose_grad[i]`; read `dose[i]`, `dleaves[i]`, `djaws[i]`, `dmu[i]`.
A None gradient entry records the forward alone for that plan.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib
from .engine import DoseEngine, _stream_ptr


class DoseBatch:
    def __init__(self, engines, leaves, jaws, mu, dose_grad=None, n_branches=4):
        self.engines = list(engines)
        n = len(self.engines)
        dev = self.engines[0].device
        self.leaves = [torch.as_tensor(leaves[i], dtype=torch.float32, device=dev).contiguous().clone()
                       for i in range(n)]
        self.jaws = [torch.as_tensor(jaws[i], dtype=torch.float32, device=dev).contiguous().clone()
                     for i in range(n)]
        self.mu = [torch.as_tensor(mu[i], dtype=torch.float32, device=dev).contiguous().clone()
                   for i in range(n)]
        self.dose = [torch.empty(e.shape, dtype=torch.float32, device=dev) for e in self.engines]
        self.dose_grad = self.dleaves = self.djaws = self.dmu = None
        if dose_grad is not None:
            # a None entry: forward only for that plan (its gradient entries stay None)
            has = [dose_grad[i] is not None for i in range(n)]
            self.dose_grad = [torch.as_tensor(dose_grad[i], dtype=torch.float32, device=dev)
                              .contiguous().clone() if has[i] else None for i in range(n)]
            self.dleaves = [torch.empty_like(t) if h else None for t, h in zip(self.leaves, has)]
            self.djaws = [torch.empty_like(t) if h else None for t, h in zip(self.jaws, has)]
            self.dmu = [torch.empty_like(t) if h else None for t, h in zip(self.mu, has)]
        ptrs = lambda ts: None if ts is None else [0 if t is None else t.data_ptr() for t in ts]
        self._batch = _lib.pdrt_batch_create(
            [e._grid for e in self.engines], [e._plan for e in self.engines], ptrs(self.leaves),
            ptrs(self.jaws), ptrs(self.mu), ptrs(self.dose), ptrs(self.dose_grad),
            ptrs(self.dleaves), ptrs(self.djaws), ptrs(self.dmu), n_branches, _stream_ptr())
        self.n = n

    def launch(self):
        _lib.pdrt_batch_launch(self._batch, _stream_ptr())

    def plan_times_ms(self) -> np.ndarray:
        """Completion time of every plan in the last launch, from its start."""
        return np.asarray(_lib.pdrt_batch_plan_times(self._batch, self.n, _stream_ptr()))

    @property
    def kernels(self) -> int:
        return _lib.pdrt_batch_kernels(self._batch)

    @property
    def pass_cp(self) -> list:
        """Control points per pass of each plan in the batch (a plan's dose
        equals its engine's forward at that chunk size bit for bit)."""
        return [_lib.pdrt_batch_pass_cp(self._batch, i) for i in range(self.n)]

    def close(self):
        if getattr(self, "_batch", None):
            _lib.pdrt_batch_destroy(self._batch)
            self._batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
