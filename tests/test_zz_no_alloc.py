"""pdrt_cp_dose_static: the allocation-free single-control-point dose.

Callers that cannot call cudaMalloc (a plug-in whose host framework owns all
device memory, a latency-critical loop that must not enter the allocator) use
this entry point; its scratch is a static device array inside the library.
The test calls it through the C ABI twice in a row and checks each result
against the existing entry point (pdrt_dose_forward on a one-point plan)
within the dose tolerance of the other GPU tests, and checks that a grid
needing more than the static scratch is rejected with a clear error.
The file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

from paper_2512_18863_gb300 import _lib
from paper_2512_18863_gb300 import synth as S
from paper_2512_18863_gb300.engine import DoseEngine

pytestmark = pytest.mark.gpu

DOSE_TOL = 1e-4


def _red(ph):
    pts = np.asarray(ph.hu_to_red, np.float64)
    return np.interp(np.asarray(ph.hu, np.float64), pts[:, 0], pts[:, 1]).astype(np.float32)


def _static_dose(w, b, red, out):
    ph, dev = w.phantom, out.device
    nz, ny, nx = ph.hu.shape
    leaves = torch.tensor(w.plan.leaves[b], dtype=torch.float32, device=dev).contiguous()
    jaws = torch.tensor(w.plan.jaws[b], dtype=torch.float32, device=dev).contiguous()
    mu = torch.tensor(w.plan.mu[b:b + 1], dtype=torch.float32, device=dev).contiguous()
    _lib.pdrt_cp_dose_static(red.data_ptr(), nx, ny, nz, *ph.spacing, list(ph.origin),
                             list(w.plan.iso), float(w.plan.gantry_deg[b]),
                             _lib.machine_struct(w.machine), leaves.data_ptr(), jaws.data_ptr(),
                             mu.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return out.cpu().numpy().astype(np.float64)


def test_static_scratch_dose_matches_plan_forward_twice():
    w = S.small_pelvis(seed=31, n=(24, 44, 44), spacing=3.0, n_cp=3, r_px=8)
    dev = torch.device("cuda", torch.cuda.current_device())
    red = torch.tensor(_red(w.phantom), device=dev)
    out = torch.empty(w.phantom.shape, dtype=torch.float32, device=dev)
    for b in (1, 2):                      # two calls in a row share the static array
        got = _static_dose(w, b, red, out)
        eng = DoseEngine(w.phantom, w.machine, w.plan.gantry_deg[b:b + 1], w.plan.iso)
        ref = eng.forward(w.plan.leaves[b:b + 1], w.plan.jaws[b:b + 1], w.plan.mu[b:b + 1])
        ref = ref.cpu().numpy().astype(np.float64)
        eng.close()
        assert ref.max() > 0
        assert np.abs(got - ref).max() <= DOSE_TOL * ref.max()


def test_static_scratch_dose_with_fluence_corrections():
    """The corrections path (penumbra blurs, off-axis profile, collimator
    rotation) uses two more carve-outs of the static array; its dose matches
    the plan forward on a one-point plan, on two calls in a row."""
    w = S.small_pelvis(seed=33, n=(24, 44, 44), spacing=3.0, n_cp=2, r_px=6)
    S.with_corrections(w.machine, seed=7, collimator_deg=23.0)
    dev = torch.device("cuda", torch.cuda.current_device())
    red = torch.tensor(_red(w.phantom), device=dev)
    out = torch.empty(w.phantom.shape, dtype=torch.float32, device=dev)
    for b in (0, 1):
        got = _static_dose(w, b, red, out)
        eng = DoseEngine(w.phantom, w.machine, w.plan.gantry_deg[b:b + 1], w.plan.iso)
        ref = eng.forward(w.plan.leaves[b:b + 1], w.plan.jaws[b:b + 1], w.plan.mu[b:b + 1])
        ref = ref.cpu().numpy().astype(np.float64)
        eng.close()
        assert ref.max() > 0
        assert np.abs(got - ref).max() <= DOSE_TOL * ref.max()


def test_static_scratch_reports_nan_input():
    """A NaN MU raises the device's input flag; the call reads it back and
    returns EINVAL instead of a silently wrong dose.  The next valid call
    succeeds (the flags are cleared at the start of each call)."""
    w = S.small_pelvis(seed=34, n=(16, 32, 32), spacing=3.0, n_cp=1, r_px=4)
    dev = torch.device("cuda", torch.cuda.current_device())
    red = torch.tensor(_red(w.phantom), device=dev)
    out = torch.empty(w.phantom.shape, dtype=torch.float32, device=dev)
    good_mu = w.plan.mu.copy()
    w.plan.mu[0] = np.nan
    with pytest.raises(_lib.PdrtError) as e:
        _static_dose(w, 0, red, out)
    assert e.value.status == 1 and "NaN" in str(e.value)
    w.plan.mu[:] = good_mu
    assert _static_dose(w, 0, red, out).max() > 0


def test_static_scratch_rejects_oversized_grid():
    w = S.small_pelvis(seed=32, n=(16, 16, 16), spacing=3.0, n_cp=1, r_px=4)
    dev = torch.device("cuda", torch.cuda.current_device())
    red = torch.zeros((1,), device=dev)
    out = torch.empty((1,), device=dev)
    ph = w.phantom
    with pytest.raises(_lib.PdrtError) as e:      # 400^3 at 1 mm needs ~256 MiB of scratch
        _lib.pdrt_cp_dose_static(red.data_ptr(), 400, 400, 400, 1.0, 1.0, 1.0,
                                 [-200.0, -200.0, -200.0], [0.0, 0.0, 0.0], 0.0,
                                 _lib.machine_struct(w.machine), red.data_ptr(), red.data_ptr(),
                                 red.data_ptr(), out.data_ptr(), 0)
    assert e.value.status == 1 and "MiB of scratch" in str(e.value)
    del ph
