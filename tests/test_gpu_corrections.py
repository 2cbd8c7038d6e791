"""GPU vs FP64 oracle parity of the fluence corrections of Sec. 2.2.2
(source penumbra, off-axis profile, collimator rotation), forward and
adjoint, through the C ABI.  Same bars as the uncorrected path: dose
max |dD| <= 1e-4 max D; gradients ||dg||_inf <= 1e-3 ||g||_inf per class."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_18863_gb300 import synth as S
from paper_2512_18863_gb300.engine import DoseEngine

pytestmark = pytest.mark.gpu

DOSE_TOL = 1e-4
GRAD_TOL = 1e-3


def _case(seed, coll, n=(20, 36, 36), n_cp=4, r_px=6, spacing=3.0, pen=(4.0, 6.0)):
    w = S.small_pelvis(seed=seed, n=n, spacing=spacing, n_cp=n_cp, r_px=r_px)
    S.with_corrections(w.machine, seed + 100, pen=pen, collimator_deg=coll)
    return w


def _engine(w, **kw):
    return DoseEngine(w.phantom, w.machine, w.plan.gantry_deg, w.plan.iso, **kw)


@pytest.mark.parametrize("conv", ["fft", "tc", "simt"])
@pytest.mark.parametrize("coll", [0.0, 30.0, -90.0])
def test_corrected_forward_matches_oracle(coll, conv):
    w = _case(31, coll)
    eng = _engine(w, conv=conv)
    gpu = eng.forward(w.plan.leaves, w.plan.jaws, w.plan.mu).cpu().numpy().astype(np.float64)
    eng.close()
    ref = O.Model(w.phantom, w.machine, w.plan).dose()
    assert ref.max() > 0
    err = np.abs(gpu - ref).max()
    assert err <= DOSE_TOL * ref.max(), f"max |dD| = {err:.3e} vs {DOSE_TOL} * {ref.max():.4e}"


def test_corrections_change_the_dose():
    """The corrected dose differs from the uncorrected one by far more than
    the tolerance (the parity above is not vacuous)."""
    w = _case(32, 25.0)
    eng = _engine(w)
    a = eng.forward(w.plan.leaves, w.plan.jaws, w.plan.mu).cpu().numpy()
    eng.close()
    w0 = S.small_pelvis(seed=32, n=(20, 36, 36), spacing=3.0, n_cp=4, r_px=6)
    eng = _engine(w0)
    b = eng.forward(w0.plan.leaves, w0.plan.jaws, w0.plan.mu).cpu().numpy()
    eng.close()
    assert np.abs(a - b).max() > 100 * DOSE_TOL * b.max()


@pytest.mark.parametrize("conv", ["fft", "tc", "simt"])
@pytest.mark.parametrize("ste,coll", [(1, 0.0), (0, 0.0), (1, 30.0), (0, -17.0)])
def test_corrected_gradients_match_oracle(ste, coll, conv):
    w = _case(33, coll, n_cp=5)
    w.machine.ste = ste
    w.plan.leaves[1, 30] = (2.1, 2.4)      # a pair under w_min
    w.plan.mu[2] = 0.004                   # below eps_mu
    g = np.random.default_rng(6).standard_normal(w.phantom.shape)
    eng = _engine(w, conv=conv)
    got = [t.cpu().numpy().astype(np.float64)
           for t in eng.backward(w.plan.leaves, w.plan.jaws, w.plan.mu, g)]
    eng.close()
    ref = O.Model(w.phantom, w.machine, w.plan).dose_grad(g)
    for name, a, b in zip(("leaves", "jaws", "mu"), got, ref):
        scale = np.abs(b).max()
        assert scale > 0
        err = np.abs(a - b).max()
        assert err <= GRAD_TOL * scale, f"{name}: |dg|_inf = {err:.3e} vs {GRAD_TOL} * {scale:.4e}"


def test_wide_penumbra_and_field_at_the_lattice_edge():
    """Blur half-windows of 4-6 px and a field covering the whole lattice: the
    blurred box is clipped to the lattice (zero padding)."""
    w = _case(34, 12.0, n=(16, 30, 30), n_cp=3, r_px=4, pen=(9.0, 12.0))
    w.plan.jaws[:, 0] = -200.0
    w.plan.jaws[:, 1] = 200.0
    w.plan.leaves[:, :, 0] = -200.0
    w.plan.leaves[:, :, 1] = 200.0
    eng = _engine(w)
    gpu = eng.forward(w.plan.leaves, w.plan.jaws, w.plan.mu).cpu().numpy().astype(np.float64)
    eng.close()
    ref = O.Model(w.phantom, w.machine, w.plan).dose()
    assert np.abs(gpu - ref).max() <= DOSE_TOL * ref.max()


def test_static_entry_applies_the_corrections():
    """The allocation-free single-control-point entry point gives the same
    corrected dose as the oracle."""
    import torch
    from tests.test_zz_no_alloc import _red, _static_dose
    w = _case(35, 20.0, n=(20, 36, 36), n_cp=2)
    dev = torch.device("cuda", torch.cuda.current_device())
    red = torch.tensor(_red(w.phantom), device=dev)
    out = torch.empty(w.phantom.shape, dtype=torch.float32, device=dev)
    got = _static_dose(w, 1, red, out)
    one = S.Plan(gantry_deg=w.plan.gantry_deg[1:2], iso=w.plan.iso, leaves=w.plan.leaves[1:2],
                 jaws=w.plan.jaws[1:2], mu=w.plan.mu[1:2])
    ref = O.Model(w.phantom, w.machine, one).dose()
    assert ref.max() > 0
    assert np.abs(got - ref).max() <= DOSE_TOL * ref.max()
