"""Pins of the oracle's output calibration (Sec. 2.4: ref_mu MU of a 10 x 10 cm
field give ref_gy Gy at 10 cm depth in water, SSD 90 cm, computed with the
beam model in a virtual water phantom).

The reference point sits on the central axis at the isocentre, so magnification
and inverse square are 1 there and the dose is T(z_ref) times the kernel
weights of the fluence under the window.  Independent checks:
  * the reference slice's depth is 100 mm at any pitch (the slab closed form
    of Sec. 2.2.4 with the partial-volume surface row);
  * while the window stays inside the field's flat part, sum K = 1 and the
    fluence is 1, so cal = ref_gy / (ref_mu T(100 mm)) with T read from the
    depth-dose table by numpy's interpolation;
  * for a window wider than the field, the fluence is the hand-worked product
    of 1-D overlaps and cal = ref_gy / (ref_mu T(100) sum_taps K F);
  * a uniform off-axis factor c0 divides cal by c0; a penumbra blur whose
    window stays inside the field leaves cal unchanged; cal scales with
    ref_gy / ref_mu.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_18863_gb300 import synth as S


def _T(m, z):
    return np.interp(z, np.arange(len(m.t_table)) * m.dz_t, m.t_table)


@pytest.mark.parametrize("pitch,sz", [(2.0, 2.0), (2.5, 2.5), (3.0, 3.0), (2.0, 3.0), (1.7, 2.3)])
def test_reference_depth_is_100_mm_and_cal_is_inverse_depth_dose(pitch, sz):
    d = max(pitch, sz)
    m = S.machine_model(11, r_px=int((50.0 - d / 2) // d))   # window inside the flat field
    cal, z_ref, dpm = O.calibrate(m, pitch, sz, details=True)
    assert z_ref == pytest.approx(100.0, abs=1e-9)
    assert dpm == pytest.approx(_T(m, 100.0), rel=1e-12)
    assert cal == pytest.approx(1.0 / (100.0 * _T(m, 100.0)), rel=1e-12)


def _overlap_1d(x, lo, hi, d):
    return np.clip(np.minimum(hi, x + d / 2) - np.maximum(lo, x - d / 2), 0.0, None) / d


@pytest.mark.parametrize("r_px", [30, 40])
def test_window_wider_than_field(r_px):
    """R = 6 / 8 cm at 2 mm: the window reaches past the field edge, so the
    reference dose is T(100) sum_{p,q} K(p,q) F(p,q) with
    F = f(u) f(v) (tau + (1 - tau) f(u)): the jaws' overlaps times the open
    leaves' (every pixel row of the field lies inside the MLC span, where the
    strip weights sum to 1)."""
    m = S.machine_model(12, r_px=r_px)
    cal = O.calibrate(m, 2.0, 2.0)
    ph = S.water_phantom(n=(8, 8, 8), spacing=(2.0, 2.0, 2.0))
    pl = S.static_field(m, 0.0)
    K = O.Model(ph, m, pl).kernel(100.0)
    t = np.arange(-r_px, r_px + 1) * 2.0
    fu = _overlap_1d(t, -50.0, 50.0, 2.0)
    F = fu[:, None] * fu[None, :] * (m.tau + (1 - m.tau) * fu[None, :])   # [v][u]
    assert fu.min() == 0.0 and 0.0 < fu[np.searchsorted(t, 50.0)] < 1.0
    dref = _T(m, 100.0) * float((K * F).sum())
    assert cal == pytest.approx(1.0 / (100.0 * dref), rel=1e-11)
    assert (K * F).sum() < 0.999   # the window does reach past the field


def test_off_axis_factor_blur_and_reference_values():
    m = S.machine_model(13, r_px=10)
    base = O.calibrate(m, 2.0, 2.0)
    m.off_axis = (1.07, 0.0, 0.0)
    assert O.calibrate(m, 2.0, 2.0) == pytest.approx(base / 1.07, rel=1e-12)
    m.off_axis = (1.0, 0.0, 0.0)
    m.pen_fwhm_u, m.pen_fwhm_v = 4.0, 6.0        # blur windows 4 / 5 px, R = 10: inside the field
    assert O.calibrate(m, 2.0, 2.0) == pytest.approx(base, rel=1e-12)
    m.pen_fwhm_u = m.pen_fwhm_v = 0.0
    assert O.calibrate(m, 2.0, 2.0, ref_mu=200.0, ref_gy=3.0) == pytest.approx(base * 1.5, rel=1e-12)
    # the collimator angle of the machine does not enter the reference field
    m.collimator_deg = 33.0
    assert O.calibrate(m, 2.0, 2.0) == pytest.approx(base, rel=1e-12)


def test_model_resolves_a_missing_factor_by_calibration():
    w = S.small_pelvis(seed=5, n=(12, 20, 20), spacing=3.0, n_cp=2, r_px=3)
    d1 = O.Model(w.phantom, w.machine, w.plan).dose()
    w.machine.cal = None
    mod = O.Model(w.phantom, w.machine, w.plan)
    assert mod.cal == pytest.approx(O.calibrate(w.machine, 3.0, 3.0), rel=1e-15)
    assert np.allclose(mod.dose(), mod.cal * d1, rtol=1e-12, atol=0)
