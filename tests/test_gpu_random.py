"""Randomised parity sweep: seeded small cases across grid shapes, voxel
sizes, kernel radii, control-point counts, field sizes and the fluence
corrections, each on the oracle's bars (dose max |dD| <= 1e-4 max D;
gradients ||dg||_inf <= 1e-3 ||g||_inf per parameter class).  The case
parameters are drawn from a fixed seed; every expected value comes from the
FP64 oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_18863_gb300 import synth as S
from paper_2512_18863_gb300.engine import DoseEngine

pytestmark = pytest.mark.gpu

DOSE_TOL = 1e-4
GRAD_TOL = 1e-3


def _case(q):
    rng = np.random.default_rng(7000 + q)
    n = (int(rng.integers(12, 30)), int(rng.integers(18, 48)), int(rng.integers(18, 48)))
    spacing = float(rng.choice([2.0, 2.5, 3.0, 4.0, 5.0]))
    n_cp = int(rng.integers(1, 7))
    r_px = int(rng.choice([1, 2, 3, 5, 8, 12, 17, 24, 30]))
    radii = tuple(float(v) for v in rng.uniform(8.0, 0.3 * min(n[1], n[2]) * spacing, 3))
    w = S.small_pelvis(seed=7100 + q, n=n, spacing=spacing, n_cp=n_cp, r_px=r_px, ptv_radii=radii)
    w.plan.gantry_deg[:] = rng.uniform(0.0, 360.0, n_cp)
    if q % 2 == 1:   # source penumbra, off-axis profile, collimator angle
        S.with_corrections(w.machine, 7200 + q, collimator_deg=float(rng.uniform(-30.0, 30.0)))
    return w


@pytest.mark.parametrize("q", range(16))
def test_random_case_matches_oracle(q):
    w = _case(q)
    eng = DoseEngine(w.phantom, w.machine, w.plan.gantry_deg, w.plan.iso)
    d = eng.forward(w.plan.leaves, w.plan.jaws, w.plan.mu).cpu().numpy().astype(np.float64)
    g = np.random.default_rng(7300 + q).standard_normal(w.phantom.shape)
    dl, dj, dm = (t.cpu().numpy().astype(np.float64)
                  for t in eng.backward(w.plan.leaves, w.plan.jaws, w.plan.mu, g))
    assert eng.status_flags() == 0
    eng.close()
    mod = O.Model(w.phantom, w.machine, w.plan)
    ref = mod.dose()
    assert ref.max() > 0, "case without dose"
    err = np.abs(d - ref).max()
    assert err <= DOSE_TOL * ref.max(), f"case {q}: max |dD| = {err:.3e} vs {ref.max():.4e}"
    for got, exp, name in zip((dl, dj, dm), mod.dose_grad(g), ("leaves", "jaws", "mu")):
        scale = np.abs(exp).max()
        if scale == 0.0:
            assert np.abs(got).max() == 0.0, f"case {q} {name}"
            continue
        e = np.abs(got - exp).max()
        assert e <= GRAD_TOL * scale, f"case {q} {name}: {e:.3e} vs {scale:.4e}"
