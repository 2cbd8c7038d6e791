"""The seeded synthetic inputs follow their stated recipe: grid shapes and
voxel sizes of the named workloads, the pelvis phantom's structures and HU
values, the 60-pair MLC, arcs whose leaves stay within +-10 mm of the
target's beam's-eye-view edge with conforming jaws, MU ranges, and the beam
model's normalisation.  These stand in for the paper's patient cohorts and
commissioning data, which are not available."""
import numpy as np
import pytest

from paper_2512_18863_gb300 import synth as S


def test_mlc_has_60_pairs_of_10_and_5_mm():
    lb = S.leaf_bounds_60()
    w = np.diff(lb)
    assert len(w) == 60 and lb[0] == -200.0 and lb[-1] == 200.0
    assert np.all(w[:10] == 10.0) and np.all(w[10:50] == 5.0) and np.all(w[50:] == 10.0)


def test_water_static_64_workload():
    w = S.water_static_64()
    ph, pl = w.phantom, w.plan
    assert ph.hu.shape == (64, 64, 64) and np.all(ph.hu == 0.0) and ph.spacing == (2.5, 2.5, 2.5)
    assert ph.origin == (-80.0, -80.0, -80.0)             # iso at voxel (32, 32, 32)
    assert pl.n_cp == 1 and pl.gantry_deg[0] == 0.0 and pl.mu[0] == 100.0
    assert np.all(pl.jaws[0] == (-50.0, 50.0, -50.0, 50.0))
    assert np.all(pl.leaves[0, :, 0] == -50.0) and np.all(pl.leaves[0, :, 1] == 50.0)
    assert w.machine.r_px == 8 and w.machine.sid == 1000.0  # 2 cm at 2.5 mm


@pytest.mark.parametrize("r_cm,r_px", [(2.0, 10), (4.0, 20), (8.0, 40)])
def test_two_arc_256_shapes_and_radii(r_cm, r_px):
    w = S.pelvis_two_arc_256(r_cm=r_cm)
    assert w.phantom.hu.shape == (160, 256, 256) and w.phantom.spacing == (2.0, 2.0, 2.0)
    assert w.machine.r_px == r_px
    g = w.plan.gantry_deg
    assert len(g) == 356
    np.testing.assert_allclose(g[:178], np.arange(178) * 360.0 / 178)
    np.testing.assert_allclose(g[178:], g[:178][::-1])     # second arc reversed
    for k in ("ptv", "bladder", "rectum"):
        assert w.phantom.masks[k].any()
    assert not (w.phantom.masks["bladder"] & w.phantom.masks["ptv"]).any()
    assert not (w.phantom.masks["rectum"] & w.phantom.masks["ptv"]).any()


@pytest.fixture(scope="module")
def c2():
    return S.pelvis_arc_128()


def test_pelvis_phantom_structures(c2):
    ph = c2.phantom
    assert ph.hu.shape == (96, 128, 128) and ph.spacing == (3.0, 3.0, 3.0)
    Z, Y, X = np.meshgrid(*(o + s * np.arange(n) for o, s, n in
                            zip(ph.origin[::-1], ph.spacing[::-1], ph.hu.shape)), indexing="ij")
    body = ph.masks["body"]
    np.testing.assert_array_equal(body, (X / 180.0) ** 2 + (Y / 120.0) ** 2 <= 1.0)
    assert np.all(ph.hu[~body] == -1000.0)
    soft = body & (ph.hu != 700.0) & (ph.hu != -1000.0)
    assert soft.sum() > 0.8 * body.sum()                                     # most of the body
    assert ph.hu[soft].min() >= 0.0 and ph.hu[soft].max() <= 40.0
    fem = ph.hu == 700.0
    assert fem.any() and np.all(Z[fem] < 0.0)                               # caudal half only
    assert np.all(np.abs(np.abs(X[fem]) - 90.0) ** 2 + Y[fem] ** 2 <= 25.0 ** 2 + 1e-6)
    air = body & (ph.hu == -1000.0)
    assert air.any() and np.all(np.abs(Y[air] - 35.0) <= 12.0)              # posterior pocket
    ptv = ph.masks["ptv"]
    np.testing.assert_array_equal(ptv, (X / 30.0) ** 2 + (Y / 25.0) ** 2 + (Z / 35.0) ** 2 <= 1.0)


def test_arc_leaves_follow_the_target_and_jaws_conform(c2):
    pl, lb = c2.plan, c2.machine.leaf_bounds
    assert pl.n_cp == 178
    np.testing.assert_allclose(pl.gantry_deg, np.arange(178) * 360.0 / 178)
    assert pl.mu.min() >= 0.5 and pl.mu.max() <= 2.0 and pl.mu.std() > 0.2
    assert np.all(pl.leaves[..., 0] <= pl.leaves[..., 1])
    moved = 0
    for b in range(pl.n_cp):
        open_rows = []
        for i in range(len(lb) - 1):
            hw, centre = S._ptv_halfwidth(pl.gantry_deg[b], lb[i], lb[i + 1], (30.0, 25.0, 35.0),
                                          (0.0, 0.0, 0.0))
            left, right = pl.leaves[b, i]
            if hw <= 0.0:
                assert left == right == centre                 # rows without target closed
                continue
            assert abs(left - (centre - hw)) <= 10.0 + 1e-9 and abs(right - (centre + hw)) <= 10.0 + 1e-9
            moved += abs(left - (centre - hw)) > 0.1
            if right > left:
                open_rows.append(i)
        assert open_rows
        x_lo = min(pl.leaves[b, i, 0] for i in open_rows)
        x_hi = max(pl.leaves[b, i, 1] for i in open_rows)
        np.testing.assert_allclose(pl.jaws[b], (x_lo, x_hi, lb[open_rows[0]], lb[open_rows[-1] + 1]))
    assert moved > 100                                         # the random walk moves the leaves


def test_beam_model_normalisation():
    m = S.machine_model(1002, r_px=20)
    assert m.t_table.max() == pytest.approx(1.0, abs=1e-15) and m.t_table.min() > 0.0
    assert 0.0 < np.argmax(m.t_table) * m.dz_t < 60.0          # build-up peak within 6 cm
    np.testing.assert_array_less(np.abs(m.beta[:, 0] / np.array([0.75, 0.18, 0.07]) - 1.0), 0.2 + 1e-12)
    assert 0.8 <= m.alpha[0, 0] <= 1.6 and 0.08 <= m.alpha[1, 0] <= 0.25 and 0.015 <= m.alpha[2, 0] <= 0.05
