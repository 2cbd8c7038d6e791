"""Pins of the FP64 oracle against facts fixed outside its own code.

Each test names the paper passage it follows and the independent fact it
checks (a closed form, an invariant, brute force or a library routine), so
that a dropped term, a wrong sign or index, or a transposed operand in the
oracle fails at least one of them.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_18863_gb300 import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _phantom(shape, spacing, hu_fn=None, iso_index=None):
    nz, ny, nx = shape
    sx, sy, sz = spacing
    ci = iso_index or (nx // 2, ny // 2, nz // 2)
    origin = (-ci[0] * sx, -ci[1] * sy, -ci[2] * sz)
    hu = np.zeros(shape, np.float32)
    if hu_fn is not None:
        Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        hu = hu_fn(X, Y, Z).astype(np.float32)
    return S.Phantom(hu=hu, spacing=tuple(spacing), origin=origin)


def _depth_dose_np(machine, z):
    return np.interp(z, np.arange(len(machine.t_table)) * machine.dz_t, machine.t_table)


# --------------------------------------------------------------------------
# Sec. 2.2.2, fractional overlap equation: hand-derived values
# --------------------------------------------------------------------------
def test_overlap_golden_values():
    rows = np.loadtxt(os.path.join(GOLDEN, "overlap_eq.txt"), comments="#")
    for d, lo, hi, D, exp in rows:
        assert O.overlap(d, lo, hi, D) == pytest.approx(exp, abs=1e-15)


def test_projection_golden_values():
    """Sec. 2.2.1: hand-derived projections of leaf and jaw pairs (both use
    the same centre / width projection, with their own w_min and F), and
    MU^ = max(MU, eps)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "projection_eq.txt"), comments="#")
    w = S.small_pelvis(n=(8, 12, 12), n_cp=1, r_px=1)
    for a, b, wmin, F, ea, eb in rows:
        m = S.Machine(**{**w.machine.__dict__, "wmin_leaf": wmin, "f_leaf": F,
                         "wmin_jaw": wmin, "f_jaw": F, "eps_mu": 0.01})
        mod = O.Model(w.phantom, m, w.plan)
        lv = w.plan.leaves.copy()
        lv[0, 7] = (a, b)
        jw = np.array([[a, b, b - 400.0, b + 400.0]])
        lv_p, jw_p, _ = mod.project(0, lv, jw, w.plan.mu)
        assert tuple(lv_p[7]) == pytest.approx((ea, eb), abs=1e-12)
        assert tuple(jw_p[:2]) == pytest.approx((ea, eb), abs=1e-12)
    for mu, exp in ((0.004, 0.01), (-1.0, 0.01), (0.01, 0.01), (2.0, 2.0)):
        _, _, mu_p = mod.project(0, w.plan.leaves, w.plan.jaws, np.array([mu]))
        assert mu_p == exp


def test_overlap_partition_of_unity():
    """T7: sum_a f(u_a; l, r) D = r - l for any l < r inside the lattice."""
    rng = np.random.default_rng(0)
    for D in (2.0, 2.5, 3.0):
        u = (np.arange(-200, 201)) * D
        for _ in range(20):
            lo, hi = np.sort(rng.uniform(-150, 150, 2))
            s = sum(O.overlap(x, lo, hi, D) for x in u) * D
            assert s == pytest.approx(hi - lo, rel=1e-13)


# --------------------------------------------------------------------------
# Sec. 2.2 (HU -> relative electron density): piecewise-linear curve
# --------------------------------------------------------------------------
def test_hu_to_red_knots_and_clamps():
    pts = S.HU_TO_RED
    hu = np.array([-2000, -1000, -500, 0, 500, 1000, 2000, 3000, 5000], float)
    exp = np.array([0.0, 0.0, 0.5, 1.0, 1.3, 1.6, 2.2, 2.8, 2.8])
    np.testing.assert_allclose(O.hu_to_red(hu, pts), exp, rtol=0, atol=1e-15)


# --------------------------------------------------------------------------
# Sec. 2.2.4 (WEPL): slab closed forms, air pocket
# --------------------------------------------------------------------------
def _slab_profile(n):
    # air | water | bone (HU 1000 -> RED 1.6) | air pocket | water
    hu = np.full(n, -1000.0)
    hu[6:14] = 0.0
    hu[14:18] = 1000.0
    hu[18:21] = -1000.0
    hu[21:29] = 0.0
    return hu


@pytest.mark.parametrize("gantry,axis,sign", [(0.0, "y", +1), (180.0, "y", -1),
                                              (90.0, "x", +1), (270.0, "x", -1)])
def test_wepl_slab_closed_form(gantry, axis, sign):
    n, s = 33, 2.0
    prof = _slab_profile(n)
    if axis == "y":
        ph = _phantom((5, n, n), (s, s, s), lambda X, Y, Z: prof[Y])
    else:
        ph = _phantom((5, n, n), (s, s, s), lambda X, Y, Z: prof[X])
    m = S.machine_model(3, r_px=2)
    plan = S.static_field(m, gantry_deg=gantry)
    mod = O.Model(ph, m, plan)
    z = mod.wepl(0)
    lat = mod.lattice
    rho = np.interp(prof, S.HU_TO_RED[:, 0], S.HU_TO_RED[:, 1])
    # exact integral of the piecewise-constant density from outside the grid
    # to each voxel centre along the beam direction
    edges = (np.arange(n + 1) - 0.5 - n // 2) * s          # voxel boundaries, mm from iso
    for k in range(lat["nw"]):
        w = (k - lat["cw"]) * lat["du"]
        pos = sign * w                                      # coordinate along +axis
        if sign > 0:
            seg = np.clip(np.minimum(edges[1:], pos) - edges[:-1], 0, None)
        else:
            seg = np.clip(edges[1:] - np.maximum(edges[:-1], pos), 0, None)
        exp = float((seg * rho).sum())
        assert z[k] == pytest.approx(exp, abs=1e-12), (k, w)
    # the air pocket (voxels 18..20) leaves the depth unchanged across it
    kk = [int(round(lat["cw"] + sign * (i - n // 2))) for i in (18, 19, 20)]
    assert z[kk[0]] == pytest.approx(z[kk[1]], abs=1e-12) == pytest.approx(z[kk[2]], abs=1e-12)


@pytest.mark.parametrize("gantry", [30.0, 45.0, 137.0, 210.0, 300.0])
def test_wepl_increments_in_a_linear_density_field(gantry):
    """Oblique central rays (Sec. 2.2.4).  HU linear in x and y within
    [0, 1000] gives a density linear in position (the calibration curve is
    linear there), and trilinear interpolation reproduces a linear function
    exactly inside the hull of the voxel centres.  So for two consecutive
    beam slices sampled inside that hull the midpoint sum increases by
    dw (rho(p_k) + rho(p_k+1)) / 2, with p_k = iso + w_k e_w and
    e_w = (sin g, cos g, 0).  A wrong step length, ray direction or axis
    assignment at a non-axial angle breaks this."""
    n, s = 41, 2.0
    half = n // 2
    ph = _phantom((3, n, n), (s, s, s), lambda X, Y, Z: 500.0 + 10.0 * (X - half) + 5.0 * (Y - half))
    m = S.machine_model(4, r_px=2)
    mod = O.Model(ph, m, S.static_field(m, gantry_deg=gantry))
    z = mod.wepl(0)
    lat = mod.lattice
    dw = lat["du"]
    g = np.deg2rad(gantry)
    ew = np.array([np.sin(g), np.cos(g)])

    def rho(p):   # RED = 1 + 0.6 HU / 1000, HU = 500 + 5 x + 2.5 y (x, y in mm)
        return 1.0 + 0.6e-3 * (500.0 + 5.0 * p[0] + 2.5 * p[1])

    lim = half * s - 1e-9
    checked = 0
    for k in range(lat["nw"] - 1):
        p0 = (k - lat["cw"]) * dw * ew
        p1 = (k + 1 - lat["cw"]) * dw * ew
        if max(np.abs(p0).max(), np.abs(p1).max()) > lim:
            continue
        exp = dw * 0.5 * (rho(p0) + rho(p1))
        assert z[k + 1] - z[k] == pytest.approx(exp, rel=1e-12), (k, p0)
        checked += 1
    assert checked >= 20


@pytest.mark.parametrize("gantry", [0.0, 23.0, 118.0, 301.0])
def test_wepl_is_the_midpoint_sum_of_trilinear_samples(gantry):
    """Sec. 2.2.4 at any angle in any density: the depth of beam slice k is
    dw (sum_{m<k} rho_m + rho_k / 2), rho_m the density sampled trilinearly
    (zero outside the grid) at the slice centre p_m = iso + w_m e_w on the
    central ray; scipy.ndimage.map_coordinates samples the same points and
    numpy's cumulative sum adds them.  Random HU, an off-centre isocentre
    between voxel centres in z, and sx != sz."""
    from scipy.ndimage import map_coordinates
    n = (9, 17, 15)
    rng = np.random.default_rng(11)
    ph = _phantom(n, (2.0, 2.0, 3.0), lambda X, Y, Z: rng.uniform(-1000.0, 3000.0, X.shape),
                  iso_index=(6, 9, 4))
    red = np.interp(ph.hu.astype(np.float64), S.HU_TO_RED[:, 0], S.HU_TO_RED[:, 1])
    m = S.machine_model(4, r_px=2)
    iso = (1.0, -0.5, 1.2)
    mod = O.Model(ph, m, S.static_field(m, gantry_deg=gantry, iso=iso))
    z = mod.wepl(0)
    lat = mod.lattice
    g = np.deg2rad(gantry)
    w = (np.arange(lat["nw"]) - lat["cw"]) * lat["du"]
    pts = np.stack([np.full_like(w, iso[2]), iso[1] + w * np.cos(g), iso[0] + w * np.sin(g)])
    idx = (pts - np.array(ph.origin[::-1])[:, None]) / np.array(ph.spacing[::-1])[:, None]
    rho = map_coordinates(red, idx, order=1, mode="grid-constant", cval=0.0)
    exp = lat["du"] * (np.concatenate([[0.0], np.cumsum(rho)[:-1]]) + 0.5 * rho)
    np.testing.assert_allclose(z, exp, rtol=1e-12, atol=1e-12)
    assert rho.max() > 0 and (rho == 0).any()      # the ray enters from outside the grid


# --------------------------------------------------------------------------
# T1: open-field water depth dose = cal MU T(z) (SID/d)^2 on the central axis
# (Sec. 2.2.3 inverse square, Sec. 2.2.4 depth, Sec. 2.2.6 kernel unit sum,
#  Sec. 2.2.7 MU weighting)
# --------------------------------------------------------------------------
def test_open_field_depth_dose_closed_form():
    w = S.water_static_64()
    mod = O.Model(w.phantom, w.machine, w.plan)
    D = mod.dose()
    iy = np.arange(64)
    depth = (iy + 0.5) * 2.5
    d = 1000.0 + (iy - 32) * 2.5
    exp = mod.cal * 100.0 * _depth_dose_np(w.machine, depth) * (1000.0 / d) ** 2
    np.testing.assert_allclose(D[32, :, 32], exp, rtol=1e-12)


def _pencil_model(gantry, jaws, sz=3.0, a=0.2, r_px=6):
    n, s = 41, 2.0
    ph = _phantom((41, n, n), (s, s, sz))
    m = S.machine_model(5, r_px=r_px)
    m.alpha = np.zeros((3, 3))
    m.alpha[:, 0] = [a, 1.0, 1.0]
    m.beta = np.zeros((3, 3))
    m.beta[0, 0] = 1.0
    plan = S.static_field(m, gantry_deg=gantry, leaf_half=60.0)
    plan.jaws[0] = jaws
    plan.mu[0] = 1.0
    return O.Model(ph, m, plan), m


def test_depth_dose_is_the_clamped_linear_interpolation_of_the_table():
    """Reading of the depth dose (Sec. 2.4): T(z) interpolates the table
    linearly and is clamped at both ends; numpy's interp (which clamps the
    same way) gives the same values, on a table with a 2.5 mm step."""
    ph = _phantom((5, 9, 9), (2.0, 2.0, 2.0))
    m = S.machine_model(13, r_px=2, n_t=41, dz_t=2.5)
    mod = O.Model(ph, m, S.static_field(m))
    zs = np.concatenate([[-5.0, 0.0, 1e-9], np.random.default_rng(2).uniform(0.0, 100.0, 50),
                         [97.5, 99.99, 100.0, 250.0]])
    exp = np.interp(zs, np.arange(41) * 2.5, m.t_table)
    got = np.array([mod.depth_dose(z) for z in zs])
    np.testing.assert_allclose(got, exp, rtol=1e-14, atol=1e-15)


def test_kernel_parameters_and_unit_sum_over_depth():
    """Sec. 2.2.5 reading: decay rates a_c(z) and raw weights w_c(z) are
    quadratics in depth (numpy's polyval evaluates them), a_c floored at
    1e-4 / mm, raw weights floored at 0 and normalised to sum 1; every
    component is normalised over the (2R+1)^2 window, so the kernel sums to 1
    at every depth, and it depends on the radius only (symmetric under
    p -> -p, q -> -q and, with square pixels, p <-> q)."""
    from numpy.polynomial import polynomial as Pn
    ph = _phantom((5, 9, 9), (2.0, 2.0, 2.0))
    m = S.machine_model(12, r_px=6)
    m.alpha[2] = (0.02, -2e-4, 0.0)           # decays to the floor beyond 100 mm
    m.beta[1] = (0.2, -2e-3, 0.0)             # raw weight clamps to 0 beyond 100 mm
    mod = O.Model(ph, m, S.static_field(m))
    R = m.r_px
    for z in (0.0, 35.0, 99.0, 150.0, 300.0):
        a, w = mod.kernel_params(z)
        a_exp = np.maximum([Pn.polyval(z, m.alpha[c]) for c in range(3)], 1e-4)
        wr = np.maximum([Pn.polyval(z, m.beta[c]) for c in range(3)], 0.0)
        np.testing.assert_allclose(a, a_exp, rtol=1e-14)
        np.testing.assert_allclose(w, wr / wr.sum(), rtol=1e-14)
        K = mod.kernel(z)
        assert K.sum() == pytest.approx(1.0, abs=1e-13)
        np.testing.assert_allclose(K, K[::-1, :], rtol=1e-14)
        np.testing.assert_allclose(K, K[:, ::-1], rtol=1e-14)
        np.testing.assert_allclose(K, K.T, rtol=1e-14)
        assert K[R, R] == K.max() and K[R, R + 1] > K[R + 1, R + 1] > K[R, R + 2]
    assert mod.kernel_params(150.0)[0][2] == 1e-4 and mod.kernel_params(150.0)[1][1] == 0.0


def test_pencil_kernel_shape_and_unit_sum():
    """Sec. 2.2.5/2.2.6: a one-pixel field at the isocentre plane (m = 1, C = 1)
    gives D = cal MU T(z_iso) K(p,q); a single-exponential kernel must then fall
    as exp(-a r) with r = sqrt((p sx)^2 + (q sz)^2) (sx != sz pins the axes)
    and sum to cal MU T over the plane."""
    a, R = 0.2, 6
    mod, m = _pencil_model(0.0, [-1.0, 1.0, -1.5, 1.5], sz=3.0, a=a, r_px=R)
    D = mod.dose()
    plane = D[:, 20, :]                       # iso plane (y index 20), [iz][ix]
    peak = plane[20, 20]
    dz, dx = np.meshgrid(np.arange(41) - 20, np.arange(41) - 20, indexing="ij")
    r = np.sqrt((dx * 2.0) ** 2 + (dz * 3.0) ** 2)
    inside = (np.abs(dx) <= R) & (np.abs(dz) <= R)
    np.testing.assert_allclose(plane[inside] / peak, np.exp(-a * r[inside]), rtol=1e-12)
    assert np.abs(plane[~inside]).max() <= 1e-14 * peak
    T_iso = _depth_dose_np(m, 20.5 * 2.0)
    assert plane.sum() == pytest.approx(m.cal * T_iso, rel=1e-12)


@pytest.mark.parametrize("gantry,peak_at", [(0.0, ("x", 21)), (90.0, ("y", 19)),
                                            (180.0, ("x", 19)), (270.0, ("y", 21))])
def test_beam_axis_orientation(gantry, peak_at):
    """Reading of the geometry (e_u = (cos g, -sin g, 0)): a pixel at u = +2 mm
    lands at x = +2 mm for gantry 0, y = -2 mm for 90, x = -2 mm for 180."""
    mod, _ = _pencil_model(gantry, [1.0, 3.0, -1.5, 1.5])
    D = mod.dose()
    if peak_at[0] == "x":
        line = D[20, 20, :]
    else:
        line = D[20, :, 20]
    assert int(np.argmax(line)) == peak_at[1]


def test_magnification_of_sharp_field_edge():
    """Sec. 2.2.3: with an impulse kernel the dose is cal MU T(z) C(d)
    F_bilinear((SID/d) x_perp): the field appears wider beyond the
    isocentre and narrower before it, scaled by the inverse square."""
    ny = 161
    ph = _phantom((9, ny, 41), (2.5, 2.5, 2.5))
    m = S.machine_model(11, r_px=3, delta_kernel=True)
    plan = S.static_field(m, 0.0, half_x=20.0, half_y=20.0, leaf_half=50.0, mu=1.0)
    mod = O.Model(ph, m, plan)
    D = mod.dose()
    lat = mod.lattice
    nu, cu = lat["nu"], lat["cu"]
    a = np.arange(nu)
    fx_nodes = np.clip(8.5 - np.abs(a - cu), 0.0, 1.0)      # 20 mm edge = half of pixel 8
    for iy in (0, 30, 80, 130, 160):
        w = (iy - 80) * 2.5
        mk = 1000.0 / (1000.0 + w)
        depth = (iy + 0.5) * 2.5
        ix = np.arange(41)
        i = ix - 20 + cu
        exp = m.cal * _depth_dose_np(m, depth) * mk ** 2 * np.interp(mk * (i - cu) + cu, a, fx_nodes)
        np.testing.assert_allclose(D[4, iy, :], exp, rtol=1e-12, atol=1e-14)


# --------------------------------------------------------------------------
# T3-T6: linearity, superposition, leakage, rotation
# --------------------------------------------------------------------------
def test_mu_linearity_and_cp_superposition():
    w = S.small_pelvis(n=(16, 28, 28), n_cp=4, r_px=3)
    mod = O.Model(w.phantom, w.machine, w.plan)
    D = mod.dose()
    np.testing.assert_allclose(mod.dose(mu=2.5 * w.plan.mu), 2.5 * D, rtol=1e-13, atol=1e-15 * D.max())
    acc = np.zeros_like(D)
    for b in range(w.plan.n_cp):
        mu = np.zeros(w.plan.n_cp)
        mu[b] = w.plan.mu[b]
        m2 = S.Machine(**{**w.machine.__dict__, "eps_mu": 0.0})
        acc += O.Model(w.phantom, m2, w.plan).dose(mu=mu)
    np.testing.assert_allclose(acc, D, rtol=0, atol=1e-13 * D.max())


def _water_model(plan_jaws, plan_leaves, gantry=30.0, wmin_leaf=0.5):
    ph = _phantom((21, 33, 33), (2.5, 2.5, 2.5))
    m = S.machine_model(13, r_px=4)
    m.wmin_leaf = wmin_leaf
    plan = S.static_field(m, gantry_deg=gantry)
    plan.jaws[0] = plan_jaws
    plan.leaves[0, :, 0] = plan_leaves[0]
    plan.leaves[0, :, 1] = plan_leaves[1]
    plan.mu[0] = 1.0
    return O.Model(ph, m, plan).dose(), m


def test_abutting_half_fields():
    """T4: f is additive over adjoining intervals, so jaw-made halves sum to
    the full field exactly; leaf-made halves add one extra leakage term
    tau * D(jaw-only field)."""
    full, _ = _water_model([-50, 50, -40, 40], (-60, 60))
    h1, _ = _water_model([-50, 0, -40, 40], (-60, 60))
    h2, _ = _water_model([0, 50, -40, 40], (-60, 60))
    np.testing.assert_allclose(h1 + h2, full, rtol=0, atol=1e-13 * full.max())
    lfull, m = _water_model([-50, 50, -40, 40], (-50, 50))
    l1, _ = _water_model([-50, 50, -40, 40], (-50, 0))
    l2, _ = _water_model([-50, 50, -40, 40], (0, 50))
    np.testing.assert_allclose(l1 + l2 - lfull, m.tau * full, rtol=0, atol=1e-13 * full.max())


def test_closed_mlc_leaves_only_leakage():
    """T5: l = r with w_min = 0 gives f_leaf = 0, so D = tau D(jaw-only)."""
    jaw_only, m = _water_model([-30, 40, -20, 30], (-80, 80), wmin_leaf=0.0)
    closed, _ = _water_model([-30, 40, -20, 30], (10, 10), wmin_leaf=0.0)
    np.testing.assert_allclose(closed, m.tau * jaw_only, rtol=0, atol=1e-14 * jaw_only.max())


def test_rotation_symmetry_90_degrees():
    """T6: on a phantom invariant under 90-degree rotation about the
    isocentre (odd grid, iso on a voxel centre), D_{g+90}(Q x) = D_g(x) with
    Q(x, y) = (y, -x)."""
    n, c = 33, 16

    def hu(X, Y, Z):
        dx, dy = X - c, Y - c
        out = np.where(dx ** 2 + dy ** 2 <= 14 ** 2, 0.0, -1000.0)
        for px, py in ((6, 0), (-6, 0), (0, 6), (0, -6)):
            out = np.where((dx - px) ** 2 + (dy - py) ** 2 <= 4, 800.0, out)
        return out

    ph = _phantom((7, n, n), (2.5, 2.5, 2.5), hu)
    m = S.machine_model(17, r_px=4)
    rng = np.random.default_rng(3)
    out = []
    for g in (30.0, 120.0):
        plan = S.static_field(m, gantry_deg=g)
        plan.jaws[0] = [-10.0, 25.0, -15.0, 10.0]
        plan.leaves[0, :, 0] = rng.uniform(-15, 0, m.n_pairs) if not out else plan_l0
        plan.leaves[0, :, 1] = rng.uniform(2, 20, m.n_pairs) if not out else plan_l1
        plan_l0, plan_l1 = plan.leaves[0, :, 0].copy(), plan.leaves[0, :, 1].copy()
        plan.mu[0] = 1.0
        out.append(O.Model(ph, m, plan).dose())
    A, B = out
    iy, ix = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    np.testing.assert_allclose(B[:, 2 * c - ix, iy], A[:, iy, ix], rtol=0, atol=1e-12 * A.max())


def test_fluence_area_closed_forms():
    """T7: jaws only: sum F dA = jaw area; leaves inside pixel-aligned jaws:
    sum F dA = tau A_jaw + (1 - tau) sum_i (r_i - l_i) |strip_i within the y jaws|.
    Rows: partition of unity of the leaf strips inside the MLC span."""
    ph = _phantom((170, 9, 41), (2.5, 2.5, 2.5))   # u lattice reaches +-55 mm
    m = S.machine_model(19, r_px=2)
    plan = S.static_field(m)
    mod = O.Model(ph, m, plan)
    du, dv = mod.lattice["du"], mod.lattice["dv"]
    lv_open = np.stack([np.full(m.n_pairs, -100.0), np.full(m.n_pairs, 100.0)], 1)
    jw = np.array([-13.3, 7.9, -21.7, 34.1])
    F = mod.fluence(lv_open, jw)
    assert F.sum() * du * dv == pytest.approx((jw[1] - jw[0]) * (jw[3] - jw[2]), rel=1e-13)
    # leaf-defined aperture, pixel-aligned jaws (edges at +-1.25 + 2.5 k)
    jw2 = np.array([-26.25, 26.25, -31.25, 18.75])
    rng = np.random.default_rng(5)
    lv = np.stack([rng.uniform(-20, -1, m.n_pairs), rng.uniform(1, 20, m.n_pairs)], 1)
    F2 = mod.fluence(lv, jw2)
    lb = m.leaf_bounds
    strip = np.clip(np.minimum(lb[1:], jw2[3]) - np.maximum(lb[:-1], jw2[2]), 0, None)
    a_jaw = (jw2[1] - jw2[0]) * (jw2[3] - jw2[2])
    exp = m.tau * a_jaw + (1 - m.tau) * ((lv[:, 1] - lv[:, 0]) * strip).sum()
    assert F2.sum() * du * dv == pytest.approx(exp, rel=1e-13)
    # leaf strips tile the MLC span: with tau = 0 and all leaves open, F = 1
    # on every row inside +-200 mm and 0 outside it
    m0 = S.Machine(**{**m.__dict__, "tau": 0.0})
    mod0 = O.Model(ph, m0, plan)
    F3 = mod0.fluence(lv_open, np.array([-50.0, 50.0, -300.0, 300.0]))
    v = (np.arange(mod0.lattice["nv"]) - mod0.lattice["cv"]) * dv
    col = F3[:, int(mod0.lattice["cu"])]
    inside = np.abs(v) < 200.0 - dv / 2
    outside = np.abs(v) > 200.0 + dv / 2
    np.testing.assert_allclose(col[inside], 1.0, rtol=0, atol=1e-14)
    np.testing.assert_allclose(col[outside], 0.0, rtol=0, atol=0)


# --------------------------------------------------------------------------
# T8: brute force on a 16^3 grid
# --------------------------------------------------------------------------
def test_convolution_is_the_same_size_zero_padded_convolution_per_slice():
    """Sec. 2.2.6: beam slice k's lateral dose is T(z_k) times the 'same'-size
    2-D convolution, zero padded at the lattice edge, of that slice's fluence
    with that slice's kernel; scipy.signal.convolve2d computes it
    independently.  The lattice has du != dv (3 and 2 mm), the fluence is
    random, non-negative and fills the lattice to its edges, some slices are
    empty, and the depths change the kernel from slice to slice."""
    from scipy.signal import convolve2d
    ph = _phantom((6, 9, 9), (3.0, 3.0, 2.0))
    m = S.machine_model(8, r_px=4)
    mod = O.Model(ph, m, S.static_field(m))
    nw, nv, nu = mod.vol_shape()
    R = m.r_px
    rng = np.random.default_rng(5)
    Phi = rng.random((nw, nv, nu))
    Phi[::4] = 0.0
    z = np.linspace(5.0, 250.0, nw)
    for brute in (False, True):
        got = mod.conv(z, Phi, brute=brute)
        for k in range(nw):
            K = mod.kernel(z[k])                 # [u offset][v offset]
            assert K[R, R + 1] > K[R + 1, R]     # a 2 mm step (v) is nearer than 3 mm (u)
            exp = mod.depth_dose(z[k]) * convolve2d(Phi[k], K.T, mode="same")
            np.testing.assert_allclose(got[k], exp, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("gantry", [0.0, 37.0, 251.0])
def test_gather_is_trilinear_sampling_with_zero_outside(gantry):
    """Sec. 2.2.7: voxel x receives the beam-frame dose sampled trilinearly at
    its beam coordinates (u, v, w) = ((x - iso).e_u, (x - iso).e_v,
    (x - iso).e_w) in lattice units; scipy.ndimage.map_coordinates (order 1,
    zero outside) samples the same points independently.  The isocentre is
    off the grid centre and sx != sz."""
    from scipy.ndimage import map_coordinates
    ph = _phantom((7, 12, 10), (3.0, 3.0, 2.0), iso_index=(3, 7, 2))
    m = S.machine_model(8, r_px=2)
    mod = O.Model(ph, m, S.static_field(m, gantry_deg=gantry))
    lat = mod.lattice
    Dp = np.random.default_rng(6).random(mod.vol_shape())
    got = mod.gather(0, Dp, scale=1.7)
    nz, ny, nx = ph.hu.shape
    Z, Y, X = np.meshgrid(*(o + s * np.arange(n) for o, s, n in
                            zip(ph.origin[::-1], ph.spacing[::-1], (nz, ny, nx))), indexing="ij")
    g = np.deg2rad(gantry)
    u = X * np.cos(g) - Y * np.sin(g)
    w = X * np.sin(g) + Y * np.cos(g)
    coords = np.stack([w / lat["du"] + lat["cw"], Z / lat["dv"] + lat["cv"], u / lat["du"] + lat["cu"]])
    exp = 1.7 * map_coordinates(Dp, coords.reshape(3, -1), order=1, mode="grid-constant",
                                cval=0.0).reshape(nz, ny, nx)
    np.testing.assert_allclose(got, exp, rtol=1e-12, atol=1e-14)


def test_fluence_volume_is_magnified_bilinear_sampling():
    """Sec. 2.2.3: Phi_k at lattice point (i, j) is (SID/d_k)^2 times the
    fluence map sampled bilinearly at the iso-plane point (SID/d_k) times the
    point's offset from the central axis, zero outside the map, with
    d_k = SID + w_k; scipy.ndimage.map_coordinates (order 1, zero outside)
    samples it independently.  A short SID makes m range well above and below
    1, so samples fall outside the map near its edges."""
    from scipy.ndimage import map_coordinates
    ph = _phantom((5, 11, 11), (3.0, 3.0, 2.0))
    m = S.machine_model(8, r_px=2)
    m.sid = 120.0
    mod = O.Model(ph, m, S.static_field(m))
    lat = mod.lattice
    F = np.random.default_rng(7).random((lat["nv"], lat["nu"]))
    Phi = mod.magnify(F)
    jj, ii = np.meshgrid(np.arange(lat["nv"]), np.arange(lat["nu"]), indexing="ij")
    for k in range(lat["nw"]):
        mk = m.sid / (m.sid + (k - lat["cw"]) * lat["du"])
        coords = np.stack([mk * (jj - lat["cv"]) + lat["cv"], mk * (ii - lat["cu"]) + lat["cu"]])
        exp = mk ** 2 * map_coordinates(F, coords.reshape(2, -1), order=1, mode="grid-constant",
                                        cval=0.0).reshape(F.shape)
        np.testing.assert_allclose(Phi[k], exp, rtol=1e-12, atol=1e-14)


def test_brute_force_16cube():
    w = S.small_pelvis(n=(16, 16, 16), spacing=4.0, n_cp=3, r_px=3, ptv_radii=(12.0, 10.0, 12.0))
    mod = O.Model(w.phantom, w.machine, w.plan)
    fast = mod.dose()
    brute = mod.dose(brute=True)
    assert fast.max() > 0
    np.testing.assert_allclose(fast, brute, rtol=0, atol=1e-12 * brute.max())
