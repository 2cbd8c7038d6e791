"""Seeded synthetic workloads shaped like the paper's prostate VMAT cases.

The paper evaluates on clinical prostate CTs (Sec. 2.5: Gold Atlas and a
private cohort; 105x224x224 grids, 180 control points, Sec. 3.4) which are not
available here.  This module builds seeded stand-ins with the same shapes and
structure: water phantoms for the commissioning-style checks (Sec. 2.5.2) and
a pelvis-like phantom (body ellipse, femoral heads, rectal air pocket, PTV,
bladder, rectum) with VMAT arcs whose MLC apertures follow the target.

It holds no dose arithmetic: only phantom geometry, machine constants and
random delivery parameters.  Both the CUDA path and the CPU oracle consume the
same objects, so the two sides always see identical inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

# HU -> relative electron density calibration points (HU, RED); a stand-in
# for the commissioned curve of Sec. 2.4.
HU_TO_RED = np.array([[-1000.0, 0.0], [0.0, 1.0], [1000.0, 1.6], [3000.0, 2.8]])


def leaf_bounds_60() -> np.ndarray:
    """Leaf-pair boundaries (mm at the isocentre plane) of a 60-pair MLC:
    10 x 10 mm outer pairs on each side and 40 x 5 mm central pairs."""
    outer_lo = -200.0 + 10.0 * np.arange(10)
    central = -100.0 + 5.0 * np.arange(40)
    outer_hi = 100.0 + 10.0 * np.arange(11)
    return np.concatenate([outer_lo, central, outer_hi]).astype(np.float64)


@dataclass
class Machine:
    """Beam-model constants (Sec. 2.2 and Sec. 2.4 list what is commissioned)."""
    r_px: int
    alpha: np.ndarray            # (3,3) kernel decay polynomials, 1/mm
    beta: np.ndarray             # (3,3) raw kernel weight polynomials
    t_table: np.ndarray          # depth-dose table at dz_t steps
    dz_t: float = 1.0
    sid: float = 1000.0
    leaf_bounds: np.ndarray = field(default_factory=leaf_bounds_60)
    tau: float = 0.002
    wmin_leaf: float = 0.5
    wmin_jaw: float = 0.5
    f_leaf: float = 150.0
    f_jaw: float = 200.0
    eps_mu: float = 0.01
    # output factor (Sec. 2.4); None: calibrated on the dose grid's pitch so
    # that cal_ref_mu MU of the 10 x 10 cm reference field give cal_ref_gy Gy
    # at 10 cm depth in water (the engine and the oracle each compute it)
    cal: Optional[float] = 1.0
    cal_ref_mu: float = 100.0
    cal_ref_gy: float = 1.0
    ste: int = 1
    # fluence corrections of Sec. 2.2.2 beyond transmission: source penumbra
    # FWHM along leaf travel (u) and across leaf pairs / Y jaws (v), mm (0 =
    # off), and the off-axis profile coefficients c0 + c1 r + c2 r^2
    pen_fwhm_u: float = 0.0
    pen_fwhm_v: float = 0.0
    off_axis: tuple = (1.0, 0.0, 0.0)
    collimator_deg: float = 0.0   # collimator angle of every control point

    @property
    def n_pairs(self) -> int:
        return len(self.leaf_bounds) - 1


@dataclass
class Phantom:
    hu: np.ndarray               # (nz, ny, nx) float32
    spacing: tuple               # (sx, sy, sz) mm
    origin: tuple                # centre of voxel (0,0,0), mm
    hu_to_red: np.ndarray = field(default_factory=lambda: HU_TO_RED.copy())
    masks: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.hu.shape


@dataclass
class Plan:
    gantry_deg: np.ndarray       # (n_cp,)
    iso: np.ndarray              # (3,) mm
    leaves: np.ndarray           # (n_cp, n_pairs, 2) left/right, mm
    jaws: np.ndarray             # (n_cp, 4) x-, x+, y-, y+, mm
    mu: np.ndarray               # (n_cp,)

    @property
    def n_cp(self) -> int:
        return len(self.gantry_deg)


@dataclass
class Workload:
    name: str
    phantom: Phantom
    machine: Machine
    plan: Plan


def machine_model(seed: int, r_px: int, n_t: int = 501, dz_t: float = 1.0,
                  delta_kernel: bool = False) -> Machine:
    """Seeded beam model.

    Depth dose: a build-up/attenuation curve T(z) = [T0 + (1-T0)(1-exp(-z/b))]
    exp(-mu z), normalised to a maximum of 1, tabulated every dz_t mm.
    Lateral kernel: three radial exponentials with decay rates near
    (1.2, 0.15, 0.03)/mm and weights near (0.75, 0.18, 0.07), both varying
    slowly with depth.  With delta_kernel=True the first component is made so
    narrow (50/mm) and dominant that the kernel is a unit impulse to FP64
    precision; used by the pins that isolate the geometry.
    """
    rng = np.random.default_rng(seed)
    beta_b = rng.uniform(8.0, 15.0)
    mu_att = rng.uniform(0.004, 0.006)
    t0 = rng.uniform(0.3, 0.5)
    z = np.arange(n_t) * dz_t
    t = (t0 + (1 - t0) * (1 - np.exp(-z / beta_b))) * np.exp(-mu_att * z)
    t = t / t.max()
    a0 = np.array([rng.uniform(0.8, 1.6), rng.uniform(0.08, 0.25), rng.uniform(0.015, 0.05)])
    alpha = np.zeros((3, 3))
    alpha[:, 0] = a0
    alpha[:, 1] = a0 * rng.uniform(-0.3, 0.3, 3) / 400.0
    alpha[:, 2] = a0 * rng.uniform(-0.05, 0.05, 3) / 400.0 ** 2
    w0 = np.array([0.75, 0.18, 0.07]) * rng.uniform(0.8, 1.2, 3)
    beta = np.zeros((3, 3))
    beta[:, 0] = w0
    beta[:, 1] = w0 * rng.uniform(-0.2, 0.2, 3) / 400.0
    if delta_kernel:
        alpha = np.zeros((3, 3))
        alpha[:, 0] = [50.0, 1.0, 1.0]
        beta = np.zeros((3, 3))
        beta[0, 0] = 1.0
    return Machine(r_px=int(r_px), alpha=alpha, beta=beta, t_table=t, dz_t=dz_t)


def with_corrections(m: Machine, seed: int, pen=(4.0, 6.0), collimator_deg: float = 0.0) -> Machine:
    """Seeded source-penumbra widths (FWHM, mm) and a mildly horned off-axis
    profile (a few per cent over 100 mm), as commissioned beam models have,
    and the given collimator angle."""
    rng = np.random.default_rng(seed)
    m.pen_fwhm_u = float(pen[0] * rng.uniform(0.8, 1.2))
    m.pen_fwhm_v = float(pen[1] * rng.uniform(0.8, 1.2))
    m.off_axis = (1.0, float(rng.uniform(1e-4, 3e-4)), float(rng.uniform(-2e-6, 2e-6)))
    m.collimator_deg = float(collimator_deg)
    return m


def water_phantom(n=(64, 64, 64), spacing=(2.5, 2.5, 2.5), hu=0.0) -> Phantom:
    """Uniform phantom; voxel index n//2 sits at 0 mm on every axis."""
    nz, ny, nx = n
    sx, sy, sz = spacing
    origin = (-(nx // 2) * sx, -(ny // 2) * sy, -(nz // 2) * sz)
    return Phantom(hu=np.full(n, hu, np.float32), spacing=tuple(spacing), origin=origin)


def _coords(ph: Phantom):
    nz, ny, nx = ph.hu.shape
    x = (ph.origin[0] + ph.spacing[0] * np.arange(nx)).astype(np.float32)
    y = (ph.origin[1] + ph.spacing[1] * np.arange(ny)).astype(np.float32)
    z = (ph.origin[2] + ph.spacing[2] * np.arange(nz)).astype(np.float32)
    return np.meshgrid(z, y, x, indexing="ij")


def pelvis_phantom(n=(160, 256, 256), spacing=(2.0, 2.0, 2.0), seed=0,
                   ptv_radii=(30.0, 25.0, 35.0), ptv_offset=(0.0, 0.0, 0.0)) -> Phantom:
    """Synthetic pelvis: water-like body ellipse (HU 0..40 smooth field),
    femoral heads (HU 700), rectal air pocket (HU -1000), PTV/bladder/rectum
    masks.  Axes: x left-right, y anterior(-)/posterior(+), z caudal(-)/cranial(+)."""
    rng = np.random.default_rng(seed)
    ph = water_phantom(n, spacing, hu=-1000.0)
    Z, Y, X = _coords(ph)
    body = (X / 180.0) ** 2 + (Y / 120.0) ** 2 <= 1.0
    field_ = np.zeros_like(X)
    for _ in range(4):
        kx, ky, kz = rng.uniform(0.005, 0.03, 3)
        phs = rng.uniform(0, 2 * np.pi, 3)
        field_ += np.cos(kx * X + phs[0]) * np.cos(ky * Y + phs[1]) * np.cos(kz * Z + phs[2])
    field_ = 20.0 + 5.0 * field_          # within [0, 40]
    hu = np.where(body, field_, -1000.0)
    for sgn in (-1.0, 1.0):
        fem = ((X - sgn * 90.0) ** 2 + Y ** 2 <= 25.0 ** 2) & (Z < 0.0)
        hu = np.where(fem & body, 700.0, hu)
    air = ((X / 15.0) ** 2 + ((Y - 35.0) / 12.0) ** 2 + (Z / 25.0) ** 2) <= 1.0
    hu = np.where(air, -1000.0, hu)
    ph.hu = hu.astype(np.float32)
    ox, oy, oz = ptv_offset
    rx, ry, rz = ptv_radii
    ph.masks["ptv"] = (((X - ox) / rx) ** 2 + ((Y - oy) / ry) ** 2 + ((Z - oz) / rz) ** 2) <= 1.0
    ph.masks["bladder"] = (((X / 35.0) ** 2 + ((Y + 30.0) / 25.0) ** 2
                            + ((Z - 30.0) / 30.0) ** 2) <= 1.0) & ~ph.masks["ptv"]
    ph.masks["rectum"] = ((X ** 2 + (Y - 35.0) ** 2 <= 15.0 ** 2) & (np.abs(Z) <= 40.0)
                          & ~ph.masks["ptv"])
    ph.masks["body"] = body
    return ph


def _ptv_halfwidth(phi_deg, v_lo, v_hi, radii, offset):
    """Half-width along the leaf-travel direction of the (undiverged) PTV
    ellipsoid cross-section inside the leaf strip [v_lo, v_hi]; 0 if none.
    Leaf travel is (cos g, -sin g, 0) in the patient frame, leaf pairs are
    stacked along z."""
    rx, ry, rz = radii
    zc = offset[2]
    lo, hi = v_lo - zc, v_hi - zc
    if hi <= -rz or lo >= rz:
        return 0.0, 0.0
    zn = 0.0 if lo <= 0.0 <= hi else min(abs(lo), abs(hi))
    s = np.sqrt(max(0.0, 1.0 - (zn / rz) ** 2))
    g = np.deg2rad(phi_deg)
    hw = s * np.sqrt((rx * np.cos(g)) ** 2 + (ry * np.sin(g)) ** 2)
    centre = offset[0] * np.cos(g) - offset[1] * np.sin(g)
    return hw, centre


def arc_plan(machine: Machine, gantry_deg: np.ndarray, seed: int,
             ptv_radii=(30.0, 25.0, 35.0), ptv_offset=(0.0, 0.0, 0.0),
             iso=(0.0, 0.0, 0.0), margin=10.0, mu_range=(0.5, 2.0)) -> Plan:
    """VMAT arc whose leaves follow the target: per leaf a smooth random walk
    (Gaussian steps of 2 mm, 5-CP moving average) around the target's
    beam's-eye-view edge, clipped to that edge +-margin, with left <= right;
    rows without target are closed at the target centre; jaws conform to the
    union of open rows; MU uniform in mu_range."""
    rng = np.random.default_rng(seed)
    n_cp = len(gantry_deg)
    lb = machine.leaf_bounds
    npairs = len(lb) - 1
    leaves = np.zeros((n_cp, npairs, 2))
    jaws = np.zeros((n_cp, 4))
    walk = rng.normal(0.0, 2.0, size=(n_cp + 4, npairs, 2)).cumsum(axis=0)
    kern = np.ones(5) / 5.0
    smooth = np.stack([np.stack([np.convolve(walk[:, i, s], kern, mode="valid")
                                 for s in range(2)], -1) for i in range(npairs)], 1)
    smooth = smooth - smooth.mean(axis=0, keepdims=True)
    for b in range(n_cp):
        lo_open, hi_open, u_lo, u_hi = None, None, np.inf, -np.inf
        for i in range(npairs):
            hw, centre = _ptv_halfwidth(gantry_deg[b], lb[i], lb[i + 1], ptv_radii, ptv_offset)
            if hw <= 0.0:
                leaves[b, i] = (centre, centre)
                continue
            left = np.clip(centre - hw + smooth[b, i, 0], centre - hw - margin, centre - hw + margin)
            right = np.clip(centre + hw + smooth[b, i, 1], centre + hw - margin, centre + hw + margin)
            if left > right:
                left = right = 0.5 * (left + right)
            leaves[b, i] = (left, right)
            if right > left:
                lo_open = lb[i] if lo_open is None else lo_open
                hi_open = lb[i + 1]
                u_lo, u_hi = min(u_lo, left), max(u_hi, right)
        if lo_open is None:
            jaws[b] = (-1.0, 1.0, -1.0, 1.0)
        else:
            jaws[b] = (u_lo, u_hi, lo_open, hi_open)
    mu = rng.uniform(mu_range[0], mu_range[1], n_cp)
    return Plan(gantry_deg=np.asarray(gantry_deg, np.float64), iso=np.asarray(iso, np.float64),
                leaves=leaves, jaws=jaws, mu=mu)


def static_field(machine: Machine, gantry_deg=0.0, half_x=50.0, half_y=50.0, leaf_half=None,
                 mu=100.0, iso=(0.0, 0.0, 0.0)) -> Plan:
    """One control point: jaws +-half_x / +-half_y, all leaf pairs at
    +-leaf_half (default: the x jaw)."""
    lh = half_x if leaf_half is None else leaf_half
    npairs = machine.n_pairs
    leaves = np.zeros((1, npairs, 2))
    leaves[0, :, 0] = -lh
    leaves[0, :, 1] = lh
    return Plan(gantry_deg=np.array([float(gantry_deg)]), iso=np.asarray(iso, np.float64),
                leaves=leaves, jaws=np.array([[-half_x, half_x, -half_y, half_y]]),
                mu=np.array([float(mu)]))


def arc_angles(n_cp: int, reverse=False) -> np.ndarray:
    a = np.arange(n_cp) * 360.0 / n_cp
    return a[::-1].copy() if reverse else a


# ----------------------------------------------------------------------------
# Named workloads.  Sizes follow the three dose configurations: a static
# 10x10 cm field on a 64^3 water phantom at 2.5 mm (kernel radius 2 cm); a
# 178-CP arc on a 128x128x96 pelvis at 3 mm (4 cm); a two-arc 2x178-CP plan on
# a 256x256x160 pelvis at 2 mm (2, 4 or 8 cm).  `scale` shrinks the grid and CP
# count for tests.
# ----------------------------------------------------------------------------
def water_static_64(seed=1000) -> Workload:
    m = machine_model(seed, r_px=8)
    m.cal = None   # calibrated to the reference conditions of Sec. 2.4
    ph = water_phantom((64, 64, 64), (2.5, 2.5, 2.5))
    return Workload("water64_static_10x10", ph, m, static_field(m))


def pelvis_arc_128(seed=1001, n_cp=178, r_cm=4.0) -> Workload:
    m = machine_model(seed, r_px=int(round(r_cm * 10.0 / 3.0)))
    m.cal = None   # calibrated to the reference conditions of Sec. 2.4
    ph = pelvis_phantom((96, 128, 128), (3.0, 3.0, 3.0), seed=seed)
    pl = arc_plan(m, arc_angles(n_cp), seed=seed)
    return Workload(f"pelvis128x128x96_arc{n_cp}_R{r_cm:g}cm", ph, m, pl)


def pelvis_two_arc_256(seed=1002, n_cp_arc=178, r_cm=4.0, shape=(160, 256, 256),
                       spacing=2.0) -> Workload:
    m = machine_model(seed, r_px=int(round(r_cm * 10.0 / spacing)))
    m.cal = None   # calibrated to the reference conditions of Sec. 2.4
    ph = pelvis_phantom(shape, (spacing,) * 3, seed=seed)
    ang = np.concatenate([arc_angles(n_cp_arc), arc_angles(n_cp_arc, reverse=True)])
    pl = arc_plan(m, ang, seed=seed)
    nz, ny, nx = shape
    return Workload(f"pelvis{nx}x{ny}x{nz}_2x{n_cp_arc}cp_R{r_cm:g}cm", ph, m, pl)


def paper_table_arc(seed=1006) -> Workload:
    """The shape of the paper's timing table (Sec. 3.4): a 180-CP arc on a
    105 x 224 x 224 grid with a 55-pixel lateral kernel (R = 27 px); voxel
    size 2.5 mm in-plane, 3 mm between slices (not stated there)."""
    m = machine_model(seed, r_px=27)
    m.cal = None   # calibrated to the reference conditions of Sec. 2.4
    ph = pelvis_phantom((105, 224, 224), (2.5, 2.5, 3.0), seed=seed)
    pl = arc_plan(m, arc_angles(180), seed=seed)
    return Workload("pelvis224x224x105_arc180_K55", ph, m, pl)


def small_pelvis(seed=7, n=(24, 40, 40), spacing=3.0, n_cp=6, r_px=4, ptv_radii=(20.0, 15.0, 18.0)):
    """Reduced pelvis case for parity tests (several CTA tiles, ragged edges)."""
    m = machine_model(seed, r_px=r_px)
    ph = pelvis_phantom(n, (spacing,) * 3, seed=seed, ptv_radii=ptv_radii)
    pl = arc_plan(m, arc_angles(n_cp) + 7.5, seed=seed, ptv_radii=ptv_radii)
    return Workload(f"pelvis{n[2]}x{n[1]}x{n[0]}_{n_cp}cp_R{r_px}px", ph, m, pl)


def uneven_batch(n_plans=32, seed=1003, r_cm=4.0):
    """Plans of uneven size for the batched launch: grid axes uniform in
    [96, 256] voxels (z capped at 160), 2-3 mm voxels, arcs of 90-356 control
    points (two arcs above 178), kernel radius r_cm."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(n_plans):
        nx, ny = (int(v) for v in rng.integers(96, 257, 2))
        nz = int(rng.integers(96, 161))
        sp = float(rng.choice([2.0, 2.5, 3.0]))
        n_cp = int(rng.integers(90, 357))
        m = machine_model(seed + 10 * q, r_px=int(round(r_cm * 10.0 / sp)))
        m.cal = None   # calibrated to the reference conditions of Sec. 2.4
        ph = pelvis_phantom((nz, ny, nx), (sp, sp, sp), seed=seed + q)
        if n_cp > 178:
            ang = np.concatenate([arc_angles(n_cp // 2), arc_angles(n_cp - n_cp // 2, reverse=True)])
        else:
            ang = arc_angles(n_cp)
        pl = arc_plan(m, ang, seed=seed + q)
        out.append(Workload(f"plan{q}_{nx}x{ny}x{nz}_{sp:g}mm_{n_cp}cp", ph, m, pl))
    return out


def warmstart_case(seed: int, n=(32, 56, 80), spacing=5.0, n_cp=36, machine_seed=1004,
                   r_px=4) -> Workload:
    """Phantoms of the learned warm start: seeded pelvis with a PTV ellipsoid of
    radii uniform in [20, 40] mm per axis at an offset uniform in [-15, 15] mm
    per axis, one machine (kernel radius 2 cm at 5 mm voxels) and an n_cp arc
    whose jaws conform to the target."""
    rng = np.random.default_rng(seed)
    radii = tuple(float(r) for r in rng.uniform(20.0, 40.0, 3))
    offset = tuple(float(o) for o in rng.uniform(-15.0, 15.0, 3))
    m = machine_model(machine_seed, r_px=r_px)
    ph = pelvis_phantom(n, (spacing,) * 3, seed=seed, ptv_radii=radii, ptv_offset=offset)
    pl = arc_plan(m, arc_angles(n_cp), seed=seed, ptv_radii=radii, ptv_offset=offset)
    nz, ny, nx = n
    return Workload(f"warmstart{nx}x{ny}x{nz}_arc{n_cp}_seed{seed}", ph, m, pl)
