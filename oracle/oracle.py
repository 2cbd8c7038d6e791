"""ctypes wrapper of the FP64 C oracle (pdrt_oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and the CPU-baseline
leg of bench.py use it; the product path never imports it.  It shares no code
with the CUDA library: the only thing both sides share is the seeded input
module paper_2512_18863_gb300.synth, which holds no dose arithmetic.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdrt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

D = C.c_double
PD = C.POINTER(C.c_double)


class OrcGrid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("sx", D), ("sy", D), ("sz", D), ("origin", D * 3), ("red", PD)]


class OrcPlan(C.Structure):
    _fields_ = [("n_cp", C.c_int), ("gantry_deg", PD), ("iso", D * 3), ("sid", D),
                ("n_pairs", C.c_int), ("leaf_bounds", PD), ("tau", D),
                ("wmin_leaf", D), ("wmin_jaw", D), ("f_leaf", D), ("f_jaw", D),
                ("eps_mu", D), ("r_px", C.c_int), ("alpha", (D * 3) * 3), ("beta", (D * 3) * 3),
                ("n_t", C.c_int), ("dz_t", D), ("t_table", PD), ("cal", D), ("ste", C.c_int),
                ("pen_fwhm_u", D), ("pen_fwhm_v", D), ("oap", D * 3),
                ("coll_deg", D)]


class OrcLattice(C.Structure):
    _fields_ = [("nu", C.c_int), ("nv", C.c_int), ("nw", C.c_int),
                ("cu", D), ("cv", D), ("cw", D), ("du", D), ("dv", D)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, ISO C11: no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_dose.restype = C.c_int
            L.orc_dose_grad.restype = C.c_int
            L.orc_beam_dose.restype = C.c_int
            L.orc_overlap.restype = D
            L.orc_overlap.argtypes = [D, D, D, D]
            L.orc_depth_dose.restype = D
            L.orc_hu_to_red_1.restype = D
            L.orc_calibrate.restype = C.c_int
            L.orc_num_threads.restype = C.c_int
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(PD)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _plan_struct(machine, gantry, iso, cal):
    """OrcPlan of a machine + gantry angles (the arrays it points to are kept
    on the returned structure)."""
    pl = OrcPlan()
    pl._keep = (gantry, _f64(machine.leaf_bounds), _f64(machine.t_table))
    pl.n_cp = len(gantry)
    pl.gantry_deg = _p(gantry)
    pl.iso[:] = list(_f64(iso))
    pl.sid = machine.sid
    pl.n_pairs = len(pl._keep[1]) - 1
    pl.leaf_bounds = _p(pl._keep[1])
    pl.tau, pl.wmin_leaf, pl.wmin_jaw = machine.tau, machine.wmin_leaf, machine.wmin_jaw
    pl.f_leaf, pl.f_jaw, pl.eps_mu = machine.f_leaf, machine.f_jaw, machine.eps_mu
    pl.r_px = int(machine.r_px)
    for c in range(3):
        for k in range(3):
            pl.alpha[c][k] = float(machine.alpha[c][k])
            pl.beta[c][k] = float(machine.beta[c][k])
    pl.n_t = len(pl._keep[2])
    pl.dz_t = machine.dz_t
    pl.t_table = _p(pl._keep[2])
    pl.cal = float(cal)
    pl.ste = int(machine.ste)
    pl.pen_fwhm_u = float(getattr(machine, "pen_fwhm_u", 0.0))
    pl.pen_fwhm_v = float(getattr(machine, "pen_fwhm_v", 0.0))
    pl.oap[:] = [float(x) for x in getattr(machine, "off_axis", (1.0, 0.0, 0.0))]
    pl.coll_deg = float(getattr(machine, "collimator_deg", 0.0))
    return pl


class Model:
    """Holds the ctypes structures (and the arrays they point to) for one
    phantom + machine + gantry-angle set."""

    def __init__(self, phantom, machine, plan):
        self.phantom, self.machine, self.plan = phantom, machine, plan
        hu = _f64(phantom.hu).ravel()
        pts = _f64(phantom.hu_to_red).ravel()
        red = np.empty_like(hu)
        lib().orc_hu_to_red(_p(hu), C.c_long(hu.size), _p(pts), C.c_int(len(pts) // 2), _p(red))
        self.red = red.reshape(phantom.hu.shape)
        g = OrcGrid()
        g.nz, g.ny, g.nx = phantom.hu.shape
        g.sx, g.sy, g.sz = phantom.spacing
        g.origin[:] = phantom.origin
        g.red = _p(self.red)
        self.grid = g
        self._gantry = _f64(plan.gantry_deg)
        cal = machine.cal
        if cal is None:   # calibrate to the reference conditions of Sec. 2.4
            cal = calibrate(machine, phantom.spacing[0], phantom.spacing[2])
        self.cal = float(cal)
        pl = _plan_struct(machine, self._gantry, plan.iso, cal=self.cal)
        self.cplan = pl
        L = OrcLattice()
        lib().orc_lattice_of(C.byref(g), C.byref(pl), C.byref(L))
        self.lat = L

    # --- lattice ----------------------------------------------------------
    @property
    def lattice(self):
        L = self.lat
        return dict(nu=L.nu, nv=L.nv, nw=L.nw, cu=L.cu, cv=L.cv, cw=L.cw, du=L.du, dv=L.dv)

    def vol_shape(self):
        return (self.lat.nw, self.lat.nv, self.lat.nu)

    # --- whole model --------------------------------------------------------
    def dose(self, leaves=None, jaws=None, mu=None, brute=False):
        leaves = _f64(self.plan.leaves if leaves is None else leaves)
        jaws = _f64(self.plan.jaws if jaws is None else jaws)
        mu = _f64(self.plan.mu if mu is None else mu)
        out = np.zeros(self.phantom.hu.shape, np.float64)
        rc = lib().orc_dose(C.byref(self.grid), C.byref(self.cplan), _p(leaves), _p(jaws),
                            _p(mu), _p(out), C.c_int(1 if brute else 0))
        if rc:
            raise RuntimeError(f"orc_dose failed: {rc}")
        return out

    def dose_grad(self, gdose, leaves=None, jaws=None, mu=None):
        leaves = _f64(self.plan.leaves if leaves is None else leaves)
        jaws = _f64(self.plan.jaws if jaws is None else jaws)
        mu = _f64(self.plan.mu if mu is None else mu)
        g = _f64(gdose)
        dl = np.zeros_like(leaves)
        dj = np.zeros_like(jaws)
        dm = np.zeros_like(mu)
        rc = lib().orc_dose_grad(C.byref(self.grid), C.byref(self.cplan), _p(leaves), _p(jaws),
                                 _p(mu), _p(g), _p(dl), _p(dj), _p(dm))
        if rc:
            raise RuntimeError(f"orc_dose_grad failed: {rc}")
        return dl, dj, dm

    # --- stages (for pins and dot-product tests) --------------------------
    def project(self, b, leaves=None, jaws=None, mu=None):
        leaves = _f64(self.plan.leaves if leaves is None else leaves)
        jaws = _f64(self.plan.jaws if jaws is None else jaws)
        mu = _f64(self.plan.mu if mu is None else mu)
        lv = np.zeros((self.machine.n_pairs, 2))
        jw = np.zeros(4)
        m = D()
        lib().orc_project_cp(C.byref(self.cplan), _p(_f64(leaves[b])), _p(_f64(jaws[b])),
                             D(float(mu[b])), _p(lv), _p(jw), C.byref(m))
        return lv, jw, m.value

    def fluence(self, lv_proj, jw_proj):
        F = np.zeros((self.lat.nv, self.lat.nu))
        lib().orc_fluence(C.byref(self.cplan), C.byref(self.lat), _p(_f64(lv_proj)),
                          _p(_f64(jw_proj)), _p(F))
        return F

    def fluence_correct(self, F):
        out = _f64(F).copy()
        lib().orc_fluence_correct(C.byref(self.cplan), C.byref(self.lat), _p(out))
        return out

    def fluence_correct_T(self, G):
        out = _f64(G).copy()
        lib().orc_fluence_correct_T(C.byref(self.cplan), C.byref(self.lat), _p(out))
        return out

    def rotate(self, F):
        """Collimator rotation of a lattice map [nv][nu] (bilinear)."""
        out = np.zeros((self.lat.nv, self.lat.nu))
        lib().orc_rotate(C.byref(self.cplan), C.byref(self.lat), _p(_f64(F)), _p(out))
        return out

    def rotate_T(self, G):
        out = np.zeros((self.lat.nv, self.lat.nu))
        lib().orc_rotate_T(C.byref(self.cplan), C.byref(self.lat), _p(_f64(G)), _p(out))
        return out

    def fluence_vjp(self, b, dF, leaves=None, jaws=None):
        leaves = _f64(self.plan.leaves if leaves is None else leaves)
        jaws = _f64(self.plan.jaws if jaws is None else jaws)
        dl = np.zeros((self.machine.n_pairs, 2))
        dj = np.zeros(4)
        lib().orc_fluence_vjp(C.byref(self.cplan), C.byref(self.lat), _p(_f64(leaves[b])),
                              _p(_f64(jaws[b])), _p(_f64(dF)), _p(dl), _p(dj))
        return dl, dj

    def wepl(self, b):
        z = np.zeros(self.lat.nw)
        lib().orc_wepl(C.byref(self.grid), C.byref(self.cplan), C.byref(self.lat), C.c_int(b), _p(z))
        return z

    def depth_dose(self, z):
        return lib().orc_depth_dose(C.byref(self.cplan), D(float(z)))

    def kernel(self, z):
        R = self.machine.r_px
        K = np.zeros((2 * R + 1, 2 * R + 1))
        lib().orc_kernel(C.byref(self.cplan), C.byref(self.lat), D(float(z)), _p(K))
        return K

    def kernel_params(self, z):
        a = np.zeros(3)
        w = np.zeros(3)
        lib().orc_kernel_params(C.byref(self.cplan), D(float(z)), _p(a), _p(w))
        return a, w

    def magnify(self, F):
        Phi = np.zeros(self.vol_shape())
        lib().orc_magnify(C.byref(self.cplan), C.byref(self.lat), _p(_f64(F)), _p(Phi))
        return Phi

    def magnify_T(self, Phi_adj):
        Fa = np.zeros((self.lat.nv, self.lat.nu))
        lib().orc_magnify_T(C.byref(self.cplan), C.byref(self.lat), _p(_f64(Phi_adj)), None, _p(Fa))
        return Fa

    def conv(self, z, Phi, brute=False):
        Dp = np.zeros(self.vol_shape())
        lib().orc_conv(C.byref(self.cplan), C.byref(self.lat), _p(_f64(z)), _p(_f64(Phi)), _p(Dp),
                       C.c_int(1 if brute else 0))
        return Dp

    def conv_T(self, z, h):
        hp = np.zeros(self.vol_shape())
        lib().orc_conv_T(C.byref(self.cplan), C.byref(self.lat), _p(_f64(z)), _p(_f64(h)), None, _p(hp))
        return hp

    def gather(self, b, Dp, scale=1.0):
        out = np.zeros(self.phantom.hu.shape)
        lib().orc_gather(C.byref(self.grid), C.byref(self.cplan), C.byref(self.lat), C.c_int(b),
                         _p(_f64(Dp)), D(scale), _p(out))
        return out

    def gather_T(self, b, g):
        h = np.zeros(self.vol_shape())
        lib().orc_gather_T(C.byref(self.grid), C.byref(self.cplan), C.byref(self.lat), C.c_int(b),
                           _p(_f64(g)), _p(h))
        return h

    def beam_dose(self, b, leaves_cp, jaws_cp):
        Dp = np.zeros(self.vol_shape())
        rc = lib().orc_beam_dose(C.byref(self.grid), C.byref(self.cplan), C.c_int(b),
                                 _p(_f64(leaves_cp)), _p(_f64(jaws_cp)), _p(Dp))
        if rc:
            raise RuntimeError("orc_beam_dose failed")
        return Dp


def overlap(x, lo, hi, d):
    return lib().orc_overlap(float(x), float(lo), float(hi), float(d))


def hu_to_red(hu, pts):
    hu = _f64(hu).ravel()
    pts = _f64(pts).ravel()
    out = np.empty_like(hu)
    lib().orc_hu_to_red(_p(hu), C.c_long(hu.size), _p(pts), C.c_int(len(pts) // 2), _p(out))
    return out


def calibrate(machine, sxy, sz, ref_mu=None, ref_gy=None, details=False):
    """Output calibration of Sec. 2.4 (orc_calibrate): the factor cal that
    makes ref_mu MU of the 10 x 10 cm reference field give ref_gy Gy at 10 cm
    depth in water (SSD = SID - 100 mm) on a grid of the given pitch.  With
    details=True also returns the reference slice's WEPL and dose per MU."""
    ref_mu = float(getattr(machine, "cal_ref_mu", 100.0) if ref_mu is None else ref_mu)
    ref_gy = float(getattr(machine, "cal_ref_gy", 1.0) if ref_gy is None else ref_gy)
    gantry = _f64([0.0])
    pl = _plan_struct(machine, gantry, (0.0, 0.0, 0.0), cal=1.0)
    cal, zr, dpm = D(), D(), D()
    rc = lib().orc_calibrate(C.byref(pl), D(float(sxy)), D(float(sz)), D(ref_mu), D(ref_gy),
                             C.byref(cal), C.byref(zr), C.byref(dpm))
    if rc:
        raise RuntimeError(f"orc_calibrate failed: {rc}")
    return (cal.value, zr.value, dpm.value) if details else cal.value


def num_threads():
    return lib().orc_num_threads()


def set_num_threads(n):
    lib().orc_set_num_threads(C.c_int(int(n)))
