"""Plain PyTorch FP64 restatement of the dose model, differentiated by autograd.

TEST INFRASTRUCTURE ONLY.  A second, independent transcription of the model
that pdrt_oracle.c defines (the paper's layers in order, Sec. 2.1-2.2.7),
written with stock torch ops so that torch.autograd provides reference
gradients with respect to leaves, jaws and MU.  It shares no code with the C
oracle or with the CUDA library; the tests check all three against each other.

Discrete readings (same as the C oracle): beam lattice of spacing sx (u, w) and
sz (v) centred on the isocentre; fractional-overlap fluence with jaw masking
and MLC transmission tau; trilinear midpoint-sum WEPL on the central ray;
three-exponential kernel normalised on its (2R+1)^2 window; depth dose T(z) per
slice; magnification SID/d and inverse square (SID/d)^2 with d = SID + w;
grouped "same" convolution; trilinear gather back to the patient grid; MU sum.
The hardware projection is passed through as the identity in the backward
pass when machine.ste is set (straight-through estimator).
"""
from __future__ import annotations

import math

import numpy as np
import torch
import torch.nn.functional as Fn

DT = torch.float64


def _lattice(phantom, iso):
    nz, ny, nx = phantom.hu.shape
    sx, sy, sz = phantom.spacing
    ox, oy, oz = phantom.origin
    xs = np.array([ox, ox + (nx - 1) * sx]) - iso[0]
    ys = np.array([oy, oy + (ny - 1) * sy]) - iso[1]
    rmax = max(math.hypot(x, y) for x in xs for y in ys)
    H = int(math.ceil(rmax / sx - 1e-9)) + 1
    return dict(nu=2 * H + 1, nw=2 * H + 1, nv=nz, cu=float(H), cw=float(H),
                cv=(iso[2] - oz) / sz, du=sx, dv=sz)


def _red(phantom):
    pts = np.asarray(phantom.hu_to_red, np.float64)
    return np.interp(np.asarray(phantom.hu, np.float64), pts[:, 0], pts[:, 1])


def _axes(g_deg):
    g = math.radians(g_deg)
    return (np.array([math.cos(g), -math.sin(g), 0.0]), np.array([0.0, 0.0, 1.0]),
            np.array([math.sin(g), math.cos(g), 0.0]))


def _trilinear_weights(f0, f1, f2, n0, n1, n2):
    """Flat indices and weights of the 8 trilinear neighbours (zero outside)."""
    b0, b1, b2 = np.floor(f0), np.floor(f1), np.floor(f2)
    t0, t1, t2 = f0 - b0, f1 - b1, f2 - b2
    b0, b1, b2 = b0.astype(np.int64), b1.astype(np.int64), b2.astype(np.int64)
    idx, wts = [], []
    for d2 in (0, 1):
        for d1 in (0, 1):
            for d0 in (0, 1):
                i0, i1, i2 = b0 + d0, b1 + d1, b2 + d2
                w = ((t0 if d0 else 1 - t0) * (t1 if d1 else 1 - t1) * (t2 if d2 else 1 - t2))
                ok = (i0 >= 0) & (i0 < n0) & (i1 >= 0) & (i1 < n1) & (i2 >= 0) & (i2 < n2)
                idx.append(np.where(ok, (i2 * n1 + i1) * n0 + i0, 0))
                wts.append(np.where(ok, w, 0.0))
    return np.stack(idx), np.stack(wts)


def _ov(x, lo, hi, d):
    return torch.clamp(torch.minimum(hi, x + d / 2) - torch.maximum(lo, x - d / 2), min=0.0) / d


def _project(pa, pb, wmin, F, ste):
    c = 0.5 * (pa + pb)
    w = pb - pa
    w2 = torch.clamp(w, min=wmin)
    c2 = torch.clamp(c, -F, F)
    a_hat, b_hat = c2 - 0.5 * w2, c2 + 0.5 * w2
    if ste:
        a_hat = pa + (a_hat - pa).detach()
        b_hat = pb + (b_hat - pb).detach()
    return a_hat, b_hat


class TorchDose:
    """dose(leaves, jaws, mu) as a differentiable torch function (FP64, CPU)."""

    def __init__(self, phantom, machine, gantry_deg, iso):
        self.ph, self.m = phantom, machine
        self.gantry = np.asarray(gantry_deg, np.float64)
        self.iso = np.asarray(iso, np.float64)
        self.L = _lattice(phantom, self.iso)
        self.red = _red(phantom)
        self._cache = {}

    # --- gradient-free pieces (Sec. 2.2.4, 2.2.5) -------------------------
    def wepl(self, b):
        L, ph = self.L, self.ph
        eu, ev, ew = _axes(self.gantry[b])
        w = (np.arange(L["nw"]) - L["cw"]) * L["du"]
        s = self.iso[None, :] + w[:, None] * ew[None, :]
        nz, ny, nx = ph.hu.shape
        f = [(s[:, d] - ph.origin[d]) / ph.spacing[d] for d in range(3)]
        idx, wts = _trilinear_weights(f[0], f[1], f[2], nx, ny, nz)
        rho = (self.red.ravel()[idx] * wts).sum(0)
        csum = np.concatenate([[0.0], np.cumsum(rho)[:-1]])
        return L["du"] * (csum + 0.5 * rho)

    def kernel(self, z):
        m, L = self.m, self.L
        R = m.r_px
        p = np.arange(-R, R + 1)
        r = np.sqrt((p[:, None] * L["du"]) ** 2 + (p[None, :] * L["dv"]) ** 2)   # [p][q]
        a = m.alpha[:, 0] + m.alpha[:, 1] * z + m.alpha[:, 2] * z * z
        a = np.maximum(a, 1e-4)
        wr = np.maximum(m.beta[:, 0] + m.beta[:, 1] * z + m.beta[:, 2] * z * z, 0.0)
        w = wr / wr.sum() if wr.sum() > 0 else np.zeros(3)
        K = np.zeros_like(r)
        for c in range(3):
            e = np.exp(-a[c] * r)
            K += w[c] * e / e.sum()
        return K

    def depth_dose(self, z):
        m = self.m
        zz = np.arange(len(m.t_table)) * m.dz_t
        return np.interp(z, zz, m.t_table)

    # --- one control point --------------------------------------------------
    def _static(self, b):
        if b in self._cache:
            return self._cache[b]
        L, ph, m = self.L, self.ph, self.m
        nu, nv, nw = L["nu"], L["nv"], L["nw"]
        z = self.wepl(b)
        # magnification stencils: Phi_k(i,j) = C_k bilinear(F, m_k(i-cu)+cu, m_k(j-cv)+cv)
        k = np.arange(nw)
        mk = m.sid / (m.sid + (k - L["cw"]) * L["du"])
        fa = mk[:, None, None] * (np.arange(nu)[None, None, :] - L["cu"]) + L["cu"]
        fc = mk[:, None, None] * (np.arange(nv)[None, :, None] - L["cv"]) + L["cv"]
        fa = np.broadcast_to(fa, (nw, nv, nu))
        fc = np.broadcast_to(fc, (nw, nv, nu))
        idx, wts = _trilinear_weights(fa, fc, np.zeros_like(fa), nu, nv, 1)
        wts = wts * (mk ** 2)[None, :, None, None]
        # kernels (flipped into conv2d's cross-correlation form) and depth dose
        R = m.r_px
        Ks = np.stack([self.kernel(zk)[::-1, ::-1].T for zk in z])   # [k][q][p]
        T = self.depth_dose(z)
        # trilinear gather of voxels from the beam volume
        eu, ev, ew = _axes(self.gantry[b])
        nzv, nyv, nxv = ph.hu.shape
        Z, Y, X = np.meshgrid(ph.origin[2] + ph.spacing[2] * np.arange(nzv) - self.iso[2],
                              ph.origin[1] + ph.spacing[1] * np.arange(nyv) - self.iso[1],
                              ph.origin[0] + ph.spacing[0] * np.arange(nxv) - self.iso[0],
                              indexing="ij")
        u = X * eu[0] + Y * eu[1] + Z * eu[2]
        v = X * ev[0] + Y * ev[1] + Z * ev[2]
        w = X * ew[0] + Y * ew[1] + Z * ew[2]
        gidx, gw = _trilinear_weights(u / L["du"] + L["cu"], v / L["dv"] + L["cv"],
                                      w / L["du"] + L["cw"], nu, nv, nw)
        st = dict(idx=torch.from_numpy(idx[:4]), wts=torch.from_numpy(wts[:4]),
                  K=torch.from_numpy(np.ascontiguousarray(Ks))[:, None], T=torch.from_numpy(T),
                  gidx=torch.from_numpy(gidx), gw=torch.from_numpy(gw))
        self._cache[b] = st
        return st

    def fluence(self, lv, jw):
        """lv: (n_pairs, 2) projected, jw: (4,) projected -> F (nv, nu)."""
        L, m = self.L, self.m
        u = (torch.arange(L["nu"], dtype=DT) - L["cu"]) * L["du"]
        v = (torch.arange(L["nv"], dtype=DT) - L["cv"]) * L["dv"]
        lb = torch.as_tensor(m.leaf_bounds, dtype=DT)
        fx = _ov(u, jw[0], jw[1], L["du"])
        fy = _ov(v, jw[2], jw[3], L["dv"])
        omega = _ov(v[None, :], lb[:-1, None], lb[1:, None], L["dv"])      # (np, nv)
        fu = _ov(u[None, :], lv[:, 0:1], lv[:, 1:2], L["du"])               # (np, nu)
        fl = omega.T @ fu
        return fy[:, None] * fx[None, :] * (m.tau + (1 - m.tau) * fl)

    def _blur_matrix(self, n, pitch, fwhm):
        """Banded Gaussian blur matrix (zero padding), taps to ceil(3 sigma)."""
        if not fwhm > 0:
            return None
        sigma = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
        rb = int(math.ceil(3.0 * sigma / pitch))
        t = np.arange(-rb, rb + 1)
        g = np.exp(-(t * pitch) ** 2 / (2 * sigma ** 2))
        g /= g.sum()
        B = np.zeros((n, n))
        for d, gv in zip(t, g):
            B += gv * np.eye(n, k=-d)
        return torch.from_numpy(B)

    def correct(self, F):
        """Penumbra blurs along u then v, the off-axis profile, then the
        collimator rotation (Sec. 2.2.2)."""
        L, m = self.L, self.m
        Bu = self._blur_matrix(L["nu"], L["du"], getattr(m, "pen_fwhm_u", 0.0))
        Bv = self._blur_matrix(L["nv"], L["dv"], getattr(m, "pen_fwhm_v", 0.0))
        if Bu is not None:
            F = F @ Bu.T
        if Bv is not None:
            F = Bv @ F
        c = getattr(m, "off_axis", (1.0, 0.0, 0.0))
        u = (np.arange(L["nu"]) - L["cu"]) * L["du"]
        v = (np.arange(L["nv"]) - L["cv"]) * L["dv"]
        r = np.sqrt(u[None, :] ** 2 + v[:, None] ** 2)
        F = F * torch.from_numpy(c[0] + c[1] * r + c[2] * r * r)
        th = math.radians(getattr(m, "collimator_deg", 0.0))
        if th != 0.0:
            F = self._rotation(th, u, v) @ F.reshape(-1, 1)
            F = F.reshape(L["nv"], L["nu"])
        return F

    def _rotation(self, th, u, v):
        """Sparse bilinear resampling matrix of the collimator rotation: the
        map at pixel x is read at R(-th) x (zero outside the lattice)."""
        L = self.L
        nu, nv = L["nu"], L["nv"]
        U, V = np.meshgrid(u, v)                          # (nv, nu)
        fa = L["cu"] + (math.cos(th) * U + math.sin(th) * V) / L["du"]
        fc = L["cv"] + (-math.sin(th) * U + math.cos(th) * V) / L["dv"]
        a0, c0 = np.floor(fa), np.floor(fc)
        ta, tc = fa - a0, fc - c0
        rows, cols, vals = [], [], []
        dst = np.arange(nu * nv).reshape(nv, nu)
        for dc, wc in ((0, 1 - tc), (1, tc)):
            for da, wa in ((0, 1 - ta), (1, ta)):
                aa, cc = a0.astype(int) + da, c0.astype(int) + dc
                ok = (aa >= 0) & (aa < nu) & (cc >= 0) & (cc < nv)
                rows.append(dst[ok]); cols.append((cc * nu + aa)[ok]); vals.append((wa * wc)[ok])
        idx = torch.from_numpy(np.stack([np.concatenate(rows), np.concatenate(cols)]))
        return torch.sparse_coo_tensor(idx, torch.from_numpy(np.concatenate(vals)), (nu * nv, nu * nv),
                                       check_invariants=True)

    def project(self, leaves_b, jaws_b, mu_b):
        m = self.m
        la, lb_ = _project(leaves_b[:, 0], leaves_b[:, 1], m.wmin_leaf, m.f_leaf, m.ste)
        jx0, jx1 = _project(jaws_b[0], jaws_b[1], m.wmin_jaw, m.f_jaw, m.ste)
        jy0, jy1 = _project(jaws_b[2], jaws_b[3], m.wmin_jaw, m.f_jaw, m.ste)
        muh = torch.clamp(mu_b, min=m.eps_mu)
        if m.ste:
            muh = mu_b + (muh - mu_b).detach()
        return torch.stack([la, lb_], 1), torch.stack([jx0, jx1, jy0, jy1]), muh

    def beam(self, b, F):
        """MU-free, cal-free dose of control point b from its fluence map F."""
        L = self.L
        st = self._static(b)
        Phi = (F.reshape(-1)[st["idx"]] * st["wts"]).sum(0)              # (nw, nv, nu)
        Dp = Fn.conv2d(Phi[None], st["K"], padding=self.m.r_px, groups=L["nw"])[0]
        Dp = Dp * st["T"][:, None, None]
        return (Dp.reshape(-1)[st["gidx"]] * st["gw"]).sum(0)

    def dose(self, leaves, jaws, mu):
        out = None
        for b in range(len(self.gantry)):
            lv, jw, muh = self.project(leaves[b], jaws[b], mu[b])
            d = self.m.cal * muh * self.beam(b, self.correct(self.fluence(lv, jw)))
            out = d if out is None else out + d
        return out
