/*
 * pdrt_oracle.c -- plain FP64 CPU oracle of the differentiable pencil-beam
 * VMAT dose model of arXiv 2512.18863 ("PyDoseRT").
 *
 * TEST INFRASTRUCTURE ONLY.  This file defines, slowly and in double
 * precision, what the GPU library must compute.  Only tests/, the smoke()
 * entry of __graft_entry__.py and the CPU-baseline leg of bench.py may load
 * it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Every step follows the paper's layer order (Sec. 2.1):
 *   BeamValidation (Sec. 2.2.1) -> FluenceMap (Sec. 2.2.2, Eq. overlap)
 *   -> FluenceVolume (Sec. 2.2.3, magnification + inverse square)
 *   -> RadiologicalDepth (Sec. 2.2.4, WEPL integral)
 *   -> PencilBeamKernel (Sec. 2.2.5) -> BeamWiseConvolution (Sec. 2.2.6)
 *   -> BeamRotation + MU-weighted sum (Sec. 2.2.7, Eq. D_total).
 * The paper leaves the discretisation open; the reading taken for each
 * open point is stated at the function that implements it.  The adjoint functions are the exact transposes of the
 * linear stages plus the derivative of the overlap formula (Sec. 2.2.2 states
 * that it gives stable subgradients); the projection of Sec. 2.2.1 is passed
 * through as the identity when ste != 0 (straight-through estimator).
 *
 * Pins (tests/test_oracle_*.py): open-field water depth dose with
 * inverse-square fall-off, WEPL slab closed forms, pencil-beam kernel shape,
 * magnification of a sharp field edge, MU linearity, abutting half fields,
 * closed-MLC leakage, 90-degree rotation symmetry, fluence partition of unity,
 * brute force on a 16^3 grid, adjoint dot products and central finite
 * differences, and the output calibration against the depth-dose table at the
 * reference depth.  No function here is "parity unpinned".
 *
 * Layouts (x fastest / last index fastest):
 *   red, dose, dose gradient : [nz][ny][nx]
 *   fluence F                : [nv][nu]        (v = patient z planes)
 *   beam-frame volumes       : [nw][nv][nu]
 *   leaves                   : [n_cp][n_pairs][2]  (left, right) in mm
 *   jaws                     : [n_cp][4]  (x-, x+, y-, y+) in mm
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 4

typedef struct {
    int nx, ny, nz;
    double sx, sy, sz;
    double origin[3];          /* centre of voxel (0,0,0), mm */
    const double *red;         /* relative electron density [nz][ny][nx] */
} orc_grid;

typedef struct {
    int n_cp;
    const double *gantry_deg;  /* [n_cp] */
    double iso[3];             /* mm, patient frame */
    double sid;                /* source-isocentre distance, mm */
    int n_pairs;
    const double *leaf_bounds; /* [n_pairs+1] ascending v (mm at iso plane) */
    double tau;                /* MLC transmission */
    double wmin_leaf, wmin_jaw;
    double f_leaf, f_jaw;      /* half travel range of the aperture centre */
    double eps_mu;
    int r_px;                  /* kernel half window, pixels */
    double alpha[3][3];        /* a_c(z) = alpha[c][0] + alpha[c][1] z + alpha[c][2] z^2 */
    double beta[3][3];         /* raw weight polynomials */
    int n_t;
    double dz_t;
    const double *t_table;     /* depth-dose table T(m dz_t), m = 0..n_t-1 */
    double cal;                /* output calibration (Sec. 2.4) */
    int ste;
    /* fluence corrections (Sec. 2.2.2): source penumbra as Gaussian blurs of
     * the given FWHM along u (leaf travel) and v (across leaf pairs / Y jaws),
     * 0 = off; off-axis profile OAP(r) = oap[0] + oap[1] r + oap[2] r^2 */
    double pen_fwhm_u, pen_fwhm_v;
    double oap[3];
    /* collimator angle (Sec. 2.2.2, last paragraph): the corrected map is
     * turned by coll_deg in the (u, v) plane about the central axis before the
     * projection; 0 = off */
    double coll_deg;
} orc_plan;

typedef struct {
    int nu, nv, nw;
    double cu, cv, cw;         /* fractional lattice index of the isocentre */
    double du, dv;             /* du = dw = sx, dv = sz */
} orc_lattice;

static const double ORC_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------ */
/* Geometry (Sec. 2.2, beam parameter vector; reading: gantry rotates about  */
/* the patient z axis, e_w = (sin g, cos g, 0), e_u = (cos g, -sin g, 0),    */
/* e_v = (0,0,1), source at iso - SID e_w).                                  */
/* ------------------------------------------------------------------------ */
void orc_beam_axes(double gantry_deg, double eu[3], double ev[3], double ew[3])
{
    double g = gantry_deg * ORC_PI / 180.0;
    ew[0] = sin(g); ew[1] = cos(g); ew[2] = 0.0;
    eu[0] = cos(g); eu[1] = -sin(g); eu[2] = 0.0;
    ev[0] = 0.0;    ev[1] = 0.0;     ev[2] = 1.0;
}

/* Beam-frame lattice: spacing sx in u and w, sz in v; v planes are the
 * patient z planes; u and w run over +-H pixels with H chosen so that every
 * voxel centre of the grid lies inside at every gantry angle (reading). */
void orc_lattice_of(const orc_grid *g, const orc_plan *p, orc_lattice *L)
{
    double rmax = 0.0;
    for (int cx = 0; cx < 2; ++cx)
        for (int cy = 0; cy < 2; ++cy) {
            double x = g->origin[0] + (cx ? g->nx - 1 : 0) * g->sx - p->iso[0];
            double y = g->origin[1] + (cy ? g->ny - 1 : 0) * g->sy - p->iso[1];
            double r = sqrt(x * x + y * y);
            if (r > rmax) rmax = r;
        }
    int H = (int)ceil(rmax / g->sx - 1e-9) + 1;
    L->nu = L->nw = 2 * H + 1;
    L->cu = L->cw = (double)H;
    L->nv = g->nz;
    L->cv = (p->iso[2] - g->origin[2]) / g->sz;
    L->du = g->sx;
    L->dv = g->sz;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2.4: HU -> relative electron density by the commissioned           */
/* piecewise-linear curve (clamped at both ends).                            */
/* ------------------------------------------------------------------------ */
double orc_hu_to_red_1(double hu, const double *pts, int n)
{
    if (hu <= pts[0]) return pts[1];
    if (hu >= pts[2 * (n - 1)]) return pts[2 * (n - 1) + 1];
    for (int m = 0; m + 1 < n; ++m) {
        double h0 = pts[2 * m], h1 = pts[2 * m + 2];
        if (hu >= h0 && hu <= h1) {
            double t = (hu - h0) / (h1 - h0);
            return pts[2 * m + 1] + t * (pts[2 * m + 3] - pts[2 * m + 1]);
        }
    }
    return pts[2 * (n - 1) + 1];
}

void orc_hu_to_red(const double *hu, long n, const double *pts, int npts, double *red)
{
    for (long i = 0; i < n; ++i) red[i] = orc_hu_to_red_1(hu[i], pts, npts);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2.1 (BeamValidationLayer): centre/width projection.                */
/* gc, gw: 1 where the clamp on centre / width is inactive (derivative of    */
/* min/max taken on the first argument at a tie).                            */
/* ------------------------------------------------------------------------ */
static void project_pair(double pa, double pb, double wmin, double F,
                         double *ah, double *bh, double *gc, double *gw)
{
    double c = 0.5 * (pa + pb);
    double w = pb - pa;
    double w2 = (w >= wmin) ? w : wmin;
    double c1 = (c >= -F) ? c : -F;
    double c2 = (c1 <= F) ? c1 : F;
    *ah = c2 - 0.5 * w2;
    *bh = c2 + 0.5 * w2;
    if (gw) *gw = (w >= wmin) ? 1.0 : 0.0;
    if (gc) *gc = ((c >= -F) ? 1.0 : 0.0) * ((c1 <= F) ? 1.0 : 0.0);
}

/* Projected leaves [n_pairs][2], jaws [4] and MU of one control point. */
void orc_project_cp(const orc_plan *p, const double *leaves_cp, const double *jaws_cp,
                    double mu, double *lv_out, double *jw_out, double *mu_out)
{
    for (int i = 0; i < p->n_pairs; ++i)
        project_pair(leaves_cp[2 * i], leaves_cp[2 * i + 1], p->wmin_leaf, p->f_leaf,
                     &lv_out[2 * i], &lv_out[2 * i + 1], NULL, NULL);
    project_pair(jaws_cp[0], jaws_cp[1], p->wmin_jaw, p->f_jaw, &jw_out[0], &jw_out[1], NULL, NULL);
    project_pair(jaws_cp[2], jaws_cp[3], p->wmin_jaw, p->f_jaw, &jw_out[2], &jw_out[3], NULL, NULL);
    *mu_out = (mu >= p->eps_mu) ? mu : p->eps_mu;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2.2, Eq. (fractional overlap): f(d; l, r) =                        */
/*   max(0, min(r, d + D/2) - max(l, d - D/2)) / D                           */
/* ------------------------------------------------------------------------ */
double orc_overlap(double x, double lo, double hi, double d)
{
    double e = x + 0.5 * d, s = x - 0.5 * d;
    double top = (hi <= e) ? hi : e;
    double bot = (lo >= s) ? lo : s;
    double X = top - bot;
    return (X > 0.0) ? X / d : 0.0;
}

/* One-sided derivatives of the overlap (ties go to the first argument of
 * min/max; no derivative where the overlap is zero). */
static double overlap_dhi(double x, double lo, double hi, double d)
{
    double e = x + 0.5 * d, s = x - 0.5 * d;
    double top = (hi <= e) ? hi : e;
    double bot = (lo >= s) ? lo : s;
    return (top - bot > 0.0 && hi <= e) ? 1.0 / d : 0.0;
}

static double overlap_dlo(double x, double lo, double hi, double d)
{
    double e = x + 0.5 * d, s = x - 0.5 * d;
    double top = (hi <= e) ? hi : e;
    double bot = (lo >= s) ? lo : s;
    return (top - bot > 0.0 && lo >= s) ? -1.0 / d : 0.0;
}

/* Sec. 2.2.2: fluence of one control point from PROJECTED parameters.
 * F = f_jaw (tau + (1 - tau) f_leaf) with
 *   f_jaw  = f(u; x-, x+) f(v; y-, y+)           (jaws: "analogous masking")
 *   f_leaf = sum_i omega_i(v) f(u; l_i, r_i),     omega_i = row overlap with leaf strip i
 * and tau the MLC transmission.  F is [nv][nu] on the iso-plane lattice. */
void orc_fluence(const orc_plan *p, const orc_lattice *L, const double *lv,
                 const double *jw, double *F)
{
    for (int c = 0; c < L->nv; ++c) {
        double v = (c - L->cv) * L->dv;
        double fy = orc_overlap(v, jw[2], jw[3], L->dv);
        for (int a = 0; a < L->nu; ++a) {
            double u = (a - L->cu) * L->du;
            double fx = orc_overlap(u, jw[0], jw[1], L->du);
            double fl = 0.0;
            for (int i = 0; i < p->n_pairs; ++i) {
                double om = orc_overlap(v, p->leaf_bounds[i], p->leaf_bounds[i + 1], L->dv);
                if (om > 0.0) fl += om * orc_overlap(u, lv[2 * i], lv[2 * i + 1], L->du);
            }
            F[(long)c * L->nu + a] = fx * fy * (p->tau + (1.0 - p->tau) * fl);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2.2, physics corrections applied in sequence to the raw aperture  */
/* fluence (readings): source penumbra = separable Gaussian blur, sigma =   */
/* FWHM / (2 sqrt(2 ln 2)), taps |t| <= ceil(3 sigma / pitch) normalised to */
/* unit sum, zero outside the lattice; then the off-axis profile            */
/* OAP(r) = c0 + c1 r + c2 r^2 with r the distance from the central axis at  */
/* the isocentre plane.  Both are linear in F; the blur matrix is symmetric. */
/* ------------------------------------------------------------------------ */
int orc_penumbra_radius(double fwhm, double pitch)
{
    if (!(fwhm > 0.0)) return 0;
    double sigma = fwhm / (2.0 * sqrt(2.0 * log(2.0)));
    return (int)ceil(3.0 * sigma / pitch);
}

static void gauss_taps(double fwhm, double pitch, int rb, double *g)
{
    double sigma = fwhm / (2.0 * sqrt(2.0 * log(2.0)));
    double s = 0.0;
    for (int t = -rb; t <= rb; ++t) {
        g[t + rb] = exp(-(t * pitch) * (t * pitch) / (2.0 * sigma * sigma));
        s += g[t + rb];
    }
    for (int t = 0; t <= 2 * rb; ++t) g[t] /= s;
}

/* In-place blur of F [nv][nu] along u (axis 0) or v (axis 1). */
static void blur_axis(double *F, int nu, int nv, int axis, double fwhm, double pitch)
{
    int rb = orc_penumbra_radius(fwhm, pitch);
    if (rb == 0) return;
    double *g = (double *)malloc(sizeof(double) * (2 * rb + 1));
    double *tmp = (double *)malloc(sizeof(double) * nu * nv);
    gauss_taps(fwhm, pitch, rb, g);
    for (int c = 0; c < nv; ++c)
        for (int a = 0; a < nu; ++a) {
            double s = 0.0;
            for (int t = -rb; t <= rb; ++t) {
                int aa = axis == 0 ? a - t : a, cc = axis == 0 ? c : c - t;
                if (aa < 0 || aa >= nu || cc < 0 || cc >= nv) continue;
                s += g[t + rb] * F[(long)cc * nu + aa];
            }
            tmp[(long)c * nu + a] = s;
        }
    memcpy(F, tmp, sizeof(double) * nu * nv);
    free(g); free(tmp);
}

double orc_off_axis(const orc_plan *p, double u, double v)
{
    double r = sqrt(u * u + v * v);
    return p->oap[0] + p->oap[1] * r + p->oap[2] * r * r;
}

/* Source position, in fractional lattice indices, that the collimator
 * rotation brings to lattice pixel (a, c).  A feature of the unrotated map at
 * s = (u, v) appears at R(theta) s, so pixel x reads the map at R(-theta) x:
 *   u' = cos(theta) u + sin(theta) v,   v' = -sin(theta) u + cos(theta) v. */
void orc_rotation_source(const orc_plan *p, const orc_lattice *L, int a, int c, double *fa,
                         double *fc)
{
    double th = p->coll_deg * ORC_PI / 180.0;
    double u = (a - L->cu) * L->du, v = (c - L->cv) * L->dv;
    double us = cos(th) * u + sin(th) * v, vs = -sin(th) * u + cos(th) * v;
    *fa = L->cu + us / L->du;
    *fc = L->cv + vs / L->dv;
}

static double bilinear2(const double *F, int nu, int nv, double fa, double fc);
static void bilinear2_T(double *F, int nu, int nv, double fa, double fc, double val);

/* out [nv][nu] = F turned by the collimator angle (bilinear, zero outside
 * the lattice). */
void orc_rotate(const orc_plan *p, const orc_lattice *L, const double *F, double *out)
{
    for (int c = 0; c < L->nv; ++c)
        for (int a = 0; a < L->nu; ++a) {
            double fa, fc;
            orc_rotation_source(p, L, a, c, &fa, &fc);
            out[(long)c * L->nu + a] = bilinear2(F, L->nu, L->nv, fa, fc);
        }
}

/* out = rotate^T G (out is overwritten). */
void orc_rotate_T(const orc_plan *p, const orc_lattice *L, const double *G, double *out)
{
    memset(out, 0, sizeof(double) * L->nu * L->nv);
    for (int c = 0; c < L->nv; ++c)
        for (int a = 0; a < L->nu; ++a) {
            double fa, fc;
            orc_rotation_source(p, L, a, c, &fa, &fc);
            bilinear2_T(out, L->nu, L->nv, fa, fc, G[(long)c * L->nu + a]);
        }
}

/* Penumbra, off-axis profile, then collimator rotation, in place on F [nv][nu]. */
void orc_fluence_correct(const orc_plan *p, const orc_lattice *L, double *F)
{
    blur_axis(F, L->nu, L->nv, 0, p->pen_fwhm_u, L->du);
    blur_axis(F, L->nu, L->nv, 1, p->pen_fwhm_v, L->dv);
    for (int c = 0; c < L->nv; ++c)
        for (int a = 0; a < L->nu; ++a)
            F[(long)c * L->nu + a] *= orc_off_axis(p, (a - L->cu) * L->du, (c - L->cv) * L->dv);
    if (p->coll_deg != 0.0) {
        double *t = (double *)malloc(sizeof(double) * L->nu * L->nv);
        orc_rotate(p, L, F, t);
        memcpy(F, t, sizeof(double) * L->nu * L->nv);
        free(t);
    }
}

/* Transpose of orc_fluence_correct (rotation, off-axis profile, then the blurs). */
void orc_fluence_correct_T(const orc_plan *p, const orc_lattice *L, double *G)
{
    if (p->coll_deg != 0.0) {
        double *t = (double *)malloc(sizeof(double) * L->nu * L->nv);
        orc_rotate_T(p, L, G, t);
        memcpy(G, t, sizeof(double) * L->nu * L->nv);
        free(t);
    }
    for (int c = 0; c < L->nv; ++c)
        for (int a = 0; a < L->nu; ++a)
            G[(long)c * L->nu + a] *= orc_off_axis(p, (a - L->cu) * L->du, (c - L->cv) * L->dv);
    blur_axis(G, L->nu, L->nv, 1, p->pen_fwhm_v, L->dv);
    blur_axis(G, L->nu, L->nv, 0, p->pen_fwhm_u, L->du);
}

/* ------------------------------------------------------------------------ */
/* Trilinear / bilinear sampling with zero outside the sampled lattice.      */
/* ------------------------------------------------------------------------ */
static double trilinear(const double *V, int n0, int n1, int n2, double f0, double f1, double f2)
{
    /* V[i2][i1][i0], f0 fastest */
    double fl0 = floor(f0), fl1 = floor(f1), fl2 = floor(f2);
    int a0 = (int)fl0, a1 = (int)fl1, a2 = (int)fl2;
    double t0 = f0 - fl0, t1 = f1 - fl1, t2 = f2 - fl2;
    double s = 0.0;
    for (int d2 = 0; d2 < 2; ++d2) {
        int i2 = a2 + d2;
        if (i2 < 0 || i2 >= n2) continue;
        double w2 = d2 ? t2 : 1.0 - t2;
        for (int d1 = 0; d1 < 2; ++d1) {
            int i1 = a1 + d1;
            if (i1 < 0 || i1 >= n1) continue;
            double w1 = d1 ? t1 : 1.0 - t1;
            for (int d0 = 0; d0 < 2; ++d0) {
                int i0 = a0 + d0;
                if (i0 < 0 || i0 >= n0) continue;
                double w0 = d0 ? t0 : 1.0 - t0;
                s += w2 * w1 * w0 * V[((long)i2 * n1 + i1) * n0 + i0];
            }
        }
    }
    return s;
}

/* Adjoint of trilinear(): V[...] += val * weight */
static void trilinear_T(double *V, int n0, int n1, int n2, double f0, double f1, double f2, double val)
{
    double fl0 = floor(f0), fl1 = floor(f1), fl2 = floor(f2);
    int a0 = (int)fl0, a1 = (int)fl1, a2 = (int)fl2;
    double t0 = f0 - fl0, t1 = f1 - fl1, t2 = f2 - fl2;
    for (int d2 = 0; d2 < 2; ++d2) {
        int i2 = a2 + d2;
        if (i2 < 0 || i2 >= n2) continue;
        double w2 = d2 ? t2 : 1.0 - t2;
        for (int d1 = 0; d1 < 2; ++d1) {
            int i1 = a1 + d1;
            if (i1 < 0 || i1 >= n1) continue;
            double w1 = d1 ? t1 : 1.0 - t1;
            for (int d0 = 0; d0 < 2; ++d0) {
                int i0 = a0 + d0;
                if (i0 < 0 || i0 >= n0) continue;
                double w0 = d0 ? t0 : 1.0 - t0;
                V[((long)i2 * n1 + i1) * n0 + i0] += w2 * w1 * w0 * val;
            }
        }
    }
}

/* Bilinear sample of F [nv][nu] at fractional indices (fa, fc), zero outside. */
static double bilinear2(const double *F, int nu, int nv, double fa, double fc)
{
    double fl0 = floor(fa), fl1 = floor(fc);
    int a0 = (int)fl0, c0 = (int)fl1;
    double ta = fa - fl0, tc = fc - fl1;
    double s = 0.0;
    for (int dc = 0; dc < 2; ++dc) {
        int c = c0 + dc;
        if (c < 0 || c >= nv) continue;
        for (int da = 0; da < 2; ++da) {
            int a = a0 + da;
            if (a < 0 || a >= nu) continue;
            s += (dc ? tc : 1.0 - tc) * (da ? ta : 1.0 - ta) * F[(long)c * nu + a];
        }
    }
    return s;
}

/* Adjoint of bilinear2(): F[...] += val * weight */
static void bilinear2_T(double *F, int nu, int nv, double fa, double fc, double val)
{
    double fl0 = floor(fa), fl1 = floor(fc);
    int a0 = (int)fl0, c0 = (int)fl1;
    double ta = fa - fl0, tc = fc - fl1;
    for (int dc = 0; dc < 2; ++dc) {
        int c = c0 + dc;
        if (c < 0 || c >= nv) continue;
        for (int da = 0; da < 2; ++da) {
            int a = a0 + da;
            if (a < 0 || a >= nu) continue;
            F[(long)c * nu + a] += (dc ? tc : 1.0 - tc) * (da ? ta : 1.0 - ta) * val;
        }
    }
}

static double bilinear(const double *F, int nu, int nv, double fa, double fc)
{
    double fla = floor(fa), flc = floor(fc);
    int a0 = (int)fla, c0 = (int)flc;
    double ta = fa - fla, tc = fc - flc;
    double s = 0.0;
    for (int dc = 0; dc < 2; ++dc) {
        int c = c0 + dc;
        if (c < 0 || c >= nv) continue;
        double wc = dc ? tc : 1.0 - tc;
        for (int da = 0; da < 2; ++da) {
            int a = a0 + da;
            if (a < 0 || a >= nu) continue;
            double wa = da ? ta : 1.0 - ta;
            s += wc * wa * F[(long)c * nu + a];
        }
    }
    return s;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2.4, Eq. (WEPL): z(x) = integral of rho_rel along the central ray. */
/* Reading: samples at the beam-slice centres s_k = iso + w_k e_w, trilinear */
/* density (zero outside the grid), midpoint cumulative sum                  */
/*   z_k = dw (sum_{m<k} rho_m + rho_k / 2).                                 */
/* ------------------------------------------------------------------------ */
void orc_wepl(const orc_grid *g, const orc_plan *p, const orc_lattice *L, int b, double *z)
{
    double eu[3], ev[3], ew[3];
    orc_beam_axes(p->gantry_deg[b], eu, ev, ew);
    double acc = 0.0;
    for (int k = 0; k < L->nw; ++k) {
        double w = (k - L->cw) * L->du;
        double s[3];
        for (int d = 0; d < 3; ++d) s[d] = p->iso[d] + w * ew[d];
        double rho = trilinear(g->red, g->nx, g->ny, g->nz,
                               (s[0] - g->origin[0]) / g->sx,
                               (s[1] - g->origin[1]) / g->sy,
                               (s[2] - g->origin[2]) / g->sz);
        z[k] = L->du * (acc + 0.5 * rho);
        acc += rho;
    }
}

/* Depth dose T(z): linear interpolation in the commissioned table, clamped
 * at both ends (reading of "percent depth dose", Sec. 2.4, applied per slice). */
double orc_depth_dose(const orc_plan *p, double z)
{
    double t = z / p->dz_t;
    if (t <= 0.0) return p->t_table[0];
    if (t >= (double)(p->n_t - 1)) return p->t_table[p->n_t - 1];
    double fl = floor(t);
    int m = (int)fl;
    double f = t - fl;
    return p->t_table[m] + f * (p->t_table[m + 1] - p->t_table[m]);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2.5: radially symmetric depth-dependent kernel.  Reading: three    */
/* radial exponentials whose decay a_c(z) and weight w_c(z) are quadratic    */
/* polynomials in the radiological depth, each component normalised to unit  */
/* sum over the discrete (2R+1)^2 window:                                    */
/*   K(p,q;z) = sum_c w_c(z) exp(-a_c(z) r_pq) / S_c(z),                     */
/*   r_pq = sqrt((p du)^2 + (q dv)^2),  S_c = sum_window exp(-a_c r_pq).     */
/* ------------------------------------------------------------------------ */
void orc_kernel_params(const orc_plan *p, double z, double a[3], double w[3])
{
    double wr[3], W = 0.0;
    for (int c = 0; c < 3; ++c) {
        a[c] = p->alpha[c][0] + p->alpha[c][1] * z + p->alpha[c][2] * z * z;
        if (a[c] < 1e-4) a[c] = 1e-4;
        wr[c] = p->beta[c][0] + p->beta[c][1] * z + p->beta[c][2] * z * z;
        if (wr[c] < 0.0) wr[c] = 0.0;
        W += wr[c];
    }
    for (int c = 0; c < 3; ++c) w[c] = (W > 0.0) ? wr[c] / W : 0.0;
}

/* K[(p+R)(2R+1) + (q+R)], p along u, q along v */
void orc_kernel(const orc_plan *p, const orc_lattice *L, double z, double *K)
{
    int R = p->r_px, n = 2 * R + 1;
    double a[3], w[3], S[3] = {0.0, 0.0, 0.0};
    orc_kernel_params(p, z, a, w);
    for (int pp = -R; pp <= R; ++pp)
        for (int q = -R; q <= R; ++q) {
            double r = sqrt((pp * L->du) * (pp * L->du) + (q * L->dv) * (q * L->dv));
            for (int c = 0; c < 3; ++c) S[c] += exp(-a[c] * r);
        }
    for (int pp = -R; pp <= R; ++pp)
        for (int q = -R; q <= R; ++q) {
            double r = sqrt((pp * L->du) * (pp * L->du) + (q * L->dv) * (q * L->dv));
            double k = 0.0;
            for (int c = 0; c < 3; ++c) k += w[c] * exp(-a[c] * r) / S[c];
            K[(pp + R) * n + (q + R)] = k;
        }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2.3 (FluenceVolumeLayer): Phi_k(i,j) = C(d_k) F(u(d_k)) with       */
/* u(d) = (SID/d) x_perp sampled bilinearly and C(d) = (SID/d)^2; reading:   */
/* d_k = SID + w_k, the axial distance of beam slice k.                      */
/* ------------------------------------------------------------------------ */
void orc_magnify(const orc_plan *p, const orc_lattice *L, const double *F, double *Phi)
{
#pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < L->nw; ++k) {
        double w = (k - L->cw) * L->du;
        double m = p->sid / (p->sid + w);
        double C = m * m;
        for (int j = 0; j < L->nv; ++j) {
            double fc = m * (j - L->cv) + L->cv;
            for (int i = 0; i < L->nu; ++i) {
                double fa = m * (i - L->cu) + L->cu;
                Phi[((long)k * L->nv + j) * L->nu + i] = C * bilinear(F, L->nu, L->nv, fa, fc);
            }
        }
    }
}

/* Transpose of orc_magnify: Fadj += sum over lattice points of C w Phiadj.
 * Serial scatter (exact transpose of the bilinear weights above). */
void orc_magnify_T(const orc_plan *p, const orc_lattice *L, const double *Phi_adj,
                   const unsigned char *mask, double *F_adj)
{
    for (int k = 0; k < L->nw; ++k) {
        double w = (k - L->cw) * L->du;
        double m = p->sid / (p->sid + w);
        double C = m * m;
        for (int j = 0; j < L->nv; ++j) {
            double fc = m * (j - L->cv) + L->cv;
            double flc = floor(fc);
            int c0 = (int)flc;
            double tc = fc - flc;
            for (int i = 0; i < L->nu; ++i) {
                long idx = ((long)k * L->nv + j) * L->nu + i;
                if (mask && !mask[idx]) continue;
                double val = Phi_adj[idx];
                if (val == 0.0) continue;
                double fa = m * (i - L->cu) + L->cu;
                double fla = floor(fa);
                int a0 = (int)fla;
                double ta = fa - fla;
                for (int dc = 0; dc < 2; ++dc) {
                    int c = c0 + dc;
                    if (c < 0 || c >= L->nv) continue;
                    double wc = dc ? tc : 1.0 - tc;
                    for (int da = 0; da < 2; ++da) {
                        int a = a0 + da;
                        if (a < 0 || a >= L->nu) continue;
                        double wa = da ? ta : 1.0 - ta;
                        F_adj[(long)c * L->nu + a] += C * wc * wa * val;
                    }
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2.6, Eq. (convolution), one grouped 2-D convolution per depth      */
/* slice ("same" size, zero padding):                                        */
/*   D'_k(i,j) = T(z_k) sum_{|p|,|q|<=R} Phi_k(i-p, j-q) K(p,q; z_k).        */
/* brute = 0 skips the taps whose input lies outside the bounding box of the */
/* non-zero Phi_k (those terms are exactly zero, so the sum is bit-equal).   */
/* ------------------------------------------------------------------------ */
void orc_conv(const orc_plan *p, const orc_lattice *L, const double *z,
              const double *Phi, double *Dp, int brute)
{
    int R = p->r_px, n = 2 * R + 1;
    int nu = L->nu, nv = L->nv;
#pragma omp parallel
    {
        double *K = (double *)malloc(sizeof(double) * n * n);
#pragma omp for schedule(dynamic)
        for (int k = 0; k < L->nw; ++k) {
            const double *P = Phi + (long)k * nv * nu;
            double *O = Dp + (long)k * nv * nu;
            int ia = nu, ib = -1, ja = nv, jb = -1;
            if (!brute) {
                for (int j = 0; j < nv; ++j)
                    for (int i = 0; i < nu; ++i)
                        if (P[(long)j * nu + i] != 0.0) {
                            if (i < ia) ia = i;
                            if (i > ib) ib = i;
                            if (j < ja) ja = j;
                            if (j > jb) jb = j;
                        }
                if (ib < 0) {
                    memset(O, 0, sizeof(double) * nu * nv);
                    continue;
                }
            } else {
                ia = 0; ib = nu - 1; ja = 0; jb = nv - 1;
            }
            orc_kernel(p, L, z[k], K);
            double T = orc_depth_dose(p, z[k]);
            for (int j = 0; j < nv; ++j)
                for (int i = 0; i < nu; ++i) {
                    double s = 0.0;
                    int p0 = i - ib, p1 = i - ia, q0 = j - jb, q1 = j - ja;
                    if (p0 < -R) p0 = -R;
                    if (p1 > R) p1 = R;
                    if (q0 < -R) q0 = -R;
                    if (q1 > R) q1 = R;
                    for (int pp = p0; pp <= p1; ++pp) {
                        int ii = i - pp;
                        if (ii < 0 || ii >= nu) continue;
                        for (int q = q0; q <= q1; ++q) {
                            int jj = j - q;
                            if (jj < 0 || jj >= nv) continue;
                            s += P[(long)jj * nu + ii] * K[(pp + R) * n + (q + R)];
                        }
                    }
                    O[(long)j * nu + i] = T * s;
                }
        }
        free(K);
    }
}

/* Transpose of orc_conv written as its own sum:
 *   hp_k(i',j') = T(z_k) sum_{p,q} h_k(i'+p, j'+q) K(p,q; z_k),
 * evaluated where mask != 0 (mask == NULL: everywhere), zero elsewhere. */
void orc_conv_T(const orc_plan *p, const orc_lattice *L, const double *z,
                const double *h, const unsigned char *mask, double *hp)
{
    int R = p->r_px, n = 2 * R + 1;
    int nu = L->nu, nv = L->nv;
#pragma omp parallel
    {
        double *K = (double *)malloc(sizeof(double) * n * n);
#pragma omp for schedule(dynamic)
        for (int k = 0; k < L->nw; ++k) {
            const double *H = h + (long)k * nv * nu;
            double *O = hp + (long)k * nv * nu;
            const unsigned char *M = mask ? mask + (long)k * nv * nu : NULL;
            int any = 0;
            if (M) {
                for (long t = 0; t < (long)nu * nv; ++t)
                    if (M[t]) { any = 1; break; }
            } else {
                any = 1;
            }
            if (!any) {
                memset(O, 0, sizeof(double) * nu * nv);
                continue;
            }
            orc_kernel(p, L, z[k], K);
            double T = orc_depth_dose(p, z[k]);
            for (int j = 0; j < nv; ++j)
                for (int i = 0; i < nu; ++i) {
                    if (M && !M[(long)j * nu + i]) {
                        O[(long)j * nu + i] = 0.0;
                        continue;
                    }
                    double s = 0.0;
                    for (int pp = -R; pp <= R; ++pp) {
                        int ii = i + pp;
                        if (ii < 0 || ii >= nu) continue;
                        for (int q = -R; q <= R; ++q) {
                            int jj = j + q;
                            if (jj < 0 || jj >= nv) continue;
                            s += H[(long)jj * nu + ii] * K[(pp + R) * n + (q + R)];
                        }
                    }
                    O[(long)j * nu + i] = T * s;
                }
        }
        free(K);
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2.7 (BeamRotationLayer + Eq. D_total): every patient voxel x       */
/* samples the beam-frame dose trilinearly at its beam coordinates           */
/*   (u,v,w) = ((x-iso).e_u, (x-iso).e_v, (x-iso).e_w)                       */
/* and D(x) += scale * sample, scale = cal * MU_b (zero outside the lattice).*/
/* ------------------------------------------------------------------------ */
void orc_gather(const orc_grid *g, const orc_plan *p, const orc_lattice *L, int b,
                const double *Dp, double scale, double *D)
{
    double eu[3], ev[3], ew[3];
    orc_beam_axes(p->gantry_deg[b], eu, ev, ew);
#pragma omp parallel for schedule(static)
    for (int iz = 0; iz < g->nz; ++iz)
        for (int iy = 0; iy < g->ny; ++iy)
            for (int ix = 0; ix < g->nx; ++ix) {
                double r[3] = {g->origin[0] + ix * g->sx - p->iso[0],
                               g->origin[1] + iy * g->sy - p->iso[1],
                               g->origin[2] + iz * g->sz - p->iso[2]};
                double u = r[0] * eu[0] + r[1] * eu[1] + r[2] * eu[2];
                double v = r[0] * ev[0] + r[1] * ev[1] + r[2] * ev[2];
                double w = r[0] * ew[0] + r[1] * ew[1] + r[2] * ew[2];
                double val = trilinear(Dp, L->nu, L->nv, L->nw,
                                       u / L->du + L->cu, v / L->dv + L->cv, w / L->du + L->cw);
                D[((long)iz * g->ny + iy) * g->nx + ix] += scale * val;
            }
}

/* Transpose of orc_gather (scale 1): h[lattice] += weight * gd[x]. Serial. */
void orc_gather_T(const orc_grid *g, const orc_plan *p, const orc_lattice *L, int b,
                  const double *gd, double *h)
{
    double eu[3], ev[3], ew[3];
    orc_beam_axes(p->gantry_deg[b], eu, ev, ew);
    for (int iz = 0; iz < g->nz; ++iz)
        for (int iy = 0; iy < g->ny; ++iy)
            for (int ix = 0; ix < g->nx; ++ix) {
                double val = gd[((long)iz * g->ny + iy) * g->nx + ix];
                if (val == 0.0) continue;
                double r[3] = {g->origin[0] + ix * g->sx - p->iso[0],
                               g->origin[1] + iy * g->sy - p->iso[1],
                               g->origin[2] + iz * g->sz - p->iso[2]};
                double u = r[0] * eu[0] + r[1] * eu[1] + r[2] * eu[2];
                double v = r[0] * ev[0] + r[1] * ev[1] + r[2] * ev[2];
                double w = r[0] * ew[0] + r[1] * ew[1] + r[2] * ew[2];
                trilinear_T(h, L->nu, L->nv, L->nw,
                            u / L->du + L->cu, v / L->dv + L->cv, w / L->du + L->cw, val);
            }
}

/* ------------------------------------------------------------------------ */
/* Whole forward model (Eq. D_total):                                        */
/*   D(x) = cal sum_b MU^_b  gather_b( conv_b( magnify_b( F_b ) ) )(x)       */
/* ------------------------------------------------------------------------ */
int orc_dose(const orc_grid *g, const orc_plan *p, const double *leaves, const double *jaws,
             const double *mu, double *dose, int brute)
{
    orc_lattice L;
    orc_lattice_of(g, p, &L);
    long nvox = (long)g->nx * g->ny * g->nz;
    long nvol = (long)L.nu * L.nv * L.nw;
    double *F = (double *)malloc(sizeof(double) * L.nu * L.nv);
    double *z = (double *)malloc(sizeof(double) * L.nw);
    double *Phi = (double *)malloc(sizeof(double) * nvol);
    double *Dp = (double *)malloc(sizeof(double) * nvol);
    double *lv = (double *)malloc(sizeof(double) * 2 * p->n_pairs);
    if (!F || !z || !Phi || !Dp || !lv) {
        free(F); free(z); free(Phi); free(Dp); free(lv);
        return ORC_ENOMEM;
    }
    memset(dose, 0, sizeof(double) * nvox);
    for (int b = 0; b < p->n_cp; ++b) {
        double jw[4], muh;
        orc_project_cp(p, leaves + (long)b * 2 * p->n_pairs, jaws + 4L * b, mu[b], lv, jw, &muh);
        orc_fluence(p, &L, lv, jw, F);
        orc_fluence_correct(p, &L, F);
        orc_wepl(g, p, &L, b, z);
        orc_magnify(p, &L, F, Phi);
        orc_conv(p, &L, z, Phi, Dp, brute);
        orc_gather(g, p, &L, b, Dp, p->cal * muh, dose);
    }
    free(F); free(z); free(Phi); free(Dp); free(lv);
    return ORC_OK;
}

/* Beam-frame dose D'_b (no MU, no cal) of one control point; Dp [nw][nv][nu]. */
int orc_beam_dose(const orc_grid *g, const orc_plan *p, int b, const double *leaves_cp,
                  const double *jaws_cp, double *Dp)
{
    orc_lattice L;
    orc_lattice_of(g, p, &L);
    long nvol = (long)L.nu * L.nv * L.nw;
    double *F = (double *)malloc(sizeof(double) * L.nu * L.nv);
    double *z = (double *)malloc(sizeof(double) * L.nw);
    double *Phi = (double *)malloc(sizeof(double) * nvol);
    double *lv = (double *)malloc(sizeof(double) * 2 * p->n_pairs);
    if (!F || !z || !Phi || !lv) {
        free(F); free(z); free(Phi); free(lv);
        return ORC_ENOMEM;
    }
    double jw[4], muh;
    orc_project_cp(p, leaves_cp, jaws_cp, 1.0, lv, jw, &muh);
    orc_fluence(p, &L, lv, jw, F);
    orc_fluence_correct(p, &L, F);
    orc_wepl(g, p, &L, b, z);
    orc_magnify(p, &L, F, Phi);
    orc_conv(p, &L, z, Phi, Dp, 0);
    free(F); free(z); free(Phi); free(lv);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Fluence vector-Jacobian product for one control point (raw parameters).   */
/* dF: dL/dF on the lattice [nv][nu], only read inside the jaw box           */
/* (elsewhere dF/dtheta = 0).  Accumulates into dleaves_cp [n_pairs][2] and  */
/* djaws_cp [4].  Projection Jacobian: identity if ste, else exact.          */
/* ------------------------------------------------------------------------ */
void orc_fluence_vjp(const orc_plan *p, const orc_lattice *L, const double *leaves_cp,
                     const double *jaws_cp, const double *dF, double *dleaves_cp, double *djaws_cp)
{
    int np = p->n_pairs;
    double *lv = (double *)malloc(sizeof(double) * 2 * np);
    double *gcl = (double *)malloc(sizeof(double) * np);
    double *gwl = (double *)malloc(sizeof(double) * np);
    double *dlh = (double *)calloc(2 * np, sizeof(double));
    double jw[4], gcj[2], gwj[2], djh[4] = {0, 0, 0, 0};
    for (int i = 0; i < np; ++i)
        project_pair(leaves_cp[2 * i], leaves_cp[2 * i + 1], p->wmin_leaf, p->f_leaf,
                     &lv[2 * i], &lv[2 * i + 1], &gcl[i], &gwl[i]);
    project_pair(jaws_cp[0], jaws_cp[1], p->wmin_jaw, p->f_jaw, &jw[0], &jw[1], &gcj[0], &gwj[0]);
    project_pair(jaws_cp[2], jaws_cp[3], p->wmin_jaw, p->f_jaw, &jw[2], &jw[3], &gcj[1], &gwj[1]);

    for (int c = 0; c < L->nv; ++c) {
        double v = (c - L->cv) * L->dv;
        double fy = orc_overlap(v, jw[2], jw[3], L->dv);
        double dfy_lo = overlap_dlo(v, jw[2], jw[3], L->dv);
        double dfy_hi = overlap_dhi(v, jw[2], jw[3], L->dv);
        for (int a = 0; a < L->nu; ++a) {
            double u = (a - L->cu) * L->du;
            double fx = orc_overlap(u, jw[0], jw[1], L->du);
            double dfx_lo = overlap_dlo(u, jw[0], jw[1], L->du);
            double dfx_hi = overlap_dhi(u, jw[0], jw[1], L->du);
            if (fx == 0.0 && dfx_lo == 0.0 && dfx_hi == 0.0) continue;
            if (fy == 0.0 && dfy_lo == 0.0 && dfy_hi == 0.0) continue;
            double gF = dF[(long)c * L->nu + a];
            if (gF == 0.0) continue;
            double fl = 0.0;
            for (int i = 0; i < np; ++i) {
                double om = orc_overlap(v, p->leaf_bounds[i], p->leaf_bounds[i + 1], L->dv);
                if (om > 0.0) fl += om * orc_overlap(u, lv[2 * i], lv[2 * i + 1], L->du);
            }
            double G = p->tau + (1.0 - p->tau) * fl;
            djh[0] += gF * dfx_lo * fy * G;
            djh[1] += gF * dfx_hi * fy * G;
            djh[2] += gF * fx * dfy_lo * G;
            djh[3] += gF * fx * dfy_hi * G;
            double fj = fx * fy;
            if (fj == 0.0) continue;
            for (int i = 0; i < np; ++i) {
                double om = orc_overlap(v, p->leaf_bounds[i], p->leaf_bounds[i + 1], L->dv);
                if (om <= 0.0) continue;
                double s = gF * fj * (1.0 - p->tau) * om;
                dlh[2 * i] += s * overlap_dlo(u, lv[2 * i], lv[2 * i + 1], L->du);
                dlh[2 * i + 1] += s * overlap_dhi(u, lv[2 * i], lv[2 * i + 1], L->du);
            }
        }
    }
    /* Projection Jacobian (Sec. 2.2.1). */
    for (int i = 0; i < np; ++i) {
        double ga = dlh[2 * i], gb = dlh[2 * i + 1];
        if (p->ste) {
            dleaves_cp[2 * i] += ga;
            dleaves_cp[2 * i + 1] += gb;
        } else {
            double s = 0.5 * (gcl[i] + gwl[i]), d = 0.5 * (gcl[i] - gwl[i]);
            dleaves_cp[2 * i] += ga * s + gb * d;
            dleaves_cp[2 * i + 1] += ga * d + gb * s;
        }
    }
    for (int pr = 0; pr < 2; ++pr) {
        double ga = djh[2 * pr], gb = djh[2 * pr + 1];
        if (p->ste) {
            djaws_cp[2 * pr] += ga;
            djaws_cp[2 * pr + 1] += gb;
        } else {
            double s = 0.5 * (gcj[pr] + gwj[pr]), d = 0.5 * (gcj[pr] - gwj[pr]);
            djaws_cp[2 * pr] += ga * s + gb * d;
            djaws_cp[2 * pr + 1] += ga * d + gb * s;
        }
    }
    free(lv); free(gcl); free(gwl); free(dlh);
}

/* ------------------------------------------------------------------------ */
/* Whole adjoint.  With A_b the linear map F_b -> MU-free dose of CP b,      */
/*   dL/dF_b  = cal MU^_b A_b^T g,   dL/dMU^_b = cal <A_b^T g, F_b>,          */
/*   A_b^T = magnify^T conv^T gather^T.                                      */
/* A_b^T g is only needed inside the jaw box (where F_b and dF_b/dtheta are  */
/* non-zero); conv^T is evaluated at the lattice points whose magnified      */
/* bilinear stencil touches that box.                                        */
/* dose_out (optional) receives the forward dose.                            */
/* ------------------------------------------------------------------------ */
int orc_dose_grad(const orc_grid *g, const orc_plan *p, const double *leaves, const double *jaws,
                  const double *mu, const double *gdose, double *dleaves, double *djaws,
                  double *dmu)
{
    orc_lattice L;
    orc_lattice_of(g, p, &L);
    long nvol = (long)L.nu * L.nv * L.nw;
    long nF = (long)L.nu * L.nv;
    int np = p->n_pairs;
    double *F = (double *)malloc(sizeof(double) * nF);
    double *gF = (double *)malloc(sizeof(double) * nF);
    double *z = (double *)malloc(sizeof(double) * L.nw);
    double *h = (double *)malloc(sizeof(double) * nvol);
    double *hp = (double *)malloc(sizeof(double) * nvol);
    unsigned char *mask = (unsigned char *)malloc(nvol);
    double *lv = (double *)malloc(sizeof(double) * 2 * np);
    if (!F || !gF || !z || !h || !hp || !mask || !lv) {
        free(F); free(gF); free(z); free(h); free(hp); free(mask); free(lv);
        return ORC_ENOMEM;
    }
    memset(dleaves, 0, sizeof(double) * 2 * np * p->n_cp);
    memset(djaws, 0, sizeof(double) * 4 * p->n_cp);
    for (int b = 0; b < p->n_cp; ++b) {
        double jw[4], muh;
        const double *lc = leaves + (long)b * 2 * np;
        const double *jc = jaws + 4L * b;
        orc_project_cp(p, lc, jc, mu[b], lv, jw, &muh);
        orc_fluence(p, &L, lv, jw, F);
        orc_fluence_correct(p, &L, F);
        orc_wepl(g, p, &L, b, z);
        /* jaw box in lattice pixels, widened by the penumbra blur radius (the
         * corrected fluence and the raw fluence's sensitivities live there) */
        int a0 = L.nu, a1 = -1, c0 = L.nv, c1 = -1;
        for (int a = 0; a < L.nu; ++a)
            if (orc_overlap((a - L.cu) * L.du, jw[0], jw[1], L.du) > 0.0) {
                if (a < a0) a0 = a;
                if (a > a1) a1 = a;
            }
        for (int c = 0; c < L.nv; ++c)
            if (orc_overlap((c - L.cv) * L.dv, jw[2], jw[3], L.dv) > 0.0) {
                if (c < c0) c0 = c;
                if (c > c1) c1 = c;
            }
        if (a1 >= 0 && c1 >= 0 && p->coll_deg != 0.0) {
            /* a turned map can reach any pixel: take the whole lattice */
            a0 = 0; a1 = L.nu - 1; c0 = 0; c1 = L.nv - 1;
        } else if (a1 >= 0 && c1 >= 0) {
            int ru = orc_penumbra_radius(p->pen_fwhm_u, L.du), rv = orc_penumbra_radius(p->pen_fwhm_v, L.dv);
            a0 = a0 - ru < 0 ? 0 : a0 - ru;
            a1 = a1 + ru >= L.nu ? L.nu - 1 : a1 + ru;
            c0 = c0 - rv < 0 ? 0 : c0 - rv;
            c1 = c1 + rv >= L.nv ? L.nv - 1 : c1 + rv;
        }
        double dmuh = 0.0;
        if (a1 >= 0 && c1 >= 0) {
            memset(h, 0, sizeof(double) * nvol);
            orc_gather_T(g, p, &L, b, gdose, h);
            /* mask: lattice points whose magnified stencil touches the box */
            for (int k = 0; k < L.nw; ++k) {
                double w = (k - L.cw) * L.du;
                double m = p->sid / (p->sid + w);
                for (int j = 0; j < L.nv; ++j) {
                    double fc = m * (j - L.cv) + L.cv;
                    int cl = (int)floor(fc);
                    int hitc = (cl + 1 >= c0 && cl <= c1);
                    for (int i = 0; i < L.nu; ++i) {
                        double fa = m * (i - L.cu) + L.cu;
                        int al = (int)floor(fa);
                        mask[((long)k * L.nv + j) * L.nu + i] =
                            (unsigned char)(hitc && al + 1 >= a0 && al <= a1);
                    }
                }
            }
            orc_conv_T(p, &L, z, h, mask, hp);
            memset(gF, 0, sizeof(double) * nF);
            orc_magnify_T(p, &L, hp, mask, gF);
            /* restrict to the box, MU gradient on the corrected fluence */
            for (int c = 0; c < L.nv; ++c)
                for (int a = 0; a < L.nu; ++a) {
                    long t = (long)c * L.nu + a;
                    if (a < a0 || a > a1 || c < c0 || c > c1) {
                        gF[t] = 0.0;
                        continue;
                    }
                    dmuh += p->cal * gF[t] * F[t];
                    gF[t] *= p->cal * muh;
                }
            /* back through the corrections to the raw aperture fluence */
            orc_fluence_correct_T(p, &L, gF);
            orc_fluence_vjp(p, &L, lc, jc, gF, dleaves + (long)b * 2 * np, djaws + 4L * b);
        }
        dmu[b] = (p->ste || mu[b] >= p->eps_mu) ? dmuh : 0.0;
    }
    free(F); free(gF); free(z); free(h); free(hp); free(mask); free(lv);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Output calibration (Sec. 2.4): the factor cal that makes ref_mu MU of the  */
/* reference field give ref_gy Gy at the reference point of a virtual water   */
/* phantom.  The paper names the reference conditions (10 cm x 10 cm field,   */
/* 10 cm depth in water, SSD 90 cm) and says the dose there is computed with  */
/* the beam model and the scaling factor adjusted; the discrete set-up is a   */
/* reading:                                                                   */
/*   - the reference point is the isocentre, 100 mm below the water surface   */
/*     on the central axis, gantry 0 (SSD = SID - 100 mm: 90 cm at SID 1 m);  */
/*   - the field is 100 mm x 100 mm at the isocentre plane: jaws (-50, 50,    */
/*     -50, 50) and every leaf pair at (-50, 50); collimator 0; the beam      */
/*     model's penumbra and off-axis profile apply;                           */
/*   - voxels sxy x sxy x sz (the patient grid's pitch, so the kernel's pixel  */
/*     radius means the same), the isocentre on a voxel centre; a voxel row   */
/*     whose centre is y holds the water fraction of its extent              */
/*     clamp((y + sxy/2 + 100) / sxy, 0, 1) as relative electron density, so   */
/*     the midpoint depth sum (Sec. 2.2.4) at the isocentre is 100 mm exactly  */
/*     at any pitch;                                                          */
/*   - the grid reaches sqrt(2) R + penumbra half-window + 2 pixels beyond    */
/*     the central axis in x and z, 100 mm + 2 voxels above the isocentre and */
/*     2 voxels below it, so every pixel the isocentre's dose reads is on the */
/*     lattice.                                                               */
/* cal = ref_gy / D(isocentre) with D computed at cal = 1.  Also returns the  */
/* WEPL of the reference slice and D per MU.                                  */
/* ------------------------------------------------------------------------ */
int orc_calibrate(const orc_plan *machine, double sxy, double sz, double ref_mu, double ref_gy,
                  double *cal_out, double *z_ref_out, double *dose_per_mu_out)
{
    if (!(sxy > 0) || !(sz > 0) || !(ref_mu > 0) || !(ref_gy > 0)) return ORC_EINVAL;
    const int R = machine->r_px;
    const double rad_mm = R * sqrt(sxy * sxy + sz * sz);
    const int hx = (int)ceil(rad_mm / sxy) + orc_penumbra_radius(machine->pen_fwhm_u, sxy) + 2;
    const int hz = (int)ceil(rad_mm / sz) + orc_penumbra_radius(machine->pen_fwhm_v, sz) + 2;
    const int n_above = (int)ceil(100.0 / sxy + 0.5) + 2;   /* rows above the isocentre */
    const int nx = 2 * hx + 1, nz = 2 * hz + 1, ny = n_above + 1 + 2;
    double *red = (double *)malloc(sizeof(double) * (size_t)nx * ny * nz);
    double *dose = (double *)malloc(sizeof(double) * (size_t)nx * ny * nz);
    double *leaves = (double *)malloc(sizeof(double) * 2 * (machine->n_pairs > 0 ? machine->n_pairs : 1));
    double *z = NULL;
    if (!red || !dose || !leaves) {
        free(red); free(dose); free(leaves);
        return ORC_ENOMEM;
    }
    for (int j = 0; j < ny; ++j) {
        double y = (j - n_above) * sxy;   /* row centre, mm; isocentre row j = n_above */
        double f = (y + 0.5 * sxy + 100.0) / sxy;
        f = f < 0.0 ? 0.0 : (f > 1.0 ? 1.0 : f);
        for (int k = 0; k < nz; ++k)
            for (int i = 0; i < nx; ++i) red[((size_t)k * ny + j) * nx + i] = f;
    }
    orc_grid g;
    g.nx = nx; g.ny = ny; g.nz = nz;
    g.sx = sxy; g.sy = sxy; g.sz = sz;
    g.origin[0] = -hx * sxy; g.origin[1] = -n_above * sxy; g.origin[2] = -hz * sz;
    g.red = red;
    orc_plan p = *machine;
    double gantry = 0.0;
    p.n_cp = 1;
    p.gantry_deg = &gantry;
    p.iso[0] = p.iso[1] = p.iso[2] = 0.0;
    p.cal = 1.0;
    p.coll_deg = 0.0;
    for (int i = 0; i < p.n_pairs; ++i) {
        leaves[2 * i] = -50.0;
        leaves[2 * i + 1] = 50.0;
    }
    double jaws[4] = {-50.0, 50.0, -50.0, 50.0};
    int rc = orc_dose(&g, &p, leaves, jaws, &ref_mu, dose, 0);
    if (rc == ORC_OK) {
        double d_ref = dose[((size_t)hz * ny + n_above) * nx + hx];
        if (!(d_ref > 0)) {
            rc = ORC_EINVAL;
        } else {
            *cal_out = ref_gy / d_ref;
            if (dose_per_mu_out) *dose_per_mu_out = d_ref / ref_mu;
            if (z_ref_out) {
                orc_lattice L;
                orc_lattice_of(&g, &p, &L);
                z = (double *)malloc(sizeof(double) * L.nw);
                if (!z) {
                    rc = ORC_ENOMEM;
                } else {
                    orc_wepl(&g, &p, &L, 0, z);
                    *z_ref_out = z[(int)L.cw];
                }
            }
        }
    }
    free(red); free(dose); free(leaves); free(z);
    return rc;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
