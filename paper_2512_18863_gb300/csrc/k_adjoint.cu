// Adjoint tail of the dose engine.
//
// k_mag_T: transpose of the divergent fluence projection (Sec. 2.2.3): every
//   fluence pixel of the support box pulls, over all beam slices, the adjoint
//   convolution output h'_k at the lattice points whose magnified bilinear
//   stencil contains the pixel (weights recomputed with mag_coord, the same
//   expression the forward tile fill uses).  No atomics.
// k_param_grad: chain rule of the fluence map (Sec. 2.2.2, piecewise-linear
//   overlap, derivative taken one-sided at pixel boundaries) and of the
//   hardware projection (Sec. 2.2.1: identity if ste, exact Jacobian
//   otherwise) to leaves, jaws and MU:
//     dL/dF_b   = cal MU^_b g_F,   dL/dMU^_b = cal <g_F, F_b>.
#include <math.h>

#include "pdrt_impl.cuh"

namespace pdrt {

constexpr int kMtA = 16, kMtC = 16;   // pixel tile of a CTA (a, c)
constexpr int kMtS = 32;               // slices per table batch
constexpr int kMtTaps = 4;             // non-zero lattice taps per pixel and axis, at most

struct MagSlice {
    float m, inv_m;   // magnification and 1 / m (staged once per slice)
    int ai0, ai1, aj0, aj1;
    long long off_a;
};

// One pixel's taps along one axis for one slice: lattice indices lo, lo + 1,
// ... with weights w[] (zero where no tap).  A lattice point idx samples the
// pixels floor(f) and floor(f) + 1 of f = mag_coord(m, idx, c); p gets a
// non-zero weight only for f in (p - 1, p + 1), an open interval of length 2
// holding at most ceil(2 / m) < 4 points (m > 1/2: the plan's source distance
// exceeds the lattice reach), and those points are consecutive.
struct MagTap {
    int lo;
    float w[kMtTaps];
};

// candidate lattice indices idx with |mag_coord(m, idx, c) - p| < 1, widened
// by a small margin (the exact weights decide); inv = 1 / m
__device__ __forceinline__ void mag_candidates(int p, float c, float inv, int lo_box, int hi_box,
                                               int &lo, int &hi)
{
    lo = max((int)floorf(c + ((float)p - 1.f - c) * inv - 1e-3f) + 1, lo_box);
    hi = min((int)ceilf(c + ((float)p + 1.f - c) * inv + 1e-3f), hi_box);   // exclusive
}

// taps of pixel p over the lattice indices [lo_box, hi_box) of one slice
__device__ __forceinline__ MagTap mag_taps(int p, float c, const MagSlice &e, int lo_box, int hi_box)
{
    MagTap t;
    t.lo = 0;
#pragma unroll
    for (int q = 0; q < kMtTaps; ++q) t.w[q] = 0.f;
    int lo, hi;
    mag_candidates(p, c, e.inv_m, lo_box, hi_box, lo, hi);
    int first = -1;
    for (int idx = lo; idx < hi; ++idx) {
        const float f = mag_coord(e.m, idx, c);
        const float bf = floorf(f);
        const int p0 = (int)bf;
        const float tf = f - bf;
        const float w = (p == p0) ? 1.f - tf : ((p == p0 + 1) ? tf : 0.f);
        if (w == 0.f) continue;
        if (first < 0) {
            first = idx;
            t.lo = idx;
        }
        if (idx - first < kMtTaps) t.w[idx - first] = w;
    }
    return t;
}

// Pull form: a CTA owns a 16 x 16 tile of fluence pixels of one control point
// and sweeps the slices in batches; per batch it tabulates the taps of its 16
// pixel rows and 16 pixel columns (they are separable), then each pixel sums
//   sum_j wc(c, j) sum_i wa(a, i) h'(i, j)
// slice by slice, j then i in increasing order (non-zero terms only).
// The kernel waits mostly on its h' loads, so it is bounded to 32 registers
// for eight resident CTAs (64 warps) per SM instead of six.
__global__ void __launch_bounds__(256, 8) k_mag_T(PlanDev P, int b0)
{
    const Lattice &L = P.lat;
    const int bl = blockIdx.x, b = b0 + bl;
    const CpTab ct = P.cptab[b];
    const int Fa = ct.fa1 - ct.fa0, Fc = ct.fc1 - ct.fc0;
    if (Fa <= 0 || Fc <= 0) return;
    __shared__ MagSlice s_sl[kMtS];
    __shared__ MagTap s_ta[kMtS][kMtA];
    __shared__ MagTap s_tc[kMtS][kMtC];
    float *gF = P.gfbuf + (long long)b * L.nu * L.nv;
    const float *hb = P.adjbuf + (long long)bl * P.cap_a;
    const SliceTab *sl = P.slices + (long long)b * L.nw;
    const int nta = (Fa + kMtA - 1) / kMtA, ntc = (Fc + kMtC - 1) / kMtC;
    const int la = (int)threadIdx.x % kMtA, lc = (int)threadIdx.x / kMtA;   // 16 x 16 threads
    for (int tile = blockIdx.y; tile < nta * ntc; tile += gridDim.y) {
        const int ta0 = (tile % nta) * kMtA, tc0 = (tile / nta) * kMtC;
        const int a = ct.fa0 + ta0 + la, c = ct.fc0 + tc0 + lc;
        const bool inside = ta0 + la < Fa && tc0 + lc < Fc;
        float s = 0.f;
        for (int kc = ct.k0; kc < ct.k1; kc += kMtS) {
            const int kn = min(kMtS, ct.k1 - kc);
            __syncthreads();   // the previous batch's tables are no longer read
            for (int q = threadIdx.x; q < kn; q += blockDim.x) {
                const SliceTab *sp = sl + kc + q;
                MagSlice e;
                e.m = sp->m;
                e.inv_m = 1.f / e.m;
                e.ai0 = sp->ai0; e.ai1 = sp->ai1; e.aj0 = sp->aj0; e.aj1 = sp->aj1;
                e.off_a = sp->off_a;
                s_sl[q] = e;
            }
            __syncthreads();
            for (int q = threadIdx.x; q < kn * (kMtA + kMtC); q += blockDim.x) {
                const int ks = q / (kMtA + kMtC), r = q - ks * (kMtA + kMtC);
                const MagSlice e = s_sl[ks];
                const bool live = e.ai1 > e.ai0 && e.aj1 > e.aj0;
                if (r < kMtA) {
                    MagTap t = live ? mag_taps(ct.fa0 + ta0 + r, L.cu, e, e.ai0, e.ai1) : MagTap{0, {0.f, 0.f, 0.f, 0.f}};
                    s_ta[ks][r] = t;
                } else {
                    MagTap t = live ? mag_taps(ct.fc0 + tc0 + r - kMtA, L.cv, e, e.aj0, e.aj1)
                                    : MagTap{0, {0.f, 0.f, 0.f, 0.f}};
                    s_tc[ks][r - kMtA] = t;
                }
            }
            __syncthreads();
            if (inside) {
                for (int ks = 0; ks < kn; ++ks) {
                    const MagTap tc = s_tc[ks][lc];
                    const MagTap ta = s_ta[ks][la];
                    const MagSlice &e = s_sl[ks];
                    const float *h = hb + e.off_a;
                    const int aw = e.ai1 - e.ai0;
#pragma unroll
                    for (int jt = 0; jt < kMtTaps; ++jt) {
                        const float wc = tc.w[jt];
                        if (wc == 0.f) continue;
                        const float *hr = h + (long long)(tc.lo + jt - e.aj0) * aw + (ta.lo - e.ai0);
                        float sr = 0.f;
#pragma unroll
                        for (int it = 0; it < kMtTaps; ++it)
                            if (ta.w[it] != 0.f) sr = fmaf(ta.w[it], hr[it], sr);
                        s = fmaf(wc, sr, s);
                    }
                }
            }
        }
        // every pixel of the tile is written (zero when no slice has work)
        if (inside) gF[(long long)(a - ct.fa0) * Fc + (c - ct.fc0)] = s;
    }
}

cudaError_t launch_mag_T(const PlanDev &P, int b0, int nb, cudaStream_t s)
{
    dim3 grid(nb, 24);   // pixel tiles of a control point, strided over blockIdx.y
    k_mag_T<<<grid, 256, 0, s>>>(P, b0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ void project_pair_grad(float pa, float pb, float wmin, float F, float &ah,
                                                  float &bh, float &gc, float &gw)
{
    float c = 0.5f * (pa + pb);
    float w = pb - pa;
    float w2 = (w >= wmin) ? w : wmin;
    float c1 = (c >= -F) ? c : -F;
    float c2 = (c1 <= F) ? c1 : F;
    ah = c2 - 0.5f * w2;
    bh = c2 + 0.5f * w2;
    gw = (w >= wmin) ? 1.f : 0.f;
    gc = ((c >= -F) ? 1.f : 0.f) * ((c1 <= F) ? 1.f : 0.f);
}

// one-sided derivatives of the overlap w.r.t. its upper / lower edge
__device__ __forceinline__ float overlap_dhi(float x, float lo, float hi, float d)
{
    float e = x + 0.5f * d, s = x - 0.5f * d;
    float top = (hi <= e) ? hi : e;
    float bot = (lo >= s) ? lo : s;
    return (top - bot > 0.f && hi <= e) ? 1.f / d : 0.f;
}

__device__ __forceinline__ float overlap_dlo(float x, float lo, float hi, float d)
{
    float e = x + 0.5f * d, s = x - 0.5f * d;
    float top = (hi <= e) ? hi : e;
    float bot = (lo >= s) ? lo : s;
    return (top - bot > 0.f && lo >= s) ? -1.f / d : 0.f;
}

template <int N>
__device__ void block_sum(float (&v)[N], float *s_red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < N; ++q) {
        float x = v[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) s_red[wid * N + q] = x;
    }
    __syncthreads();
    if (threadIdx.x < N) {
        float x = 0.f;
        for (int w = 0; w < nwarp; ++w) x += s_red[w * N + threadIdx.x];
        s_red[32 * N + threadIdx.x] = x;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < N; ++q) v[q] = s_red[32 * N + q];
    __syncthreads();
}

// Adjoint of the fluence corrections (collimator rotation, off-axis profile,
// then the penumbra blurs; transposes in reverse order) for control point b:
// reads the fluence adjoint in gfbuf over the final box, leaves the raw-map
// adjoint in fbuf over the raw box (the corrected map there is no longer
// needed).  The rotation transpose is a pull: every pixel of the blurred box
// sums the final pixels whose bilinear source stencil contains it, with the
// forward's own weights (rotation_source).  One block per control point.
__device__ void uncorrect_adjoint(const PlanDev &P, int b, const CpTab &ct)
{
    const MachineDev &M = P.mach;
    const Lattice &L = P.lat;
    const long long slot = (long long)b * L.nu * L.nv;
    const int Ca = ct.ca1 - ct.ca0, Cc = ct.cc1 - ct.cc0;
    const int Fc = ct.fc1 - ct.fc0;
    float *gF = P.gfbuf + slot;
    float *gb;   // OAP-weighted adjoint of the blurred map over the blurred box
    __syncthreads();   // every thread is done reading gF for dMU
    if (M.rot) {
        gb = P.tbuf + slot;
        // (a, c) - iso = Minv ((fa, fc) - iso), Minv = [[cos, -sin r], [sin / r, cos]], r = dv/du
        const float r = L.dv / L.du;
        const float ha = fabsf(M.rot_c) + fabsf(M.rot_s) * r + 0.01f;
        const float hc = fabsf(M.rot_s) / r + fabsf(M.rot_c) + 0.01f;
        for (int t = threadIdx.x; t < Ca * Cc; t += blockDim.x) {
            const int ap = ct.ca0 + t / Cc, cp = ct.cc0 + t % Cc;
            const float xa = (float)ap - L.cu, xc = (float)cp - L.cv;
            const float a_s = L.cu + M.rot_c * xa - M.rot_s * r * xc;
            const float c_s = L.cv + M.rot_s / r * xa + M.rot_c * xc;
            const int alo = max((int)ceilf(a_s - ha), ct.fa0), ahi = min((int)floorf(a_s + ha), ct.fa1 - 1);
            const int clo = max((int)ceilf(c_s - hc), ct.fc0), chi = min((int)floorf(c_s + hc), ct.fc1 - 1);
            float s = 0.f;
            for (int c = clo; c <= chi; ++c)
                for (int a = alo; a <= ahi; ++a) {
                    float fa, fc;
                    rotation_source(M, L, a, c, fa, fc);
                    const float ba = floorf(fa), bc = floorf(fc);
                    const int ia = (int)ba, ic = (int)bc;
                    const float wa = (ap == ia) ? 1.f - (fa - ba) : ((ap == ia + 1) ? fa - ba : 0.f);
                    const float wc = (cp == ic) ? 1.f - (fc - bc) : ((cp == ic + 1) ? fc - bc : 0.f);
                    if (wa != 0.f && wc != 0.f)
                        s = fmaf(wa * wc, gF[(long long)(a - ct.fa0) * Fc + (c - ct.fc0)], s);
                }
            gb[t] = s * off_axis_factor(M, L, ap, cp);
        }
    } else {
        gb = gF;   // final box = blurred box
        for (int t = threadIdx.x; t < Ca * Cc; t += blockDim.x)
            gb[t] *= off_axis_factor(M, L, ct.ca0 + t / Cc, ct.cc0 + t % Cc);
    }
    __syncthreads();
    // transposed blurs: raw(a, c) <- sum_s gv[s] sum_t gu[t] gb(a + t, c + s)
    float *graw = P.fbuf + slot;
    const int Ra = ct.ra1 - ct.ra0, Rc = ct.rc1 - ct.rc0;
    for (int t = threadIdx.x; t < Ra * Rc; t += blockDim.x) {
        const int a = ct.ra0 + t / Rc, c = ct.rc0 + t % Rc;
        float s = 0.f;
        for (int dv = -M.rbv; dv <= M.rbv; ++dv) {
            const int cs = c + dv;
            if (cs < ct.cc0 || cs >= ct.cc1) continue;
            float q = 0.f;
            for (int du = -M.rbu; du <= M.rbu; ++du) {
                const int as = a + du;
                if (as < ct.ca0 || as >= ct.ca1) continue;
                q = fmaf(M.gu[du + M.rbu], gb[(long long)(as - ct.ca0) * Cc + (cs - ct.cc0)], q);
            }
            s = fmaf(M.gv[dv + M.rbv], q, s);
        }
        graw[t] = s;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_param_grad(PlanDev P, const float *__restrict__ leaves,
                                                    const float *__restrict__ jaws,
                                                    const float *__restrict__ mu,
                                                    float *__restrict__ dleaves,
                                                    float *__restrict__ djaws,
                                                    float *__restrict__ dmu)
{
    const int b = blockIdx.x;
    const Lattice &L = P.lat;
    const MachineDev &M = P.mach;
    const int np = M.n_pairs;
    __shared__ float s_lo[PDRT_MAX_PAIRS], s_hi[PDRT_MAX_PAIRS], s_lb[PDRT_MAX_PAIRS + 1];
    __shared__ float s_gc[PDRT_MAX_PAIRS], s_gw[PDRT_MAX_PAIRS];
    __shared__ float s_j[4], s_jgc[2], s_jgw[2];
    __shared__ float s_red[33 * 5];
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const float pa = leaves[((long long)b * np + i) * 2], pb = leaves[((long long)b * np + i) * 2 + 1];
        project_pair_grad(pa, pb, M.wmin_leaf, M.f_leaf, s_lo[i], s_hi[i], s_gc[i], s_gw[i]);
    }
    for (int i = threadIdx.x; i <= np; i += blockDim.x) s_lb[i] = P.leaf_bounds[i];
    if (threadIdx.x == 0) {
        project_pair_grad(jaws[4LL * b], jaws[4LL * b + 1], M.wmin_jaw, M.f_jaw, s_j[0], s_j[1],
                          s_jgc[0], s_jgw[0]);
        project_pair_grad(jaws[4LL * b + 2], jaws[4LL * b + 3], M.wmin_jaw, M.f_jaw, s_j[2], s_j[3],
                          s_jgc[1], s_jgw[1]);
    }
    __syncthreads();
    const CpTab ct = P.cptab[b];
    const float dscale = ct.cal_mu;   // dL/dF = cal MU^ g_F
    const float hdv = 0.5f * L.dv;
    float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    // g: adjoint of the raw aperture map over the box [ga0,ga1) x [gc0,gc1)
    const float *g_raw;
    int ga0, ga1, gc0, gc1;
    if (M.corr) {
        // dMU^ on the corrected map, then the adjoint back through the corrections
        const int Fa = ct.fa1 - ct.fa0, Fc = ct.fc1 - ct.fc0;
        const float *gF = P.gfbuf + (long long)b * L.nu * L.nv;
        const float *F = P.fbuf + (long long)b * L.nu * L.nv;
        for (int t = threadIdx.x; t < Fa * Fc; t += blockDim.x) acc[0] = fmaf(gF[t], F[t], acc[0]);
        uncorrect_adjoint(P, b, ct);
        g_raw = P.fbuf + (long long)b * L.nu * L.nv;
        ga0 = ct.ra0; ga1 = ct.ra1; gc0 = ct.rc0; gc1 = ct.rc1;
    } else {
        g_raw = P.gfbuf + (long long)b * L.nu * L.nv;
        ga0 = ct.fa0; ga1 = ct.fa1; gc0 = ct.fc0; gc1 = ct.fc1;
    }
    const int Fa = ga1 - ga0, Fc = gc1 - gc0;
    const float *gF = g_raw;
    const float *F = P.fbuf + (long long)b * L.nu * L.nv;
    // dMU^ (no corrections) and the four jaw edges: reduction over the box
    if (Fa > 0 && Fc > 0) {
        for (int t = threadIdx.x; t < Fa * Fc; t += blockDim.x) {
            const int a = ga0 + t / Fc, c = gc0 + t % Fc;
            const float g = gF[t];
            if (!M.corr) acc[0] = fmaf(g, F[t], acc[0]);
            const float u = ((float)a - L.cu) * L.du, v = ((float)c - L.cv) * L.dv;
            const float fx = overlap_f(u, s_j[0], s_j[1], L.du);
            const float fy = overlap_f(v, s_j[2], s_j[3], L.dv);
            const float dxl = overlap_dlo(u, s_j[0], s_j[1], L.du), dxh = overlap_dhi(u, s_j[0], s_j[1], L.du);
            const float dyl = overlap_dlo(v, s_j[2], s_j[3], L.dv), dyh = overlap_dhi(v, s_j[2], s_j[3], L.dv);
            if (dxl == 0.f && dxh == 0.f && dyl == 0.f && dyh == 0.f) continue;
            // G = tau + (1 - tau) f_leaf
            int lo = 0, hi = np;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (s_lb[mid + 1] > v - hdv) hi = mid; else lo = mid + 1;
            }
            float fl = 0.f;
            for (int i = lo; i < np && s_lb[i] < v + hdv; ++i) {
                const float om = overlap_f(v, s_lb[i], s_lb[i + 1], L.dv);
                if (om > 0.f) fl += om * overlap_f(u, s_lo[i], s_hi[i], L.du);
            }
            const float G = M.tau + (1.f - M.tau) * fl;
            const float gd = g * dscale;
            acc[1] = fmaf(gd, dxl * fy * G, acc[1]);
            acc[2] = fmaf(gd, dxh * fy * G, acc[2]);
            acc[3] = fmaf(gd, fx * dyl * G, acc[3]);
            acc[4] = fmaf(gd, fx * dyh * G, acc[4]);
        }
    }
    block_sum<5>(acc, s_red);
    if (threadIdx.x == 0) {
        const float dmuh = M.cal * acc[0];
        const float m = mu[b];
        dmu[b] = (M.ste || m >= M.eps_mu) ? dmuh : 0.f;
        for (int pr = 0; pr < 2; ++pr) {
            const float ga = acc[1 + 2 * pr], gb = acc[2 + 2 * pr];
            if (M.ste) {
                djaws[4LL * b + 2 * pr] = ga;
                djaws[4LL * b + 2 * pr + 1] = gb;
            } else {
                const float sp = 0.5f * (s_jgc[pr] + s_jgw[pr]), dp = 0.5f * (s_jgc[pr] - s_jgw[pr]);
                djaws[4LL * b + 2 * pr] = ga * sp + gb * dp;
                djaws[4LL * b + 2 * pr + 1] = ga * dp + gb * sp;
            }
        }
    }
    // leaf edges: one thread per pair, over the rows its strip overlaps
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        float gl = 0.f, gr = 0.f;
        if (Fa > 0 && Fc > 0) {
            const float lb0 = s_lb[i], lb1 = s_lb[i + 1];
            // rows c whose pixel [v - dv/2, v + dv/2] overlaps the strip
            const int c_lo = max((int)floorf(L.cv + lb0 / L.dv - 0.5f), gc0);
            const int c_hi = min((int)ceilf(L.cv + lb1 / L.dv + 0.5f) + 1, gc1);
            for (int c = c_lo; c < c_hi; ++c) {
                const float v = ((float)c - L.cv) * L.dv;
                const float om = overlap_f(v, lb0, lb1, L.dv);
                if (om <= 0.f) continue;
                const float fy = overlap_f(v, s_j[2], s_j[3], L.dv);
                if (fy <= 0.f) continue;
                for (int a = ga0; a < ga1; ++a) {
                    const float u = ((float)a - L.cu) * L.du;
                    const float dl = overlap_dlo(u, s_lo[i], s_hi[i], L.du);
                    const float dr = overlap_dhi(u, s_lo[i], s_hi[i], L.du);
                    if (dl == 0.f && dr == 0.f) continue;
                    const float fx = overlap_f(u, s_j[0], s_j[1], L.du);
                    const float s = gF[(long long)(a - ga0) * Fc + (c - gc0)] * dscale * fx * fy *
                                    (1.f - M.tau) * om;
                    gl = fmaf(s, dl, gl);
                    gr = fmaf(s, dr, gr);
                }
            }
        }
        float ol, orr;
        if (M.ste) {
            ol = gl;
            orr = gr;
        } else {
            const float sp = 0.5f * (s_gc[i] + s_gw[i]), dp = 0.5f * (s_gc[i] - s_gw[i]);
            ol = gl * sp + gr * dp;
            orr = gl * dp + gr * sp;
        }
        dleaves[((long long)b * np + i) * 2] = ol;
        dleaves[((long long)b * np + i) * 2 + 1] = orr;
    }
}

cudaError_t launch_param_grad(const PlanDev &P, const float *leaves, const float *jaws,
                              const float *mu, float *dleaves, float *djaws, float *dmu,
                              cudaStream_t s)
{
    k_param_grad<<<P.n_cp, 256, 0, s>>>(P, leaves, jaws, mu, dleaves, djaws, dmu);
    return cudaGetLastError();
}

}  // namespace pdrt
