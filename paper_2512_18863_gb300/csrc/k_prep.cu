// Preparation kernels of the dose engine:
//   k_hu_to_red  HU -> relative electron density (Sec. 2.2, commissioned curve)
//   k_raster     hardware projection (Sec. 2.2.1) + fluence map (Sec. 2.2.2)
//   k_tables     central-ray WEPL (Sec. 2.2.4), depth dose, kernel parameters
//                (Sec. 2.2.5), magnification (Sec. 2.2.3) and the work boxes of
//                every beam slice
#include <math.h>

#include "pdrt_impl.cuh"

namespace pdrt {

// ---------------------------------------------------------------------------
// HU -> RED, piecewise linear, clamped at both ends
// ---------------------------------------------------------------------------
struct HuTable {
    float h[PDRT_MAX_HU_POINTS], r[PDRT_MAX_HU_POINTS];
    int n;
};

__global__ void k_hu_to_red(const float *__restrict__ hu, float *__restrict__ red, long long n,
                            HuTable t)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float x = hu[i];
        float y;
        if (x <= t.h[0]) {
            y = t.r[0];
        } else if (x >= t.h[t.n - 1]) {
            y = t.r[t.n - 1];
        } else {
            y = t.r[t.n - 1];
            for (int m = 0; m + 1 < t.n; ++m) {
                if (x >= t.h[m] && x <= t.h[m + 1]) {
                    float f = (x - t.h[m]) / (t.h[m + 1] - t.h[m]);
                    y = t.r[m] + f * (t.r[m + 1] - t.r[m]);
                    break;
                }
            }
        }
        red[i] = y;
    }
}

cudaError_t launch_hu_to_red(const float *hu, float *red, long long n, const float *pts, int npts,
                             cudaStream_t s)
{
    HuTable t;
    t.n = npts;
    for (int i = 0; i < npts; ++i) {
        t.h[i] = pts[2 * i];
        t.r[i] = pts[2 * i + 1];
    }
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) blocks = 1;
    k_hu_to_red<<<(unsigned)blocks, 256, 0, s>>>(hu, red, n, t);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Projection (Sec. 2.2.1): centre/width, minimum opening, travel clamp.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void project_pair(float pa, float pb, float wmin, float F, float &ah,
                                             float &bh)
{
    float c = 0.5f * (pa + pb);
    float w = pb - pa;
    float w2 = (w >= wmin) ? w : wmin;
    float c1 = (c >= -F) ? c : -F;
    float c2 = (c1 <= F) ? c1 : F;
    ah = c2 - 0.5f * w2;
    bh = c2 + 0.5f * w2;
}

// Pixel index range [lo, hi) whose overlap with (e0, e1) can be non-zero:
// pixel centre x = (a - c) d, so a in (c + e0/d - 1/2, c + e1/d + 1/2); one
// extra pixel on each side absorbs rounding (those evaluate to exactly 0).
__device__ __forceinline__ void support_range(float e0, float e1, float c, float d, int n, int &lo,
                                              int &hi)
{
    if (!(e1 > e0)) {
        lo = hi = 0;
        return;
    }
    float x0 = c + e0 / d - 0.5f, x1 = c + e1 / d + 0.5f;
    int a0 = (int)floorf(fmaxf(x0, -4.f));
    int a1 = (int)ceilf(fminf(x1, (float)n + 4.f)) + 1;
    lo = max(a0, 0);
    hi = min(a1, n);
    if (hi <= lo) lo = hi = 0;
}

// Box of the pixels whose rotation source falls inside the bilinear reach of
// the corrected box [ca0,ca1) x [cc0,cc1): sources with a in (ca0-1, ca1) and
// c in (cc0-1, cc1).  The source rectangle's corners are turned forward by
// R(angle); one extra pixel on each side absorbs rounding (the exact weights
// of those pixels are 0).
__device__ void rotated_box(const MachineDev &M, const Lattice &L, int ca0, int ca1, int cc0,
                            int cc1, int &a0, int &a1, int &c0, int &c1)
{
    const float us[2] = {((float)(ca0 - 1) - L.cu) * L.du, ((float)ca1 - L.cu) * L.du};
    const float vs[2] = {((float)(cc0 - 1) - L.cv) * L.dv, ((float)cc1 - L.cv) * L.dv};
    float amin = 1e30f, amax = -1e30f, cmin = 1e30f, cmax = -1e30f;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            const float x = M.rot_c * us[i] - M.rot_s * vs[j];
            const float y = M.rot_s * us[i] + M.rot_c * vs[j];
            amin = fminf(amin, x); amax = fmaxf(amax, x);
            cmin = fminf(cmin, y); cmax = fmaxf(cmax, y);
        }
    a0 = max((int)floorf(L.cu + amin / L.du) - 1, 0);
    a1 = min((int)ceilf(L.cu + amax / L.du) + 2, L.nu);
    c0 = max((int)floorf(L.cv + cmin / L.dv) - 1, 0);
    c1 = min((int)ceilf(L.cv + cmax / L.dv) + 2, L.nv);
    if (a1 <= a0 || c1 <= c0) a0 = a1 = c0 = c1 = 0;
}

// Fluence corrections of Sec. 2.2.2 after the raw aperture map of control
// point b is in tbuf over the raw box:
//   blurred(a, c) = OAP(a, c) sum_s gv[s] sum_t gu[t] raw(a - t, c - s)
// over the blurred box (the raw map is zero outside its box, which lies in
// the lattice, so this is the blur along u then v with zero padding), into
// fbuf, or into gfbuf when the collimator rotation then resamples it into
// fbuf over the final box.  One block per control point.
__device__ void correct_fluence(const PlanDev &P, int b)
{
    const MachineDev &M = P.mach;
    const Lattice &L = P.lat;
    __syncthreads();
    const CpTab ct = P.cptab[b];
    const long long slot = (long long)b * L.nu * L.nv;
    const float *raw = P.tbuf + slot;
    const int Rc = ct.rc1 - ct.rc0;
    const int Ca = ct.ca1 - ct.ca0, Cc = ct.cc1 - ct.cc0;
    float *blur = (M.rot ? P.gfbuf : P.fbuf) + slot;
    for (int t = threadIdx.x; t < Ca * Cc; t += blockDim.x) {
        const int a = ct.ca0 + t / Cc, c = ct.cc0 + t % Cc;
        float s = 0.f;
        for (int dv = -M.rbv; dv <= M.rbv; ++dv) {
            const int cs = c - dv;
            if (cs < ct.rc0 || cs >= ct.rc1) continue;
            float r = 0.f;
            for (int du = -M.rbu; du <= M.rbu; ++du) {
                const int as = a - du;
                if (as < ct.ra0 || as >= ct.ra1) continue;
                r = fmaf(M.gu[du + M.rbu], raw[(long long)(as - ct.ra0) * Rc + (cs - ct.rc0)], r);
            }
            s = fmaf(M.gv[dv + M.rbv], r, s);
        }
        blur[t] = s * off_axis_factor(M, L, a, c);
    }
    if (!M.rot) return;
    __syncthreads();
    float *F = P.fbuf + slot;
    const int Fc = ct.fc1 - ct.fc0, Fa = ct.fa1 - ct.fa0;
    for (int t = threadIdx.x; t < Fa * Fc; t += blockDim.x) {
        const int a = ct.fa0 + t / Fc, c = ct.fc0 + t % Fc;
        float fa, fc;
        rotation_source(M, L, a, c, fa, fc);
        const float ba = floorf(fa), bc = floorf(fc);
        const int ia = (int)ba, ic = (int)bc;
        const float ta = fa - ba, tc = fc - bc;
        float v = 0.f;
        for (int dc = 0; dc < 2; ++dc) {
            const int cc = ic + dc;
            if (cc < ct.cc0 || cc >= ct.cc1) continue;
            const float wc = dc ? tc : 1.f - tc;
            for (int da = 0; da < 2; ++da) {
                const int aa = ia + da;
                if (aa < ct.ca0 || aa >= ct.ca1) continue;
                v = fmaf(wc * (da ? ta : 1.f - ta), blur[(long long)(aa - ct.ca0) * Cc + (cc - ct.cc0)], v);
            }
        }
        F[t] = v;
    }
}

__global__ void __launch_bounds__(256) k_raster(PlanDev P, const float *__restrict__ leaves,
                                                const float *__restrict__ jaws,
                                                const float *__restrict__ mu)
{
    const int b = blockIdx.x;
    const MachineDev &M = P.mach;
    const Lattice &L = P.lat;
    const int np = M.n_pairs;
    __shared__ float s_lo[PDRT_MAX_PAIRS], s_hi[PDRT_MAX_PAIRS], s_lb[PDRT_MAX_PAIRS + 1];
    __shared__ float s_j[4];
    __shared__ int s_box[4];
    __shared__ unsigned s_bad;
    if (threadIdx.x == 0) s_bad = 0u;
    __syncthreads();
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        float pa = leaves[((long long)b * np + i) * 2];
        float pb = leaves[((long long)b * np + i) * 2 + 1];
        if (!isfinite(pa) || !isfinite(pb)) atomicOr(&s_bad, 1u);
        project_pair(pa, pb, M.wmin_leaf, M.f_leaf, s_lo[i], s_hi[i]);
    }
    for (int i = threadIdx.x; i <= np; i += blockDim.x) s_lb[i] = P.leaf_bounds[i];
    if (threadIdx.x == 0) {
        float j[4], m = mu[b];
        for (int q = 0; q < 4; ++q) {
            j[q] = jaws[4LL * b + q];
            if (!isfinite(j[q])) atomicOr(&s_bad, 1u);
        }
        if (!isfinite(m)) atomicOr(&s_bad, 1u);
        project_pair(j[0], j[1], M.wmin_jaw, M.f_jaw, s_j[0], s_j[1]);
        project_pair(j[2], j[3], M.wmin_jaw, M.f_jaw, s_j[2], s_j[3]);
        float muh = (m >= M.eps_mu) ? m : M.eps_mu;
        int a0, a1, c0, c1;
        support_range(s_j[0], s_j[1], L.cu, L.du, L.nu, a0, a1);
        support_range(s_j[2], s_j[3], L.cv, L.dv, L.nv, c0, c1);
        if (a1 <= a0 || c1 <= c0) a0 = a1 = c0 = c1 = 0;
        s_box[0] = a0; s_box[1] = a1; s_box[2] = c0; s_box[3] = c1;
        CpTab &ct = P.cptab[b];
        ct.mu_hat = muh;
        ct.cal_mu = M.cal * muh;
        ct.ra0 = a0; ct.ra1 = a1; ct.rc0 = c0; ct.rc1 = c1;
        int ca0 = a0, ca1 = a1, cc0 = c0, cc1 = c1;
        if (M.corr && a1 > a0) {
            ca0 = max(a0 - M.rbu, 0); ca1 = min(a1 + M.rbu, L.nu);
            cc0 = max(c0 - M.rbv, 0); cc1 = min(c1 + M.rbv, L.nv);
        }
        ct.ca0 = ca0; ct.ca1 = ca1; ct.cc0 = cc0; ct.cc1 = cc1;
        if (M.rot && ca1 > ca0) {
            rotated_box(M, L, ca0, ca1, cc0, cc1, ct.fa0, ct.fa1, ct.fc0, ct.fc1);
        } else {
            ct.fa0 = ca0; ct.fa1 = ca1; ct.fc0 = cc0; ct.fc1 = cc1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_bad) atomicOr(P.flags, (unsigned)PDRT_FLAG_NAN_INPUT);
    const int a0 = s_box[0], c0 = s_box[2];
    const int Fa = s_box[1] - a0, Fc = s_box[3] - c0;
    // raw aperture map: straight into the fluence buffer, or into the scratch
    // map that the corrections read
    float *F = (M.corr ? P.tbuf : P.fbuf) + (long long)b * L.nu * L.nv;
    const float hdv = 0.5f * L.dv;
    for (int t = threadIdx.x; t < Fa * Fc; t += blockDim.x) {
        const int a = a0 + t / Fc, c = c0 + t % Fc;
        const float u = ((float)a - L.cu) * L.du;
        const float v = ((float)c - L.cv) * L.dv;
        const float fx = overlap_f(u, s_j[0], s_j[1], L.du);
        const float fy = overlap_f(v, s_j[2], s_j[3], L.dv);
        float val = 0.f;
        if (fx > 0.f && fy > 0.f) {
            // first pair whose upper bound is above the row's lower edge
            int lo = 0, hi = np;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (s_lb[mid + 1] > v - hdv) hi = mid; else lo = mid + 1;
            }
            float fl = 0.f;
            for (int i = lo; i < np && s_lb[i] < v + hdv; ++i) {
                float om = overlap_f(v, s_lb[i], s_lb[i + 1], L.dv);
                if (om > 0.f) fl += om * overlap_f(u, s_lo[i], s_hi[i], L.du);
            }
            val = fx * fy * (M.tau + (1.f - M.tau) * fl);
        }
        F[(long long)(a - a0) * Fc + (c - c0)] = val;
    }
    if (M.corr) correct_fluence(P, b);
}

cudaError_t launch_raster(const PlanDev &P, const float *leaves, const float *jaws,
                          const float *mu, cudaStream_t s)
{
    k_raster<<<P.n_cp, 256, 0, s>>>(P, leaves, jaws, mu);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Slice tables.  One block per control point walks the beam slices in tiles
// of blockDim: trilinear density on the central ray, block prefix sum
// (midpoint rule: z_k = dw (sum_{m<k} rho_m + rho_k / 2)), depth dose,
// kernel parameters and their window sums, work boxes and buffer offsets.
// ---------------------------------------------------------------------------
constexpr int kTabThreads = 512;

template <typename T>
__device__ T block_excl_scan(T v, T *s_warp, T &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T x = v;
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T w = (lane < nw) ? s_warp[lane] : T(0);
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) s_warp[lane] = w;
    }
    __syncthreads();
    T before = (wid > 0) ? s_warp[wid - 1] : T(0);
    total = s_warp[nw - 1];
    __syncthreads();
    return before + x - v;
}

__device__ float red_trilinear(const PlanDev &P, float fx, float fy, float fz)
{
    float bx = floorf(fx), by = floorf(fy), bz = floorf(fz);
    int x0 = (int)bx, y0 = (int)by, z0 = (int)bz;
    float tx = fx - bx, ty = fy - by, tz = fz - bz;
    float s = 0.f;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz) {
        int z = z0 + dz;
        if (z < 0 || z >= P.nz) continue;
        float wz = dz ? tz : 1.f - tz;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            int y = y0 + dy;
            if (y < 0 || y >= P.ny) continue;
            float wy = dy ? ty : 1.f - ty;
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                int x = x0 + dx;
                if (x < 0 || x >= P.nx) continue;
                float wx = dx ? tx : 1.f - tx;
                s += wz * wy * wx * __ldg(&P.red[((long long)z * P.ny + y) * P.nx + x]);
            }
        }
    }
    return s;
}

__device__ __forceinline__ float depth_dose_at(const PlanDev &P, float z)
{
    const MachineDev &M = P.mach;
    float t = z / M.depth_step;
    if (t <= 0.f) return P.depth_dose[0];
    if (t >= (float)(M.n_depth - 1)) return P.depth_dose[M.n_depth - 1];
    float fl = floorf(t);
    int m = (int)fl;
    float f = t - fl;
    float t0 = P.depth_dose[m], t1 = P.depth_dose[m + 1];
    return t0 + f * (t1 - t0);
}

// conservative lattice range of the points whose magnified bilinear stencil
// touches pixel range [p0, p1): idx in (c + (p0 - 1 - c)/m, c + (p1 - c)/m)
__device__ __forceinline__ void mag_range(int p0, int p1, float c, float m, int n, int &lo,
                                          int &hi, long long &exact)
{
    float l = c + ((float)p0 - 1.f - c) / m;
    float r = c + ((float)p1 - c) / m;
    int e0 = max((int)floorf(l) + 1, 0), e1 = min((int)ceilf(r) - 1, n - 1);
    exact = (e1 >= e0) ? (long long)(e1 - e0 + 1) : 0;
    lo = max((int)floorf(l), 0);
    hi = min((int)ceilf(r) + 1, n);
    if (hi < lo) hi = lo;
}

__global__ void __launch_bounds__(kTabThreads) k_tables(PlanDev P)
{
    const int b = blockIdx.x;
    const Lattice &L = P.lat;
    const MachineDev &M = P.mach;
    const CpGeo g = P.cpgeo[b];
    const int fa0 = P.cptab[b].fa0, fa1 = P.cptab[b].fa1;
    const int fc0 = P.cptab[b].fc0, fc1 = P.cptab[b].fc1;
    const bool fempty = (fa1 <= fa0) || (fc1 <= fc0);
    const int R = M.R;
    __shared__ float s_wf[32];
    __shared__ long long s_wl[32];
    __shared__ int s_u0, s_u1, s_v0, s_v1, s_k0, s_k1;
    __shared__ unsigned long long s_sup, s_reg, s_act;
    if (threadIdx.x == 0) {
        s_u0 = L.nu; s_u1 = 0; s_v0 = L.nv; s_v1 = 0; s_k0 = L.nw; s_k1 = 0;
        s_sup = s_reg = s_act = 0ull;
    }
    __syncthreads();
    float carry = 0.f;
    long long carry_o = 0, carry_a = 0;
    for (int t0 = 0; t0 < L.nw; t0 += blockDim.x) {
        const int k = t0 + threadIdx.x;
        const bool valid = k < L.nw;
        float rho = 0.f;
        if (valid) {
            float dk = (float)k - L.cw;
            rho = red_trilinear(P, fmaf(dk, g.sx_w, g.px0), fmaf(dk, g.sy_w, g.py0), g.pz0);
        }
        float tot;
        float excl = block_excl_scan<float>(rho, s_wf, tot);
        long long so = 0, sa = 0;
        SliceTab st;
        if (valid) {
            const float z = L.du * (carry + excl + 0.5f * rho);
            const float w = ((float)k - L.cw) * L.du;
            const float m = M.sid / (M.sid + w);
            st.z = z;
            st.tdd = depth_dose_at(P, z);
            st.m = m;
            st.c2 = m * m;
            float wr[3], W = 0.f;
            for (int c = 0; c < 3; ++c) {
                float a = M.alpha[c][0] + M.alpha[c][1] * z + M.alpha[c][2] * z * z;
                st.a[c] = (a < 1e-4f) ? 1e-4f : a;
                float ww = M.beta[c][0] + M.beta[c][1] * z + M.beta[c][2] * z * z;
                wr[c] = (ww < 0.f) ? 0.f : ww;
                W += wr[c];
            }
            // window sums S_c over |p|,|q| <= R using the four-fold symmetry
            float S[3] = {0.f, 0.f, 0.f};
            for (int p = 0; p <= R; ++p) {
                const float pu = p * L.du;
                for (int q = 0; q <= R; ++q) {
                    const float qv = q * L.dv;
                    const float r = sqrtf(pu * pu + qv * qv);
                    const float mult = (p == 0 ? 1.f : 2.f) * (q == 0 ? 1.f : 2.f);
                    for (int c = 0; c < 3; ++c) S[c] += mult * expf(-st.a[c] * r);
                }
            }
            for (int c = 0; c < 3; ++c) st.wn[c] = (W > 0.f) ? (wr[c] / W) / S[c] : 0.f;
            st.pad0 = st.pad1 = 0.f;
            // work boxes
            const int2 ur = P.ukr[(long long)b * L.nw + k];
            st.pi0 = st.pi1 = st.pj0 = st.pj1 = 0;
            st.oi0 = st.oi1 = st.oj0 = st.oj1 = 0;
            st.ai0 = st.ai1 = st.aj0 = st.aj1 = 0;
            if (!fempty && ur.y > ur.x) {
                long long ei, ej;
                mag_range(fa0, fa1, L.cu, m, L.nu, st.pi0, st.pi1, ei);
                mag_range(fc0, fc1, L.cv, m, L.nv, st.pj0, st.pj1, ej);
                st.oi0 = max(st.pi0 - R, ur.x);
                st.oi1 = min(st.pi1 + R, ur.y);
                st.oj0 = max(st.pj0 - R, 0);
                st.oj1 = min(st.pj1 + R, L.nv);
                if (st.pi1 > st.pi0 && st.pj1 > st.pj0 && st.oi1 > st.oi0 && st.oj1 > st.oj0) {
                    st.ai0 = max(st.pi0, st.oi0 - R);
                    st.ai1 = min(st.pi1, st.oi1 + R);
                    st.aj0 = max(st.pj0, st.oj0 - R);
                    st.aj1 = min(st.pj1, st.oj1 + R);
                    if (st.ai1 <= st.ai0 || st.aj1 <= st.aj0) st.ai0 = st.ai1 = st.aj0 = st.aj1 = 0;
                    so = (long long)(st.oi1 - st.oi0) * (st.oj1 - st.oj0);
                    sa = (long long)(st.ai1 - st.ai0) * (st.aj1 - st.aj0);
                    atomicMin(&s_u0, st.oi0);
                    atomicMax(&s_u1, st.oi1);
                    atomicMin(&s_v0, st.oj0);
                    atomicMax(&s_v1, st.oj1);
                    atomicMin(&s_k0, k);
                    atomicMax(&s_k1, k + 1);
                    atomicAdd(&s_sup, (unsigned long long)(ei * ej));
                    atomicAdd(&s_reg, (unsigned long long)so);
                    atomicAdd(&s_act, 1ull);
                } else {
                    st.oi0 = st.oi1 = st.oj0 = st.oj1 = 0;
                }
            }
        }
        long long to, ta;
        long long eo = block_excl_scan<long long>(so, s_wl, to);
        long long ea = block_excl_scan<long long>(sa, s_wl, ta);
        if (valid) {
            st.off_o = carry_o + eo;
            st.off_a = carry_a + ea;
            // the plan's scratch bound is an upper bound by construction; if it
            // were ever exceeded the slice is dropped (and flagged) instead of
            // being written past the buffer
            if (st.off_o + so > P.cap_o || st.off_a + sa > P.cap_a) {
                st.oi0 = st.oi1 = st.oj0 = st.oj1 = 0;
                st.ai0 = st.ai1 = st.aj0 = st.aj1 = 0;
                atomicOr(P.flags, (unsigned)PDRT_FLAG_CAPACITY);
            }
            P.slices[(long long)b * L.nw + k] = st;
            // offsets fit 31 bits (cap_o is checked at upload); v bounds 16 bits
            P.gbox[(long long)b * L.nw + k] =
                make_int4((int)st.off_o, st.oi0, st.oi1 - st.oi0, st.oj0 | (st.oj1 << 16));
        }
        carry += tot;
        carry_o += to;
        carry_a += ta;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        CpTab &ct = P.cptab[b];
        ct.ui0 = s_u0; ct.ui1 = s_u1; ct.vj0 = s_v0; ct.vj1 = s_v1;
        ct.k0 = s_k0; ct.k1 = s_k1;
        ct.tot_o = carry_o;
        ct.tot_a = carry_a;
        ct.n_support = (long long)s_sup;
        ct.n_region = (long long)s_reg;
        ct.n_active = (long long)s_act;
    }
}

cudaError_t launch_tables(const PlanDev &P, cudaStream_t s)
{
    k_tables<<<P.n_cp, kTabThreads, 0, s>>>(P);
    return cudaGetLastError();
}

}  // namespace pdrt
