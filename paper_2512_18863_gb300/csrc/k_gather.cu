// Rotation back to the patient grid and MU-weighted accumulation
// (Sec. 2.2.7, Eq. D_total), and its transpose.
//
// k_gather: one thread per voxel column (ix, iy) of two z planes (a warp:
//   8 x 4 columns), looping over the control points of a chunk; the voxel
//   samples the beam-frame dose D'_b bilinearly in (u, w) (its v coordinate
//   is an exact lattice plane, so trilinear reduces to bilinear), sums
//   cal * MU_b * sample in a register and writes the voxel once per chunk.
//   (u, w), the slice records and the weights depend on (ix, iy) only, so
//   they serve both planes.  No atomics; the CP order of each voxel's sum is
//   fixed.  A CTA (32 x 8 columns of two planes) skips a control point when
//   its footprint misses the CTA.
// k_gather_T: pull form of the transpose: every beam-frame point (i, j, k) of
//   the output box gathers the dose gradient of the voxels of plane j whose
//   bilinear stencil contains it (all inside a 3 x 3 window); the voxel's beam coordinates
//   come from the same float expression as in k_gather (voxel_to_beam) and
//   the weight 1 - |f - n| equals the forward's 1 - t or t, so this is the
//   transpose of the forward up to summation order.  No atomics.  The taps
//   of a lattice column (i, k) do not depend on the plane j: a thread owns
//   one column of one slice, builds its taps once and sweeps the planes two
//   at a time.  A warp holds 8 columns x 4 adjacent slices, a small patch of
//   the rotated lattice, so its loads touch few cache lines at any gantry
//   angle (32 columns of one slice touched up to 32).
#include <math.h>

#include "pdrt_impl.cuh"

namespace pdrt {

// D'_b sampled bilinearly in (u, w) at planes iz (va) and iz + 1 (vb), zero
// outside the slices' output boxes and the lattice; the coordinate and
// slice-record work is shared by the two planes.  The voxel's beam
// coordinates (fu, fw) use the same float expression as voxel_to_beam.
template <class PL>
__device__ __forceinline__ void sample_cp2(const PL &P, int bl, int b, float fu, float fw, int iz,
                                           float &va, float &vb)
{
    const Lattice &L = P.lat;
    const float bu = floorf(fu), bw = floorf(fw);
    const int i0 = (int)bu, k0 = (int)bw;
    const float tu = fu - bu, tw = fw - bw;
    const float *base = P.region + (long long)bl * P.cap_o;
    va = 0.f;
    vb = 0.f;
#pragma unroll
    for (int dk = 0; dk < 2; ++dk) {
        const int k = k0 + dk;
        if (k < 0 || k >= L.nw) continue;
        const int4 gb = __ldg(&P.gbox[(long long)b * L.nw + k]);
        const int ox = gb.y, ow = gb.z, oj0 = gb.w & 0xFFFF, oj1 = gb.w >> 16;
        if (iz + 1 < oj0 || iz >= oj1 || i0 + 1 < ox || i0 >= ox + ow) continue;
        const bool lo_ok = i0 >= ox, hi_ok = i0 + 1 < ox + ow;
        const float wk = dk ? tw : 1.f - tw;
        if (iz >= oj0) {
            const float *row = base + gb.x + (long long)(iz - oj0) * ow;
            const float v0 = lo_ok ? __ldg(&row[i0 - ox]) : 0.f;
            const float v1 = hi_ok ? __ldg(&row[i0 + 1 - ox]) : 0.f;
            va += wk * ((1.f - tu) * v0 + tu * v1);
        }
        if (iz + 1 < oj1) {
            const float *row = base + gb.x + (long long)(iz + 1 - oj0) * ow;
            const float v0 = lo_ok ? __ldg(&row[i0 - ox]) : 0.f;
            const float v1 = hi_ok ? __ldg(&row[i0 + 1 - ox]) : 0.f;
            vb += wk * ((1.f - tu) * v0 + tu * v1);
        }
    }
}

// CTA (tx, ty, tz) of one plan's gather: voxel columns 32 tx .. + 31,
// 8 ty .. + 7 of planes 2 tz and 2 tz + 1
template <class PL>
__device__ __forceinline__ void gather_block(const PL &P, int b0, int nb, float *__restrict__ dose, int first,
                                             int tx, int ty, int tz)
{
    // warp w covers voxels 8 x 4 (x, y) of the CTA's 32 x 8: whatever the
    // gantry angle, a warp's samples then fall in few beam slices and rows
    const int wq = threadIdx.x >> 5, lq = threadIdx.x & 31;
    const int ix = tx * 32 + (wq & 3) * 8 + (lq & 7);
    const int iy = ty * 8 + (wq >> 2) * 4 + (lq >> 3);
    const int iz = 2 * tz;                  // planes iz and iz + 1 (if inside)
    const bool has1 = iz + 1 < P.nz;
    const bool inside = ix < P.nx && iy < P.ny;
    const float bx0 = (float)(tx * 32), bx1 = (float)min(tx * 32 + 31, P.nx - 1);
    const float by0 = (float)(ty * 8), by1 = (float)min(ty * 8 + 7, P.ny - 1);
    __shared__ int s_list[kMaxCpPerChunk];
    __shared__ int s_wcnt[8];
    __shared__ float4 s_geo[kMaxCpPerChunk];    // au, bu, cu0, cal * MU
    __shared__ float2 s_geo2[kMaxCpPerChunk];   // aw, bw
    __shared__ float s_cw0[kMaxCpPerChunk];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // 1) one thread per control point of the chunk tests whether its footprint
    //    (union of output boxes; fu, fw are affine in (ix, iy)) meets this CTA
    bool hit = false;
    if ((int)threadIdx.x < nb) {
        const int b = b0 + threadIdx.x;
        const CpTab &ct = P.cptab[b];
        if (iz + (has1 ? 1 : 0) >= ct.vj0 && iz < ct.vj1) {
            const CpGeo g = P.cpgeo[b];
            const float u00 = fmaf(g.au, bx0, fmaf(g.bu, by0, g.cu0));
            const float u10 = fmaf(g.au, bx1, fmaf(g.bu, by0, g.cu0));
            const float u01 = fmaf(g.au, bx0, fmaf(g.bu, by1, g.cu0));
            const float u11 = fmaf(g.au, bx1, fmaf(g.bu, by1, g.cu0));
            const float w00 = fmaf(g.aw, bx0, fmaf(g.bw, by0, g.cw0));
            const float w10 = fmaf(g.aw, bx1, fmaf(g.bw, by0, g.cw0));
            const float w01 = fmaf(g.aw, bx0, fmaf(g.bw, by1, g.cw0));
            const float w11 = fmaf(g.aw, bx1, fmaf(g.bw, by1, g.cw0));
            const float umin = fminf(fminf(u00, u10), fminf(u01, u11));
            const float umax = fmaxf(fmaxf(u00, u10), fmaxf(u01, u11));
            const float wmin = fminf(fminf(w00, w10), fminf(w01, w11));
            const float wmax = fmaxf(fmaxf(w00, w10), fmaxf(w01, w11));
            hit = !(umax < (float)ct.ui0 - 1.f || umin > (float)ct.ui1 ||
                    wmax < (float)ct.k0 - 1.f || wmin > (float)ct.k1);
        }
    }
    // 2) ordered compaction (keeps the CP order of the sum fixed)
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (lane == 0) s_wcnt[wid] = __popc(m);
    __syncthreads();
    int off = 0, total = 0;
    for (int w = 0; w < 8; ++w) {
        off += (w < wid) ? s_wcnt[w] : 0;
        total += s_wcnt[w];
    }
    if (hit) s_list[off + __popc(m & ((1u << lane) - 1u))] = threadIdx.x;
    __syncthreads();
    // 3) per-CP constants of the listed control points into shared memory
    for (int n = threadIdx.x; n < total; n += blockDim.x) {
        const int b = b0 + s_list[n];
        const CpGeo g = P.cpgeo[b];
        s_geo[n] = make_float4(g.au, g.bu, g.cu0, P.cptab[b].cal_mu);
        s_geo2[n] = make_float2(g.aw, g.bw);
        s_cw0[n] = g.cw0;
    }
    __syncthreads();
    // 4) every voxel column samples the listed control points in order, two
    //    at a time so that their slice-table and region loads overlap (a
    //    control point listed for one plane only adds exact zeros to the other)
    float acc0 = 0.f, acc1 = 0.f;
    if (inside) {
        const float fx = (float)ix, fy = (float)iy;
        int n = 0;
        for (; n + 1 < total; n += 2) {
            float va[2], vb[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int bl = s_list[n + q], b = b0 + bl;
                const float4 gu = s_geo[n + q];
                const float2 gw = s_geo2[n + q];
                const float fu = fmaf(gu.x, fx, fmaf(gu.y, fy, gu.z));
                const float fw = fmaf(gw.x, fx, fmaf(gw.y, fy, s_cw0[n + q]));
                sample_cp2(P, bl, b, fu, fw, iz, va[q], vb[q]);
            }
            acc0 = fmaf(s_geo[n].w, va[0], acc0);
            acc0 = fmaf(s_geo[n + 1].w, va[1], acc0);
            acc1 = fmaf(s_geo[n].w, vb[0], acc1);
            acc1 = fmaf(s_geo[n + 1].w, vb[1], acc1);
        }
        if (n < total) {
            const int bl = s_list[n], b = b0 + bl;
            const float4 gu = s_geo[n];
            const float2 gw = s_geo2[n];
            const float fu = fmaf(gu.x, fx, fmaf(gu.y, fy, gu.z));
            const float fw = fmaf(gw.x, fx, fmaf(gw.y, fy, s_cw0[n]));
            float va, vb;
            sample_cp2(P, bl, b, fu, fw, iz, va, vb);
            acc0 = fmaf(gu.w, va, acc0);
            acc1 = fmaf(gu.w, vb, acc1);
        }
        const long long plane = (long long)P.ny * P.nx;
        const long long idx = (long long)iz * plane + (long long)iy * P.nx + ix;
        dose[idx] = first ? acc0 : dose[idx] + acc0;
        if (has1) dose[idx + plane] = first ? acc1 : dose[idx + plane] + acc1;
    }
}

__global__ void __launch_bounds__(256) k_gather(PlanDev P, int b0, int nb, float *__restrict__ dose,
                                                int first)
{
    gather_block(P, b0, nb, dose, first, blockIdx.x, blockIdx.y, blockIdx.z);
}

cudaError_t launch_gather(const PlanDev &P, int b0, int nb, float *dose, bool first, cudaStream_t s)
{
    dim3 grid((P.nx + 31) / 32, (P.ny + 7) / 8, (P.nz + 1) / 2);
    k_gather<<<grid, 256, 0, s>>>(P, b0, nb, dose, first ? 1 : 0);
    return cudaGetLastError();
}

namespace {
constexpr int kGtS = 4;              // beam slices per CTA of k_gather_T
constexpr int kGtW = 8;              // lattice columns per warp (x kGtS slices = 32 lanes)
constexpr int kGtCols = 8 * kGtW;    // lattice columns per pass of a CTA (8 warps)
}

// One CTA per control point and group of kGtS consecutive beam slices; lane
// (c, s) of a warp owns lattice column i0 + c of slice k0 + s, so a warp's
// 8 x 4 points form a small patch of the rotated lattice whose voxel taps
// fall in few cache lines at any gantry angle.  Each thread builds its
// column's taps once (they do not depend on the plane) and sweeps its
// slice's planes two at a time.
template <class PL>
__device__ __forceinline__ void gather_t_block(const PL &P, int b0, const float *__restrict__ gd, int tg, int bl)
{
    const Lattice &L = P.lat;
    const int kg = tg * kGtS, b = b0 + bl;
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    const int sl = lane / kGtW, cl = lane % kGtW;   // slice and column of this lane
    const int k = kg + sl;
    int4 ob = make_int4(0, 0, 0, 0);                // oi0, oi1, oj0, oj1
    long long off_o = 0;
    if (k < L.nw) {
        const SliceTab *sp = &P.slices[(long long)b * L.nw + k];
        ob = *reinterpret_cast<const int4 *>(&sp->oi0);
        off_o = sp->off_o;
    }
    const bool live = ob.y > ob.x && ob.w > ob.z;
    // the group's union of u ranges (every thread computes the same)
    int ui0 = 1 << 30, ui1 = -(1 << 30);
#pragma unroll
    for (int q = 0; q < kGtS; ++q) {
        const int kq = kg + q;
        if (kq >= L.nw) break;
        const int4 oq = *reinterpret_cast<const int4 *>(&P.slices[(long long)b * L.nw + kq].oi0);
        if (oq.y > oq.x && oq.w > oq.z) {
            ui0 = min(ui0, oq.x);
            ui1 = max(ui1, oq.y);
        }
    }
    if (ui1 <= ui0) return;   // no slice of the group has work (uniform)
    const CpGeo g = P.cpgeo[b];
    const int ow = ob.y - ob.x, oh = ob.w - ob.z;
    float *out = P.region + (long long)bl * P.cap_o + off_o;
    __shared__ GtTap s_tap[9 * 256];   // tap q of thread t at [q * 256 + t]
    const long long plane = (long long)P.ny * P.nx;
    for (int c0 = ui0; c0 < ui1; c0 += kGtCols) {
        const int i = c0 + warp * kGtW + cl;
        if (live && i >= ob.x && i < ob.y) {
            const int n = gather_t_taps(g, L, P.nx, P.ny, i, k, s_tap + threadIdx.x, 256);
            for (int jj = 0; jj < oh; jj += 2) {
                const float *gp = gd + (long long)(ob.z + jj) * plane;
                const bool two = jj + 1 < oh;
                float sum0 = 0.f, sum1 = 0.f;
                for (int q = 0; q < n; ++q) {
                    const GtTap tp = s_tap[q * 256 + threadIdx.x];
                    sum0 = fmaf(tp.w, __ldg(&gp[tp.off]), sum0);
                    if (two) sum1 = fmaf(tp.w, __ldg(&gp[plane + tp.off]), sum1);
                }
                out[(long long)jj * ow + (i - ob.x)] = sum0;
                if (two) out[(long long)(jj + 1) * ow + (i - ob.x)] = sum1;
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_gather_T(PlanDev P, int b0, const float *__restrict__ gd)
{
    gather_t_block(P, b0, gd, blockIdx.x, blockIdx.y);
}

cudaError_t launch_gather_T(const PlanDev &P, int b0, int nb, const float *g, cudaStream_t s)
{
    dim3 grid((P.lat.nw + kGtS - 1) / kGtS, nb);
    k_gather_T<<<grid, 256, 0, s>>>(P, b0, g);
    return cudaGetLastError();
}

// Batched forms: one launch over the CTAs of several plans' passes (the
// gather of a round of the batched graph, or its transpose).  Entry e owns
// CTAs A.ent[e].blk0 .. A.ent[e + 1].blk0 - 1 of the one-dimensional grid,
// in the order of its plan's own grid (x fastest); its plan view, pass
// and buffers sit in the kernel parameters (grid constant), read through
// the constant cache.  Each CTA does exactly what the per-plan kernel's CTA
// of the same coordinates does, so the results are the per-plan ones bit
// for bit.
struct GatherBatchArgs {
    GatherEntry ent[kGatherBatchMax];
    int n_ent, n_blk;
};
static_assert(sizeof(GatherBatchArgs) <= 32000, "kernel parameters above 32 KB");

__device__ __forceinline__ int gather_entry_of(const GatherBatchArgs &A, int blk)
{
    int e = 0;
    while (e + 1 < A.n_ent && A.ent[e + 1].blk0 <= blk) ++e;
    return e;
}

__global__ void __launch_bounds__(256) k_gather_multi(const __grid_constant__ GatherBatchArgs A)
{
    const int e = gather_entry_of(A, (int)blockIdx.x);
    const GatherEntry &E = A.ent[e];
    const int t = (int)blockIdx.x - E.blk0;
    const int tx = t % E.gx, r = t / E.gx;
    gather_block(E.p, E.b0, E.nb, E.dose, E.first, tx, r % E.gy, r / E.gy);
}

__global__ void __launch_bounds__(256) k_gather_T_multi(const __grid_constant__ GatherBatchArgs A)
{
    const int e = gather_entry_of(A, (int)blockIdx.x);
    const GatherEntry &E = A.ent[e];
    const int t = (int)blockIdx.x - E.blk0;
    gather_t_block(E.p, E.b0, E.gd, t % E.gx, t / E.gx);
}

cudaError_t launch_gather_multi(const GatherEntry *ents, int n, bool transpose, cudaStream_t s)
{
    static thread_local GatherBatchArgs A;   // ~20 KB: not on the stack
    for (int g0 = 0; g0 < n; g0 += kGatherBatchMax) {
        const int ne = n - g0 < kGatherBatchMax ? n - g0 : kGatherBatchMax;
        A.n_ent = ne;
        long long blk = 0;
        for (int e = 0; e < ne; ++e) {
            GatherEntry E = ents[g0 + e];
            const GatherPlan &P = E.p;
            if (transpose) {
                if (!E.gd) return cudaErrorInvalidValue;
                E.gx = (P.lat.nw + kGtS - 1) / kGtS;
                E.gy = E.nb;
            } else {
                if (!E.dose) return cudaErrorInvalidValue;
                E.gx = (P.nx + 31) / 32;
                E.gy = (P.ny + 7) / 8;
            }
            const long long nblk = transpose ? (long long)E.gx * E.gy
                                             : (long long)E.gx * E.gy * ((P.nz + 1) / 2);
            E.blk0 = (int)blk;
            blk += nblk;
            A.ent[e] = E;
        }
        if (blk >= (1LL << 31)) return cudaErrorInvalidValue;
        A.n_blk = (int)blk;
        if (!blk) continue;
        if (transpose)
            k_gather_T_multi<<<(unsigned)blk, 256, 0, s>>>(A);
        else
            k_gather_multi<<<(unsigned)blk, 256, 0, s>>>(A);
        const cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

}  // namespace pdrt
