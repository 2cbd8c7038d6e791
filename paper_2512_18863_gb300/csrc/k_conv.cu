// Per-slice lateral convolution (Sec. 2.2.6, Eq. D(x_perp, z)):
//   forward   D'_k(i,j) = T_k C_k sum_{p,q} F~_k(i-p, j-q) K_k(p,q)
//   adjoint   h'_k(i,j) = T_k C_k sum_{p,q} h_k(i+p, j+q)  K_k(p,q)
// where F~_k is the fluence map sampled at the magnified position of lattice
// point (i,j) (Sec. 2.2.3) and K_k the radial three-exponential kernel of the
// slice's radiological depth (Sec. 2.2.5).  K is symmetric in p and in q, so
// both directions run the same inner loop.
//
// This is a dense direct stencil bound by FP32 FMA throughput.  Mapping:
//   * a persistent grid pulls (control point, slice) items from a counter;
//   * a CTA (4 warps) owns a 32-row x 64-column output tile; lane l owns
//     output row i = ibase + l and 16 consecutive output columns (registers);
//   * the input rows the tile needs (tile +- R, clipped to the non-zero
//     input box) are staged in shared memory as [row][column], so every lane
//     of a warp reads the same 16 B of an input row (broadcast), while each
//     lane reads the 4-tap weight quad of its own kernel row |i - u'|
//     (row stride 4*odd floats keeps the 8 lanes of a phase conflict-free);
//   * per 4-tap quad a lane issues 2 shared loads and 64 FMAs.
#include <math.h>

#include "pdrt_impl.cuh"

namespace pdrt {

__host__ __device__ constexpr int conv_tile_width(int nq4) { return kConvCols + 4 * nq4; }

// Output rows per warp: the forward (large halo output box, small input box)
// keeps 32 rows per warp; the adjoint (small output box) uses 8 rows x 4
// column blocks, which wastes fewer lanes on rows outside the box.
constexpr int kFwdRowsPerWarp = 32;
constexpr int kAdjRowsPerWarp = 8;

__host__ __device__ inline int kstride_for(int nq4) { return 4 * ((nq4 & 1) ? nq4 : nq4 + 1); }

template <int NQ4>
__device__ __forceinline__ void conv_row(float (&acc)[kConvTJ], const float *__restrict__ seg,
                                         const float *__restrict__ kr, int c_lo, int c_hi)
{
    float win[kConvTJ + 4];
#pragma unroll
    for (int x = 0; x < kConvTJ + 4; x += 4) {
        const float4 v = *reinterpret_cast<const float4 *>(seg + x);
        win[x] = v.x; win[x + 1] = v.y; win[x + 2] = v.z; win[x + 3] = v.w;
    }
#pragma unroll
    for (int c = 0; c < NQ4; ++c) {
        if (c >= c_lo && c < c_hi) {   // warp-uniform: chunk touches non-zero input columns
            const float4 w4 = *reinterpret_cast<const float4 *>(kr + 4 * c);
            const float wq[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
#pragma unroll
                for (int t = 0; t < kConvTJ; ++t) acc[t] = fmaf(wq[qq], win[t + qq], acc[t]);
            }
        }
        if (c + 1 < NQ4) {
#pragma unroll
            for (int x = 0; x < kConvTJ; ++x) win[x] = win[x + 4];
            const float4 v = *reinterpret_cast<const float4 *>(seg + 4 * c + kConvTJ + 4);
            win[kConvTJ] = v.x; win[kConvTJ + 1] = v.y; win[kConvTJ + 2] = v.z; win[kConvTJ + 3] = v.w;
        }
    }
}

// G = output rows per warp (32, 16 or 8); a warp's lanes cover G rows x 32/G
// blocks of 16 columns, the CTA's 4 warps tile 32 rows x 64 columns.
template <int NQ4, bool ADJ, int G>
__global__ void __launch_bounds__(kConvThreads) k_conv(PlanDev P, int b0, int nb,
                                                       unsigned int *__restrict__ counter)
{
    static_assert(G == 8 || G == 16 || G == 32, "rows per warp");
    constexpr int NB = 32 / G;                 // column blocks per warp
    constexpr int WPR = 32 / G;                // warps stacked along rows
    extern __shared__ float4 smem4[];
    float *smem = reinterpret_cast<float *>(smem4);
    constexpr int W = conv_tile_width(NQ4);
    const Lattice &L = P.lat;
    const int R = P.mach.R;
    const int S = kstride_for(NQ4);
    float *krow = smem;                       // (R + 2) rows x S
    float *tile = smem + (R + 2) * S;         // (32 + 2R) rows x W
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n_items = nb * L.nw;
    __shared__ int s_item;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= n_items) break;
        const int bl = item / L.nw, k = item - bl * L.nw, b = b0 + bl;
        const SliceTab st = P.slices[(long long)b * L.nw + k];
        if (tc_takes_slice(st, ADJ, R, P.tc_enabled)) continue;   // done on the tensor cores
        int in_i0, in_i1, in_j0, in_j1, out_i0, out_i1, out_j0, out_j1;
        float *dst;
        if (ADJ) {
            in_i0 = st.oi0; in_i1 = st.oi1; in_j0 = st.oj0; in_j1 = st.oj1;
            out_i0 = st.ai0; out_i1 = st.ai1; out_j0 = st.aj0; out_j1 = st.aj1;
            dst = P.adjbuf + (long long)bl * P.cap_a + st.off_a;
        } else {
            in_i0 = st.pi0; in_i1 = st.pi1; in_j0 = st.pj0; in_j1 = st.pj1;
            out_i0 = st.oi0; out_i1 = st.oi1; out_j0 = st.oj0; out_j1 = st.oj1;
            dst = P.region + (long long)bl * P.cap_o + st.off_o;
        }
        if (out_i1 <= out_i0 || out_j1 <= out_j0) continue;
        const int out_w = out_i1 - out_i0;

        // kernel rows |p| = 0..R, taps q' = 0..4*NQ4-1 holding K(p, q'-R); row R+1 is zero
        for (int idx = threadIdx.x; idx < (R + 2) * S; idx += blockDim.x) {
            const int p = idx / S, qp = idx - p * S;
            float v = 0.f;
            if (p <= R && qp <= 2 * R) {
                const float pu = p * L.du, qv = (qp - R) * L.dv;
                const float r = sqrtf(pu * pu + qv * qv);
                v = st.wn[0] * expf(-st.a[0] * r) + st.wn[1] * expf(-st.a[1] * r) +
                    st.wn[2] * expf(-st.a[2] * r);
            }
            krow[idx] = v;
        }

        const float scale = st.tdd * st.c2;
        const int n_ug = (out_w + kConvRows - 1) / kConvRows;
        const int n_vg = (out_j1 - out_j0 + kConvCols - 1) / kConvCols;
        const float *fmap = P.fbuf + (long long)b * L.nu * L.nv;
        int fa0 = 0, fa1 = 0, fc0 = 0, fc1 = 0;
        if (!ADJ) {
            fa0 = P.cptab[b].fa0; fa1 = P.cptab[b].fa1;
            fc0 = P.cptab[b].fc0; fc1 = P.cptab[b].fc1;
        }
        const float *hsrc = P.region + (long long)bl * P.cap_o + st.off_o;
        const int h_w = st.oi1 - st.oi0;

        const int rsub = warp % WPR, csub = warp / WPR;
        const int lr = lane % G, lg = lane / G;
        for (int unit = 0; unit < n_ug * n_vg; ++unit) {
            const int ug = unit / n_vg, vg = unit - ug * n_vg;
            const int ibase = out_i0 + kConvRows * ug;
            const int jbase = out_j0 + kConvCols * vg;
            const int r0 = max(ibase - R, in_i0);
            const int r1 = min(ibase + kConvRows + R, in_i1);
            const int cbase = jbase - R;
            __syncthreads();   // previous unit finished reading the tile; krow written
            if (ADJ) {
                // rows fastest: coalesced reads of the [j][i] input box
                const int nr = r1 - r0;
                for (int idx = threadIdx.x; idx < nr * W; idx += blockDim.x) {
                    const int cc = idx / nr, rr = idx - cc * nr;
                    const int u = r0 + rr, jj = cbase + cc;
                    float v = 0.f;
                    if (jj >= in_j0 && jj < in_j1) v = hsrc[(long long)(jj - st.oj0) * h_w + (u - st.oi0)];
                    tile[rr * W + cc] = v;
                }
            } else {
                for (int idx = threadIdx.x; idx < (r1 - r0) * W; idx += blockDim.x) {
                    const int rr = idx / W, cc = idx - rr * W;
                    const int u = r0 + rr, jj = cbase + cc;
                    float v = 0.f;
                    if (jj >= in_j0 && jj < in_j1)
                        v = fluence_sample(fmap, fa0, fa1, fc0, fc1, mag_coord(st.m, u, L.cu),
                                           mag_coord(st.m, jj, L.cv));
                    tile[idx] = v;
                }
            }
            __syncthreads();

            // this warp: rows [wi0, wi0 + G), column blocks [cb0, cb0 + NB)
            const int wi0 = ibase + rsub * G;
            const int wi_last = min(wi0 + G, out_i1) - 1;
            const int cb0 = csub * NB;
            const int wj0 = jbase + kConvTJ * cb0;
            const int wj_end = min(jbase + kConvTJ * (cb0 + NB), out_j1);
            if (wi_last < wi0 || wj0 >= out_j1) continue;   // warp-uniform
            // input rows within R of the warp's rows
            const int ur0 = max(r0, wi0 - R), ur1 = min(r1, wi_last + R + 1);
            // 4-tap chunks that touch non-zero input columns for some block of the
            // warp: chunk c of the block starting at column jw reads input columns
            // jw - R + [4c, 4c + TJ + 3); the union over the warp's blocks takes its
            // lower bound from the last block and its upper bound from the first.
            const int wj_last = wj0 + kConvTJ * (NB - 1);
            const int lo_num = in_j0 - wj_last + R - (kConvTJ + 2);   // need 4c >= lo_num
            const int hi_num = in_j1 - 1 - wj0 + R;                    // need 4c <= hi_num
            const int c_lo = lo_num > 0 ? (lo_num + 3) / 4 : 0;
            const int c_hi = hi_num >= 0 ? min(NQ4, hi_num / 4 + 1) : 0;
            float acc[kConvTJ];
#pragma unroll
            for (int t = 0; t < kConvTJ; ++t) acc[t] = 0.f;
            const int i = wi0 + lr;
            const int jw0 = wj0 + kConvTJ * lg;
            const float *segbase = tile + (jw0 - jbase);
            for (int u = ur0; c_lo < c_hi && u < ur1; ++u) {
                int row = abs(i - u);
                row = row > R ? R + 1 : row;
                conv_row<NQ4>(acc, segbase + (u - r0) * W, krow + row * S, c_lo, c_hi);
            }
            if (i < out_i1 && jw0 < wj_end) {
                float *o = dst + (i - out_i0);
#pragma unroll
                for (int t = 0; t < kConvTJ; ++t) {
                    const int j = jw0 + t;
                    if (j < out_j1) o[(long long)(j - out_j0) * out_w] = acc[t] * scale;
                }
            }
        }
    }
}

// Instantiated tap-quad counts; a radius R uses the smallest NQ4 with
// 4*NQ4 >= 2R+1 (extra taps hold zero weights).
#define PDRT_NQ4_LIST(X) X(3) X(5) X(6) X(7) X(9) X(11) X(14) X(17) X(21) X(23)

int conv_nq4_for_radius(int R)
{
    const int need = (2 * R + 1 + 3) / 4;
    int best = -1;
#define PDRT_PICK(n) if (best < 0 && (n) >= need) best = (n);
    PDRT_NQ4_LIST(PDRT_PICK)
#undef PDRT_PICK
    return best;
}

int conv_smem_bytes(const MachineDev &m)
{
    const int S = kstride_for(m.nq4);
    const int W = conv_tile_width(m.nq4);
    return (int)sizeof(float) * ((m.R + 2) * S + (kConvRows + 2 * m.R) * W);
}

template <int NQ4, bool ADJ>
static cudaError_t launch_one(const PlanDev &P, int b0, int nb, unsigned int *counter, int blocks,
                              cudaStream_t s)
{
    k_conv<NQ4, ADJ, ADJ ? kAdjRowsPerWarp : kFwdRowsPerWarp>
        <<<blocks, kConvThreads, conv_smem_bytes(P.mach), s>>>(P, b0, nb, counter);
    return cudaGetLastError();
}

cudaError_t launch_conv(const PlanDev &P, int b0, int nb, bool adjoint, unsigned int *counter,
                        int grid_blocks, cudaStream_t s)
{
    switch (P.mach.nq4) {
#define PDRT_CASE(n)                                                                        \
    case n:                                                                                 \
        return adjoint ? launch_one<n, true>(P, b0, nb, counter, grid_blocks, s)            \
                       : launch_one<n, false>(P, b0, nb, counter, grid_blocks, s);
        PDRT_NQ4_LIST(PDRT_CASE)
#undef PDRT_CASE
    default:
        return cudaErrorInvalidValue;
    }
}

template <int NQ4, bool ADJ>
static cudaError_t prepare_one(int smem, int *blocks_per_sm)
{
    auto kern = k_conv<NQ4, ADJ, ADJ ? kAdjRowsPerWarp : kFwdRowsPerWarp>;
    cudaError_t e = allow_full_smem(kern);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, kConvThreads, smem);
}

// Sets the dynamic shared-memory limit of the instantiation a machine model
// uses (both directions) on the current device and returns its occupancy.
cudaError_t conv_prepare(const MachineDev &m, int *fwd_blocks_per_sm, int *adj_blocks_per_sm)
{
    const int smem = conv_smem_bytes(m);
    cudaError_t e = cudaErrorInvalidValue;
    switch (m.nq4) {
#define PDRT_PREP(q)                                                                        \
    case q:                                                                                 \
        e = prepare_one<q, false>(smem, fwd_blocks_per_sm);                                 \
        if (e == cudaSuccess) e = prepare_one<q, true>(smem, adj_blocks_per_sm);            \
        break;
        PDRT_NQ4_LIST(PDRT_PREP)
#undef PDRT_PREP
    default:
        break;
    }
    return e;
}

}  // namespace pdrt
