// Per-slice lateral convolution (Sec. 2.2.6) on the 5th-generation tensor
// cores (tcgen05.mma, BF16 operands, FP32 accumulation in tensor memory).
//
// For one beam slice, out(i, j) = scale * sum_p sum_s in(i - p, s) K(|p|, j - s)
// (forward: in = magnified fluence, out = D'; adjoint: in = gathered gradient,
// out = h'; K is symmetric, so both are this sum).  Per kernel row p it is a
// GEMM  D[m][n] += A_p[m][k] B_p[n][k]  with m = output row (M = 128 per
// tile, or 64 for a last tile of at most 64 rows), n = output column,
// k = input column (N, K <= 128):
//   * A_p[m][k] = in(i0 + m - p, s_k).  The input tile is stored K-major in
//     8 x 16-byte core matrices with its rows 16 bytes apart, so the shift by
//     p is just a descriptor start address (R - p rows further).
//   * B_p[n][k] = K(|p|, j0 + n - s_k) is Toeplitz in (n, k).  With the K
//     order reversed (s_k = s_end - 1 - k, applied to both operands, which
//     leaves the sum unchanged) it becomes Hankel, h[n + k]; its core matrix
//     (g, c) then depends only on g + c, so one 128-byte core matrix per
//     diagonal is stored and the descriptor uses LBO = SBO = 128 bytes.
// FP32 accuracy: each operand is split x = hi + lo into two BF16 values and
// three products (hi.hi + hi.lo + lo.hi) are accumulated (relative error per
// product <~ 3 * 2^-16).
//
// One CTA (8 warps) per slice, persistent over a work counter.  Warp 0
// issues the MMAs of the kernel rows +p (the whole warp runs the issuing
// loop on warp-uniform descriptors, lane 0 executes the MMAs); in the
// adjoint, for column tiles of at most 64 columns, warp 1 issues those of -p
// into a second accumulator (tensor memory columns 64..127), since one
// issuing thread delivers an MMA only every ~50 cycles while an M = 64 MMA
// with N <= 64 takes ~30.  The kernel-row operands are built in phases of
// PHASE rows (chosen per plan: the deepest phase that keeps the most CTAs per
// SM) into three buffers: while the issuing warps issue phase ph, the other
// warps build phase ph + 1 into the buffer that phase ph - 2 read, after
// waiting for its MMAs; one CTA barrier per phase.  Completion is signalled
// through one mbarrier per issuer and operand buffer (tcgen05.commit); all
// waits are bounded and raise PDRT_FLAG_TIMEOUT.  With the per direction
// tile limits three forward or four adjoint CTAs fit on an SM at R = 20 px,
// and the resident CTAs overlap one another's input-tile builds and
// epilogues with their MMAs.
// Boxes wider than one tile are split into output-column tiles of at most
// MAXN columns and, per column tile, chunks of at most MAXK of the input
// columns within R of it; the chunks accumulate in tensor memory.  With
// tensor cores on this kernel takes every slice; the FP32 SIMT kernel
// (k_conv) skips the slices taken here (tc_takes_slice).
#include <cuda_bf16.h>
#include <math.h>

#include <type_traits>

#include "pdrt_impl.cuh"
#include "tc_ptx.cuh"

namespace pdrt {

namespace {

constexpr int kTcM = 128;
constexpr int kTcThreads = 256;      // 8 warps: two per tensor-memory lane quarter
constexpr uint32_t kTmemCols = 128;   // >= the largest tile width N, power of two
constexpr uint32_t kAcc1Col = 64;     // second accumulator (tiles of N <= 64)
constexpr int kTcBufs = 3;            // kernel-row operand buffers

}  // namespace

__host__ __device__ inline int tc_rows(int R) { return ((kTcM + 2 * R + 7) / 8) * 8; }

template <bool ADJ>
struct TcLimits {
    static constexpr int MAXN = ADJ ? kTcAdjMaxN : kTcFwdMaxN;
    static constexpr int MAXK = ADJ ? kTcAdjMaxK : kTcFwdMaxK;
    static constexpr int ND = MAXN / 8 + MAXK / 8 - 1;   // Hankel diagonals per kernel row
};

// shared memory: [0,128) barriers / tmem address / broadcasts; kernel rows;
// input tile hi+lo [2][K/8][rows][16 B]; kernel-row operands, three buffers
// of `phase` rows x hi+lo x ND core matrices
int conv_tc_smem_bytes(int R, bool adjoint, int phase)
{
    const int rows = tc_rows(R);
    const int maxk = adjoint ? kTcAdjMaxK : kTcFwdMaxK;
    const int nd = adjoint ? TcLimits<true>::ND : TcLimits<false>::ND;
    const int krow = ((R + 1) * (2 * R + 1) * 4 + 127) / 128 * 128;
    const int a = 2 * rows * maxk * 2;
    const int bsz = kTcBufs * phase * 2 * nd * 128;
    return 128 + krow + a + bsz;
}

// Occupancy: the forward at most 80 registers per thread, so three CTAs of
// 256 threads fit the register file (its shared memory with three operand
// buffers allows three per SM); the adjoint at most 64, four CTAs (its
// 48-column input chunks keep the shared memory at four per SM, and four x
// 128 tensor-memory columns fill the 512).  More resident CTAs overlap one
// CTA's input-tile build and epilogue with another's MMAs and add issuing
// warps: the adjoint ran 17 % faster at four CTAs than at two.
template <bool ADJ>
__global__ void __launch_bounds__(kTcThreads, ADJ ? 4 : 3) k_conv_tc(PlanDev P, int b0, int nb,
                                                           unsigned int *__restrict__ counter,
                                                           const int *__restrict__ list,
                                                           const unsigned int *__restrict__ list_n)
{
    using Lim = TcLimits<ADJ>;
    extern __shared__ __align__(128) unsigned char smem[];
    const Lattice &L = P.lat;
    const int R = P.mach.R;
    const int rows = tc_rows(R);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);   // [buffer * 2 + issuer], 6
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + 48);
    int *s_item = reinterpret_cast<int *>(smem + 52);
    // a wait gave up: [phase parity] in the phase loop, [2] in its drain
    volatile int *s_flag = reinterpret_cast<volatile int *>(smem + 56);
    float *krow = reinterpret_cast<float *>(smem + 128);
    const int krow_bytes = ((R + 1) * (2 * R + 1) * 4 + 127) / 128 * 128;
    unsigned char *abase = smem + 128 + krow_bytes;
    const int a_copy = rows * Lim::MAXK * 2;                    // bytes of one (hi or lo) tile
    unsigned char *bbase = abase + 2 * a_copy;
    const int b_row = 2 * Lim::ND * 128;                        // hi + lo of one kernel row
    const int PHASE = ADJ ? P.tc_phase[1] : P.tc_phase[0];   // kernel rows per operand phase
    const int b_buf = PHASE * b_row;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_items = nb * L.nw;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int q = 0; q < 2 * kTcBufs; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[q])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_flag[0] = s_flag[1] = s_flag[2] = 0;
    }
    fence_before();
    __syncthreads();
    fence_after();
    // values the issuing loop depends on are made warp-uniform (lane 0's
    // value) so that its descriptor arithmetic stays warp-uniform
    const uint32_t tmem = __shfl_sync(0xffffffffu, *s_tmem, 0);
    // every thread tracks, in bit q, the parity of the number of commits to
    // barrier q so far (cpar) and whether q was ever committed (cused); the
    // commits are a function of the phase sequence, identical in all threads
    uint32_t cpar = 0u, cused = 0u;
    bool timed_out = false;

    while (!timed_out) {
        if (tid == 0) {
            // list mode: the items the FFT kernel left (slices beyond its size
            // limit), else every item of the chunk
            const int q = (int)atomicAdd(counter, 1u);
            *s_item = list ? (q < (int)*list_n ? list[q] : n_items) : q;
        }
        __syncthreads();
        const int item = *s_item;
        __syncthreads();
        if (item >= n_items) break;
        const int bl = item / L.nw, k = item - bl * L.nw, b = b0 + bl;
        const SliceTab st = P.slices[(long long)b * L.nw + k];
        if (!tc_takes_slice(st, ADJ, R, 1)) continue;
        const TcBoxes bx = tc_boxes(st, ADJ, R);
        const int out_w = bx.out_i1 - bx.out_i0;
        float *dst = ADJ ? P.adjbuf + (long long)bl * P.cap_a + st.off_a
                         : P.region + (long long)bl * P.cap_o + st.off_o;
        const float scale = st.tdd * st.c2;

        // kernel rows K(|p|, q), q in [-R, R]; K(|p|, -q) = K(|p|, q) (the same
        // float expression: r depends on q * q), so q >= 0 is computed and mirrored
        for (int idx = tid; idx < (R + 1) * (R + 1); idx += blockDim.x) {
            const int p = idx / (R + 1), q = idx - p * (R + 1);
            const float pu = p * L.du, qv = q * L.dv;
            const float r = sqrtf(pu * pu + qv * qv);
            const float v = st.wn[0] * expf(-st.a[0] * r) + st.wn[1] * expf(-st.a[1] * r) +
                            st.wn[2] * expf(-st.a[2] * r);
            krow[p * (2 * R + 1) + R + q] = v;
            krow[p * (2 * R + 1) + R - q] = v;
        }
        __syncthreads();
        // Tiling of the slice: output-column tiles of at most MAXN columns
        // (balanced widths), and per column tile chunks of at most MAXK of the
        // input columns within R of it; the chunks accumulate in tensor memory.
        int nt = 16, kt = 16, nd = 1, s_end = 0, c0 = 0;
        // Hankel core matrices of kernel rows |p| in [p0, p1) into buffer `buf`:
        // element (r, t) of diagonal d = K(|p|, 8d + r + t + c0), c0 = j0 - s_end + 1
        auto build_b = [&](int p0, int p1, int buf, const int nd, const int c0, int t0, int ts) {
            const int n = (p1 - p0) * nd * 8;
            for (int idx = t0; idx < n; idx += ts) {
                const int pl = idx / (nd * 8), rem = idx - pl * nd * 8, d = rem >> 3, r = rem & 7;
                const int p = p0 + pl;
                uint32_t hw[4], lw[4];
#pragma unroll
                for (int t = 0; t < 8; t += 2) {
                    __nv_bfloat16 h0, l0, h1, l1;
                    const int q0 = 8 * d + r + t + c0, q1 = q0 + 1;
                    const float v0 = (q0 >= -R && q0 <= R) ? krow[p * (2 * R + 1) + q0 + R] : 0.f;
                    const float v1 = (q1 >= -R && q1 <= R) ? krow[p * (2 * R + 1) + q1 + R] : 0.f;
                    split_bf16(v0, h0, l0);
                    split_bf16(v1, h1, l1);
                    hw[t >> 1] = pack2(h0, h1);
                    lw[t >> 1] = pack2(l0, l1);
                }
                unsigned char *bp = bbase + (size_t)buf * b_buf + (size_t)pl * b_row + (size_t)d * 128 + r * 16;
                *reinterpret_cast<uint4 *>(bp) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                *reinterpret_cast<uint4 *>(bp + (size_t)Lim::ND * 128) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
        };
        const int n_ph = (R + PHASE) / PHASE;   // phases over |p| = 0..R
        const float *fmap = P.fbuf + (long long)b * L.nu * L.nv;
        const int fa0 = P.cptab[b].fa0, fa1 = P.cptab[b].fa1, fc0 = P.cptab[b].fc0, fc1 = P.cptab[b].fc1;
        const float *hsrc = P.region + (long long)bl * P.cap_o + st.off_o;
        const int h_w = st.oi1 - st.oi0;
        const int lbo_a = rows * 16;
        // Descriptors are built once; every operand offset is a multiple of 16
        // bytes and smem addresses stay below 256 KB, so the descriptor of
        // base + off is the base descriptor + (off >> 4) in its 14-bit
        // start-address field (no carry out of the field).
        const uint32_t a_hi0 = smem_u32(abase);
        const uint64_t da_hi0 = smem_desc(a_hi0, lbo_a, 128);
        const uint64_t da_lo0 = smem_desc(a_hi0 + (uint32_t)a_copy, lbo_a, 128);
        const uint64_t db0 = smem_desc(smem_u32(bbase), 128, 128);
        const uint32_t a_ks = (2u * (uint32_t)lbo_a) >> 4;   // per K step
        const uint32_t b_ks = (2u * 128u) >> 4;
        const uint32_t desc_hi = (uint32_t)(da_hi0 >> 32);    // SBO 128 and version: common to all operands
        const uint64_t b_lo_off = (uint64_t)(((uint32_t)Lim::ND * 128u) >> 4);
        uint32_t acc = 0;   // per issuing warp: its accumulator holds a partial sum
        // Phase ph (kernel rows |p| in [ph*PHASE, ...)) reads operand buffer
        // ph % 3; each issuer commits to mbar[2 (ph % 3) + issuer].  Issuer 0
        // (warp 0) takes the rows +p into columns [0, N); with two issuers,
        // issuer 1 (warp 1) takes the rows -p into columns [64, 64 + N),
        // otherwise issuer 0 takes both and issuer 1 does nothing.  Each
        // issuer's lane 0 executes its MMAs and commits.
        // (the issuer is a compile-time constant: the issuing warp's
        // instruction stream bounds the MMA rate, so its loop stays lean)
        auto issue = [&](int ph, const int n_ks, const uint32_t idesc, auto who_c, const bool two) {
            constexpr int who = decltype(who_c)::value;
            const int p0 = ph * PHASE, p1 = min(p0 + PHASE, R + 1), buf = ph % kTcBufs;
            const uint64_t db_buf = db0 + (uint64_t)(((uint32_t)(buf * b_buf)) >> 4);
            const uint32_t dacc = tmem + (who ? kAcc1Col : 0u);
            for (int ap = (who ? max(p0, 1) : p0); ap < p1; ++ap) {
                const uint64_t dbh_row = db_buf + (uint64_t)(((uint32_t)((ap - p0) * b_row)) >> 4);
                const uint64_t dbl_row = dbh_row + b_lo_off;
                // issuer 0: sign +1, and -1 too unless a second issuer takes it;
                // issuer 1: sign -1 (ap >= 1)
                const int sg0 = who ? -1 : ((ap == 0 || two) ? 1 : -1);
                const int sg1 = who ? -1 : 1;
                for (int sg = sg0; sg <= sg1; sg += 2) {
                    // descriptor low words (start address >> 4 in bits 0-13)
                    const uint32_t row = (uint32_t)(R - sg * ap);      // rows 16 B apart
                    uint32_t dah = (uint32_t)da_hi0 + row, dal = (uint32_t)da_lo0 + row;
                    uint32_t dbh = (uint32_t)dbh_row, dbl = (uint32_t)dbl_row;
                    for (int ks = 0; ks < n_ks; ++ks) {
                        mma3_warp(dacc, dah, dal, dbh, dbl, desc_hi, idesc, acc);
                        acc = 1;
                        dah += a_ks;
                        dal += a_ks;
                        dbh += b_ks;
                        dbl += b_ks;
                    }
                }
            }
            // issuer 1 commits only in phases where it issued (rows |p| >= 1)
            if (who == 0 || p1 > max(p0, 1)) mma_commit_warp(&mbar[2 * buf + who]);
        };
        using Iss0 = std::integral_constant<int, 0>;
        using Iss1 = std::integral_constant<int, 1>;
        // does issuer 1 commit in phase ph (it takes rows |p| >= 1 only)
        auto commits1 = [&](int ph, const bool two) {
            const int p0 = ph * PHASE, p1 = min(p0 + PHASE, R + 1);
            return two && p1 > max(p0, 1);
        };
        // all threads note the commits of phase ph
        auto note_commits = [&](int ph, const bool two) {
            const uint32_t m = (commits1(ph, two) ? 3u : 1u) << (2 * (ph % kTcBufs));
            cpar ^= m;
            cused |= m;
        };
        // bounded wait of a warp (its lane 0 polls) for the latest commit to
        // barrier q
        auto poll_q = [&](int q) -> bool {
            int ok = 1;
            if (lane == 0) {
                const uint32_t par = ((cpar >> q) & 1u) ^ 1u;
                long long spins = 0;
                while (!mbar_try(&mbar[q], par)) {
                    if (++spins > (1LL << 28)) {
                        ok = 0;
                        break;
                    }
                }
            }
            __syncwarp();
            return __shfl_sync(0xffffffffu, ok, 0) != 0;
        };
        // the commits of phase ph (no later phase has reused its buffer)
        auto poll_phase = [&](int ph, const bool two) -> bool {
            const int q = 2 * (ph % kTcBufs);
            bool ok = poll_q(q);
            if (ok && commits1(ph, two)) ok = poll_q(q + 1);
            return ok;
        };
        const int ow = bx.out_j1 - bx.out_j0;
        const int n_ct = (ow + Lim::MAXN - 1) / Lim::MAXN;
        const int w_ct = (((ow + n_ct - 1) / n_ct) + 15) & ~15;   // <= MAXN (a multiple of 16)

        int tile_m = kTcM;
        for (int i0 = bx.out_i0; i0 < bx.out_i1 && !timed_out; i0 += tile_m) {
            // a last tile of at most 64 rows runs as M = 64 (half the A reads).
            // Forward: every A row the MMAs read, [0, M + 2R), is built (zero
            // outside the input box).  Adjoint: only rows [0, h + 2R) for the
            // h output rows of the tile (measured faster); the rows after them
            // keep earlier contents and feed only accumulator rows >= h, which
            // are never stored.
            tile_m = (bx.out_i1 - i0 <= 64) ? 64 : kTcM;
            const int arows = min(rows, ((min(tile_m, ADJ ? bx.out_i1 - i0 : tile_m) + 2 * R + 7) / 8) * 8);
            const int r0 = i0 - R;   // input row of tile row 0
            for (int ct = 0; ct < n_ct && !timed_out; ++ct) {
                const int j0 = bx.out_j0 + ct * w_ct, j1 = min(bx.out_j1, j0 + w_ct);
                nt = ((j1 - j0) + 15) & ~15;
                const uint32_t idesc = __shfl_sync(0xffffffffu, instr_desc(tile_m, nt), 0);
                // second issuer and accumulator (adjoint: measured faster; the
                // forward's wider tiles keep one issuer)
                const bool two = __shfl_sync(0xffffffffu, (int)(ADJ && nt <= (int)kAcc1Col && R >= 1), 0) != 0;
                const int sa = max(bx.in_j0, j0 - R), sb = min(bx.in_j1, j0 + nt + R);
                const int n_kc = sb > sa ? (sb - sa + Lim::MAXK - 1) / Lim::MAXK : 0;
                const int w_kc = n_kc ? (((sb - sa + n_kc - 1) / n_kc) + 15) & ~15 : 16;
                acc = 0;
                for (int kc_i = 0; kc_i < n_kc && !timed_out; ++kc_i) {
                    // input columns [ka, kb) of this chunk; K position k holds
                    // column s_end - 1 - k (reversed order, Hankel kernel operand)
                    const int ka = sa + kc_i * w_kc, kb = min(sb, ka + w_kc);
                    kt = ((kb - ka) + 15) & ~15;
                    s_end = ka + kt;
                    c0 = j0 - s_end + 1;
                    nd = nt / 8 + kt / 8 - 1;
                    // the previous chunk's MMAs have completed (waited); before the
                    // first chunk the previous epilogue's barrier already holds
                    if (kc_i > 0) __syncthreads();
                    // input tile: element (row, k) = in(r0 + row, s_end - 1 - k), hi/lo BF16,
                    // 8 consecutive k per thread item (one 16-byte core-matrix row)
                    for (int idx = tid; idx < arows * (kt / 8); idx += blockDim.x) {
                        const int kcol = idx / arows, row = idx - kcol * arows;
                        const int u = r0 + row;
                        unsigned char *ap = abase + (size_t)kcol * lbo_a + row * 16;
                        // the item's 8 input columns, s_end - 8 (kcol + 1) .. s_end - 1 - 8 kcol
                        const int s_hi = s_end - 1 - 8 * kcol, s_lo = s_hi - 7;
                        if (u < bx.in_i0 || u >= bx.in_i1 || s_hi < ka || s_lo >= kb) {
                            // outside the input box: zeros
                            *reinterpret_cast<uint4 *>(ap) = make_uint4(0u, 0u, 0u, 0u);
                            *reinterpret_cast<uint4 *>(ap + a_copy) = make_uint4(0u, 0u, 0u, 0u);
                            continue;
                        }
                        // forward: the row's magnified coordinate, once per item
                        float ta = 0.f;
                        int a0 = 0;
                        if (!ADJ) {
                            const float fa = mag_coord(st.m, u, L.cu);
                            const float ba = floorf(fa);
                            a0 = (int)ba;
                            ta = fa - ba;
                        }
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int t = 0; t < 8; t += 2) {
                            float v[2];
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                const int s = s_hi - (t + e);
                                float x = 0.f;
                                if (s >= ka && s < kb) {
                                    if (ADJ) {
                                        x = hsrc[(long long)(s - st.oj0) * h_w + (u - st.oi0)];
                                    } else {
                                        const float fc = mag_coord(st.m, s, L.cv);
                                        const float bc = floorf(fc);
                                        const int cc0 = (int)bc;
                                        const float tc = fc - bc;
                                        const int Fc = fc1 - fc0;
#pragma unroll
                                        for (int da = 0; da < 2; ++da) {
                                            const int a = a0 + da;
                                            if (a < fa0 || a >= fa1) continue;
                                            const float wa = da ? ta : 1.f - ta;
#pragma unroll
                                            for (int dc = 0; dc < 2; ++dc) {
                                                const int c = cc0 + dc;
                                                if (c < fc0 || c >= fc1) continue;
                                                const float wc = dc ? tc : 1.f - tc;
                                                x += wa * wc * __ldg(&fmap[(long long)(a - fa0) * Fc + (c - fc0)]);
                                            }
                                        }
                                    }
                                }
                                v[e] = x;
                            }
                            __nv_bfloat16 h0, l0, h1, l1;
                            split_bf16(v[0], h0, l0);
                            split_bf16(v[1], h1, l1);
                            hw[t >> 1] = pack2(h0, h1);
                            lw[t >> 1] = pack2(l0, l1);
                        }
                        *reinterpret_cast<uint4 *>(ap) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        *reinterpret_cast<uint4 *>(ap + a_copy) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    }
                    const int n_ks = __shfl_sync(0xffffffffu, kt / 16, 0);
                    // Three operand buffers: the issuing warps issue phase ph
                    // from buffer ph % 3 while the other warps build phase ph + 1
                    // into buffer (ph + 1) % 3, which phase ph - 2 read last
                    // (its commits are waited on first); one CTA barrier per
                    // phase.
                    const int n_iw = two ? 2 : 1;   // issuing warps
                    build_b(0, min(PHASE, R + 1), 0, nd, c0, tid, kTcThreads);
                    fence_proxy_async();   // generic-proxy smem writes -> tensor core reads
                    fence_before();
                    __syncthreads();
                    fence_after();
                    for (int ph = 0; ph < n_ph; ++ph) {
                        if (warp == 0) {
                            issue(ph, n_ks, idesc, Iss0{}, two);
                        } else if (ADJ && two && warp == 1) {
                            issue(ph, n_ks, idesc, Iss1{}, two);
                        } else if (ph + 1 < n_ph) {
                            if (ph < 2 || poll_phase(ph - 2, two))
                                build_b((ph + 1) * PHASE, min((ph + 2) * PHASE, R + 1), (ph + 1) % kTcBufs, nd, c0,
                                        tid - 32 * n_iw, kTcThreads - 32 * n_iw);
                            else
                                s_flag[ph & 1] = 1;
                        }
                        note_commits(ph, two);
                        fence_proxy_async();
                        fence_before();
                        __syncthreads();
                        fence_after();
                        // a flag is written before the barrier of its own phase
                        // only and read by every thread before the next barrier,
                        // so all threads take the same branch
                        if (s_flag[ph & 1]) {
                            timed_out = true;
                            break;
                        }
                    }
                    // every MMA of the chunk complete before the epilogue or the
                    // next chunk: the phases not yet waited on (the last three)
                    if (!timed_out) {
                        for (int ph = max(n_ph - kTcBufs, 0); ph < n_ph; ++ph)
                            if (!poll_phase(ph, two)) s_flag[2] = 1;
                        fence_before();
                        __syncthreads();
                        fence_after();
                        if (s_flag[2]) timed_out = true;
                    }
                }
                if (timed_out) {
                    if (tid == 0) {
                        atomicOr(P.flags, (unsigned)PDRT_FLAG_TIMEOUT);
                        // second bounded waits for MMAs still in flight before the
                        // tensor memory is released
                        for (int q = 0; q < 2 * kTcBufs; ++q) {
                            long long spins = 0;
                            while (((cused >> q) & 1u) && !mbar_try(&mbar[q], ((cpar >> q) & 1u) ^ 1u) &&
                                   ++spins < (1LL << 28)) {
                            }
                        }
                    }
                    break;
                }
                // epilogue: warp w reads TMEM lanes [32 (w % 4), +32); accumulator
                // row m sits in lane m (M = 128) or in lane 32 (m / 16) + m % 16
                // (M = 64: lanes 16..31 of each quarter unused).  The two warps
                // of a lane quarter take alternate 16-column blocks; the tile
                // writes its own columns [j0, j1); with two issuers the output
                // is the sum of both accumulators (fixed order).
                const int quarter = warp & 3, half = warp >> 2;
                const bool lane_ok = tile_m == kTcM || lane < 16;
                const int i = i0 + (tile_m == kTcM ? 32 : 16) * quarter + lane;
                const uint32_t trow = tmem + ((uint32_t)(32 * quarter) << 16);
                for (int cb = 16 * half; cb < nt; cb += 32) {
                    float v[16];
                    if (n_kc > 0) {
                        tmem_ld16(trow + (uint32_t)cb, v);
                        if (two) {
                            float v1[16];
                            tmem_ld16(trow + kAcc1Col + (uint32_t)cb, v1);
#pragma unroll
                            for (int q = 0; q < 16; ++q) v[q] += v1[q];
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; ++q) v[q] = 0.f;
                    }
                    if (lane_ok && i < bx.out_i1) {
                        float *o = dst + (i - bx.out_i0);
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const int j = j0 + cb + q;
                            if (j < j1) o[(long long)(j - bx.out_j0) * out_w] = v[q] * scale;
                        }
                    }
                }
                fence_before();
                __syncthreads();   // TMEM reads done before the next tile's MMAs
                fence_after();
            }
        }
    }
    __syncthreads();
    fence_after();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

cudaError_t launch_conv_tc(const PlanDev &P, int b0, int nb, bool adjoint, unsigned int *counter,
                           int grid_blocks, cudaStream_t s, const int *list, const unsigned int *list_n)
{
    const int smem = conv_tc_smem_bytes(P.mach.R, adjoint, P.tc_phase[adjoint ? 1 : 0]);
    if (adjoint)
        k_conv_tc<true><<<grid_blocks, kTcThreads, smem, s>>>(P, b0, nb, counter, list, list_n);
    else
        k_conv_tc<false><<<grid_blocks, kTcThreads, smem, s>>>(P, b0, nb, counter, list, list_n);
    return cudaGetLastError();
}

// CTAs of one direction that fit on an SM: shared memory (with the per-block
// reservation), registers and tensor-memory columns.  Computed from the
// device limits; the persistent kernel is correct with any grid (CTAs only
// pull work items and never wait for one another), so a grid larger than
// what is resident only queues.
template <bool ADJ>
static cudaError_t tc_ctas_per_sm(int R, int phase, int *out)
{
    int dev = 0, smem_sm = 0, resv = 0, regs_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_conv_tc<ADJ>);
    if (e != cudaSuccess) return e;
    const int per_cta = conv_tc_smem_bytes(R, ADJ, phase) + (int)fa.sharedSizeBytes + resv;
    const int by_smem = smem_sm / per_cta;
    const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
    const int by_regs = regs_sm / (regs_warp * (kTcThreads / 32));
    const int by_tmem = 512 / (int)kTmemCols;   // each CTA holds kTmemCols of 512 columns
    int n = by_smem < by_regs ? by_smem : by_regs;
    n = n < by_tmem ? n : by_tmem;
    *out = n;
    return cudaSuccess;
}

cudaError_t conv_tc_ctas(int R, bool adjoint, int phase, int *ctas)
{
    *ctas = 0;
    if (phase < 1 || conv_tc_smem_bytes(R, adjoint, phase) > 220 * 1024) return cudaSuccess;
    return adjoint ? tc_ctas_per_sm<true>(R, phase, ctas) : tc_ctas_per_sm<false>(R, phase, ctas);
}

// Per direction: the phase depth (kernel rows per operand buffer, 4..1) that
// gives the most CTAs per SM, the deepest one among equals (fewer barriers).
template <bool ADJ>
static cudaError_t pick_phase(int R, int *blocks, int *phase)
{
    *blocks = 0;
    *phase = 1;
    for (int ph = 4; ph >= 1; --ph) {
        if (conv_tc_smem_bytes(R, ADJ, ph) > 220 * 1024) continue;
        int n = 0;
        cudaError_t e = tc_ctas_per_sm<ADJ>(R, ph, &n);
        if (e != cudaSuccess) return e;
        if (n > *blocks) {
            *blocks = n;
            *phase = ph;
        }
    }
    return cudaSuccess;
}

cudaError_t conv_tc_prepare(int R, int *fwd_blocks_per_sm, int *adj_blocks_per_sm, int *fwd_phase,
                            int *adj_phase)
{
    cudaError_t e = allow_full_smem(k_conv_tc<false>);
    if (e == cudaSuccess) e = allow_full_smem(k_conv_tc<true>);
    if (e == cudaSuccess) e = pick_phase<false>(R, fwd_blocks_per_sm, fwd_phase);
    if (e == cudaSuccess) e = pick_phase<true>(R, adj_blocks_per_sm, adj_phase);
    return e;
}

}  // namespace pdrt
