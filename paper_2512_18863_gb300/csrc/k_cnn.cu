// Warm-start network kernels: a 5-layer BF16 CNN (FP32 accumulation) that
// maps beam's-eye-view projections of the target and organs at risk to leaf
// positions and MU per control point (the learned proposal the paper names as
// a future direction in its Discussion), trained by these kernels.
//
// Every contraction of the network (forward, input gradient, weight
// gradient of the four 3x3 stride-2 convolutions and of the dense head) runs
// through one tcgen05 GEMM kernel
//      D[m][n] = sum_k A[m][k] B[n][k]        (A, B BF16, D FP32 in TMEM)
// whose A and B tiles are gathered by threads straight from the NHWC
// activation / weight arrays (implicit im2col, zero outside the image), so no
// im2col matrix is ever written to HBM.  Tiles: M = 128, N = 64 or 128,
// K = 64 per stage, two stages (loads of stage s+1 overlap the MMAs of
// stage s), split-K over blockIdx.z for the weight gradients.  The epilogue
// (bias, ReLU, BF16 rounding, ReLU-mask of the backward pass, split-K
// partials) reads the accumulator with tcgen05.ld.
//
// Data layouts (device, owned by the network handle):
//   activations h_l   [n][H_l][H_l][C_l] BF16 (NHWC), H = 64, 32, 16, 8, 4
//   conv weights W_l  [64][3][3][C_in]   (o, ky, kx, c), K index (ky*3+kx)*C_in + c
//   dense W_5         [121][1024]        input index (y*4 + x)*64 + c
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "pdrt_cnn.h"
#include "pdrt_impl.cuh"
#include "tc_ptx.cuh"

namespace pdrt {
namespace cnn {

constexpr int kGemmThreads = 128;     // 4 warps: warp w owns TMEM lanes 32w..32w+31
constexpr int kBM = 128, kBK = 64;

enum GemmMode {
    G_CONV_FWD = 0,    // z = conv(h_in) + b, out = bf16(relu(z))       M pixels_out, N 64, K 9 C_in
    G_DENSE_FWD = 1,   // out = W5 h4 + b5 (FP32)                      M n, N 121, K 1024
    G_DENSE_DGRAD = 2, // dz4 = bf16((g5 W5) * [h4 > 0])               M n, N 1024, K 121
    G_DENSE_WGRAD = 3, // dW5 = g5^T h4 (split-K partials)              M 121, N 1024, K n
    G_CONV_DGRAD = 4,  // dz_in = bf16(col2im(g_out W) * [h_in > 0])    M pixels_in, N C_in, K 9*64
    G_CONV_WGRAD = 5   // dW = sum_pixels g_out (x) im2col(h_in)        M 9 C_in, N 64, K pixels_out
};

struct GemmArgs {
    int M, N, K;
    int k_per_split;               // multiple of kBK
    const __nv_bfloat16 *a;        // main operand sources (mode-specific)
    const __nv_bfloat16 *b;
    const __nv_bfloat16 *mask;     // ReLU mask source of the dgrad modes
    const float *bias;
    void *out;
    float *part;                   // split-K partials [splits][M * N layout of the mode]
    long long part_stride;         // floats per split
    int hin, hout, cin;            // convolution geometry
    unsigned *flags;
};

__device__ __forceinline__ float bf(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

__device__ __forceinline__ uint4 pack8(const float (&v)[8])
{
    uint4 r;
    r.x = pack2(__float2bfloat16_rn(v[0]), __float2bfloat16_rn(v[1]));
    r.y = pack2(__float2bfloat16_rn(v[2]), __float2bfloat16_rn(v[3]));
    r.z = pack2(__float2bfloat16_rn(v[4]), __float2bfloat16_rn(v[5]));
    r.w = pack2(__float2bfloat16_rn(v[6]), __float2bfloat16_rn(v[7]));
    return r;
}

// Input pixel of output pixel (oy, ox) under kernel tap (ky, kx): 2o + k - 1.
// Element A[m][k] of the implicit im2col matrix of h_in (m = output pixel,
// k = (ky*3 + kx) * cin + c), zero outside the image.
__device__ __forceinline__ const __nv_bfloat16 *im2col_ptr(const GemmArgs &g, int m, int k)
{
    const int per = g.hout * g.hout;
    const int b = m / per, r = m - b * per, oy = r / g.hout, ox = r - oy * g.hout;
    const int kk = k / g.cin, c = k - kk * g.cin, ky = kk / 3, kx = kk - ky * 3;
    const int y = 2 * oy + ky - 1, x = 2 * ox + kx - 1;
    if (y < 0 || y >= g.hin || x < 0 || x >= g.hin) return nullptr;
    return g.a + (((long long)b * g.hin + y) * g.hin + x) * g.cin + c;
}

// 8 consecutive k of row m of A (zero outside [0, M) x [0, K)).
template <int MODE>
__device__ __forceinline__ uint4 load_a8(const GemmArgs &g, int m, int k0)
{
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    if (m >= g.M || k0 >= g.K) return zero;
    if (MODE == G_CONV_FWD) {
        if ((g.cin & 7) == 0) {                     // 8 channels of one tap: one 16-byte load
            const __nv_bfloat16 *p = im2col_ptr(g, m, k0);
            return p ? *reinterpret_cast<const uint4 *>(p) : zero;
        }
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const __nv_bfloat16 *p = (k0 + e < g.K) ? im2col_ptr(g, m, k0 + e) : nullptr;
            v[e] = p ? bf(p) : 0.f;
        }
        return pack8(v);
    } else if (MODE == G_DENSE_FWD) {               // h4 [n][1024]
        return *reinterpret_cast<const uint4 *>(g.a + (long long)m * g.K + k0);
    } else if (MODE == G_DENSE_DGRAD) {             // g5 [n][128] (zero padded past 121)
        return *reinterpret_cast<const uint4 *>(g.a + (long long)m * 128 + k0);
    } else if (MODE == G_DENSE_WGRAD) {             // A[o][b] = g5[b][o]
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = (k0 + e < g.K) ? bf(g.a + (long long)(k0 + e) * 128 + m) : 0.f;
        return pack8(v);
    } else if (MODE == G_CONV_DGRAD) {
        // A[m = input pixel][k = (ky*3+kx)*64 + o] = g_out[b][oy][ox][o] where
        // 2 oy + ky - 1 = y and 2 ox + kx - 1 = x (zero if no such output pixel)
        const int per = g.hin * g.hin;
        const int b = m / per, r = m - b * per, y = r / g.hin, x = r - y * g.hin;
        const int kk = k0 >> 6, o = k0 & 63, ky = kk / 3, kx = kk - ky * 3;
        const int ty = y + 1 - ky, tx = x + 1 - kx;
        if (ty < 0 || tx < 0 || (ty & 1) || (tx & 1)) return zero;
        const int oy = ty >> 1, ox = tx >> 1;
        if (oy >= g.hout || ox >= g.hout) return zero;
        return *reinterpret_cast<const uint4 *>(g.a + (((long long)b * g.hout + oy) * g.hout + ox) * 64 + o);
    } else {                                        // G_CONV_WGRAD: A[(tap, c)][pixel] = im2col^T
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const __nv_bfloat16 *p = (k0 + e < g.K) ? im2col_ptr(g, k0 + e, m) : nullptr;
            v[e] = p ? bf(p) : 0.f;
        }
        return pack8(v);
    }
}

// 8 consecutive k of row n of B (zero outside [0, N) x [0, K)).
template <int MODE>
__device__ __forceinline__ uint4 load_b8(const GemmArgs &g, int n, int k0)
{
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    if (n >= g.N || k0 >= g.K) return zero;
    if (MODE == G_CONV_FWD || MODE == G_DENSE_FWD) {   // weights [N][K] row-major
        if ((g.K & 7) == 0) return *reinterpret_cast<const uint4 *>(g.b + (long long)n * g.K + k0);
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = (k0 + e < g.K) ? bf(g.b + (long long)n * g.K + k0 + e) : 0.f;
        return pack8(v);
    } else if (MODE == G_DENSE_DGRAD) {             // B[i][o] = W5[o][i]
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = (k0 + e < g.K) ? bf(g.b + (long long)(k0 + e) * 1024 + n) : 0.f;
        return pack8(v);
    } else if (MODE == G_DENSE_WGRAD) {             // B[i][b] = h4[b][i]
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = (k0 + e < g.K) ? bf(g.b + (long long)(k0 + e) * 1024 + n) : 0.f;
        return pack8(v);
    } else if (MODE == G_CONV_DGRAD) {              // B[c][(tap)*64 + o] = W[o][tap][c]
        float v[8];
        const int kk = k0 >> 6, o = k0 & 63;
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = bf(g.b + ((long long)(o + e) * 9 + kk) * g.cin + n);
        return pack8(v);
    } else {                                        // G_CONV_WGRAD: B[o][pixel] = g_out[pixel][o]
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = (k0 + e < g.K) ? bf(g.b + (long long)(k0 + e) * 64 + n) : 0.f;
        return pack8(v);
    }
}

// Bounded wait on an mbarrier phase by thread 0; false after ~2^26 polls.
__device__ __forceinline__ bool wait_bounded(void *mbar, uint32_t parity)
{
    long long spins = 0;
    while (!mbar_try(mbar, parity))
        if (++spins > (1LL << 26)) return false;
    return true;
}

template <int MODE>
__device__ __forceinline__ void store16(const GemmArgs &g, int m, int n0, const float (&v)[16], int z)
{
    if (m >= g.M) return;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int n = n0 + q;
        if (n >= g.N) continue;
        const float x = v[q];
        if (MODE == G_CONV_FWD) {
            const float y = fmaxf(x + g.bias[n], 0.f);
            reinterpret_cast<__nv_bfloat16 *>(g.out)[(long long)m * g.N + n] = __float2bfloat16_rn(y);
        } else if (MODE == G_DENSE_FWD) {
            reinterpret_cast<float *>(g.out)[(long long)m * g.N + n] = x + g.bias[n];
        } else if (MODE == G_DENSE_DGRAD || MODE == G_CONV_DGRAD) {
            const long long idx = (long long)m * g.N + n;
            const float y = __bfloat162float(g.mask[idx]) > 0.f ? x : 0.f;
            reinterpret_cast<__nv_bfloat16 *>(g.out)[idx] = __float2bfloat16_rn(y);
        } else if (MODE == G_DENSE_WGRAD) {         // partial of dW5[o = m][i = n]
            g.part[(long long)z * g.part_stride + (long long)m * g.N + n] = x;
        } else {                                    // partial of dW[o = n][(tap, c) = m]
            g.part[(long long)z * g.part_stride + (long long)n * g.M + m] = x;
        }
    }
}

// D tile (128 x NT) of one (m-tile, n-tile, k-split).  Smem per stage: A 128
// rows and B NT rows, K-major core matrices with rows 16 bytes apart: element
// (row, k) at (k / 8) * rows * 16 + row * 16 + (k % 8) * 2.
template <int MODE, int NT>
__global__ void __launch_bounds__(kGemmThreads) k_gemm(GemmArgs g)
{
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);          // [2]
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + 16);
    int *s_ok = reinterpret_cast<int *>(smem + 20);
    unsigned char *stage0 = smem + 128;
    constexpr int kA = kBM * kBK * 2, kB = NT * kBK * 2, kStage = kA + kB;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * NT, z = blockIdx.z;
    const int kb = z * g.k_per_split, ke = min(g.K, kb + g.k_per_split);
    const int n_chunks = ke > kb ? (ke - kb + kBK - 1) / kBK : 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(s_tmem)), "r"((uint32_t)NT));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[0])), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[1])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *s_tmem;
    const uint32_t idesc = instr_desc(kBM, NT);
    uint32_t parity[2] = {0u, 0u};
    bool ok = true;

    for (int c = 0; c < n_chunks && ok; ++c) {
        const int s = c & 1;
        if (c >= 2) {   // stage s was last read by the MMAs of chunk c - 2
            if (tid == 0) *s_ok = wait_bounded(&mbar[s], parity[s]) ? 1 : 0;
            __syncthreads();
            ok = *s_ok != 0;
            parity[s] ^= 1u;
            fence_after();
            if (!ok) break;
        }
        unsigned char *sa = stage0 + s * kStage, *sb = sa + kA;
        const int k0 = kb + c * kBK;
        for (int idx = tid; idx < kBM * (kBK / 8); idx += kGemmThreads) {
            const int kc = idx / kBM, row = idx - kc * kBM;
            *reinterpret_cast<uint4 *>(sa + kc * (kBM * 16) + row * 16) = load_a8<MODE>(g, m0 + row, k0 + 8 * kc);
        }
        for (int idx = tid; idx < NT * (kBK / 8); idx += kGemmThreads) {
            const int kc = idx / NT, row = idx - kc * NT;
            *reinterpret_cast<uint4 *>(sb + kc * (NT * 16) + row * 16) = load_b8<MODE>(g, n0 + row, k0 + 8 * kc);
        }
        fence_proxy_async();
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0) {
            const uint32_t a_s = smem_u32(sa), b_s = smem_u32(sb);
#pragma unroll
            for (int ks = 0; ks < kBK / 16; ++ks) {
                const uint64_t da = smem_desc(a_s + (uint32_t)(2 * ks * kBM * 16), kBM * 16, 128);
                const uint64_t db = smem_desc(b_s + (uint32_t)(2 * ks * NT * 16), NT * 16, 128);
                mma_bf16(tmem, da, db, idesc, (c > 0 || ks > 0) ? 1u : 0u);
            }
            mma_commit(&mbar[s]);
        }
    }
    // drain: the last one or two chunks
    if (ok) {
        for (int c = max(n_chunks - 2, 0); c < n_chunks; ++c) {
            const int s = c & 1;
            if (tid == 0) *s_ok = wait_bounded(&mbar[s], parity[s]) ? 1 : 0;
            __syncthreads();
            ok = ok && *s_ok != 0;
            parity[s] ^= 1u;
            __syncthreads();
        }
    }
    fence_after();
    if (!ok) {
        if (tid == 0) {
            atomicOr(g.flags, (unsigned)PDRT_FLAG_TIMEOUT);
            // bounded waits for MMAs still in flight before the columns are freed
            wait_bounded(&mbar[0], parity[0]);
            wait_bounded(&mbar[1], parity[1]);
        }
    } else {
        const int m = m0 + 32 * warp + lane;
        const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
        for (int cb = 0; cb < NT; cb += 16) {
            float v[16];
            if (n_chunks > 0) {
                tmem_ld16(trow + (uint32_t)cb, v);
            } else {
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = 0.f;
            }
            store16<MODE>(g, m, n0 + cb, v, z);
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)NT));
}

// ---------------------------------------------------------------------------
// Loss, packing, reductions, optimiser
// ---------------------------------------------------------------------------
constexpr int kLossThreads = 1024;

// MSE over n x 121 entries: loss[0] = mean (out - t)^2; g5[b][j] =
// bf16(2 (out - t) / (n 121)) (row stride 128, padding left at 0).
__global__ void __launch_bounds__(kLossThreads) k_mse(const float *__restrict__ out,
                                                     const float *__restrict__ target, int n,
                                                     __nv_bfloat16 *__restrict__ g5,
                                                     float *__restrict__ loss)
{
    __shared__ float s_red[kLossThreads / 32];
    const int total = n * PDRT_CNN_OUT;
    const float inv = 1.f / (float)total;
    float acc = 0.f;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const float d = out[i] - target[i];
        acc = fmaf(d, d, acc);
        const int b = i / PDRT_CNN_OUT, j = i - b * PDRT_CNN_OUT;
        g5[b * 128 + j] = __float2bfloat16_rn(2.f * d * inv);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < kLossThreads / 32 ? s_red[threadIdx.x] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0 && loss) loss[0] = v * inv;
    }
}

// g5[b][j] = bf16(dout[b][j]) for an external upstream gradient.
__global__ void k_pack_g5(const float *__restrict__ dout, int n, __nv_bfloat16 *__restrict__ g5)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * PDRT_CNN_OUT; i += gridDim.x * blockDim.x) {
        const int b = i / PDRT_CNN_OUT, j = i - b * PDRT_CNN_OUT;
        g5[b * 128 + j] = __float2bfloat16_rn(dout[i]);
    }
}

// Column sums of a BF16 matrix [rows][ld] over its first `cols` columns,
// one partial per block: part[blockIdx.x][c] (rows split evenly).
__global__ void __launch_bounds__(256) k_colsum(const __nv_bfloat16 *__restrict__ src, long long rows,
                                                int ld, int cols, float *__restrict__ part)
{
    __shared__ float s_acc[256];
    const long long per = (rows + gridDim.x - 1) / gridDim.x;
    const long long r0 = blockIdx.x * per, r1 = min(rows, r0 + per);
    for (int c0 = 0; c0 < cols; c0 += 64) {
        const int c = c0 + (threadIdx.x & 63), rg = threadIdx.x >> 6;   // 4 row groups
        float acc = 0.f;
        if (c < cols)
            for (long long r = r0 + rg; r < r1; r += 4) acc += __bfloat162float(src[r * ld + c]);
        s_acc[threadIdx.x] = acc;
        __syncthreads();
        if (threadIdx.x < 64 && c < cols)
            part[(long long)blockIdx.x * cols + c] = s_acc[threadIdx.x] + s_acc[threadIdx.x + 64] +
                                                     s_acc[threadIdx.x + 128] + s_acc[threadIdx.x + 192];
        __syncthreads();
    }
}

// dst[i] = sum_z part[z * stride + i], i < count (fixed order: deterministic).
__global__ void k_reduce_parts(const float *__restrict__ part, int splits, long long stride,
                               long long count, float *__restrict__ dst)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += part[z * stride + i];
        dst[i] = s;
    }
}

// Adam (Kingma and Ba, Algorithm 1) on the FP32 master parameters, with the
// BF16 copy the forward reads written in the same pass.  bc1 = 1 - beta1^t,
// bc2 = 1 - beta2^t.
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, __nv_bfloat16 *__restrict__ pbf, long long n, float lr,
                       float beta1, float beta2, float eps, float bc1, float bc2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = beta1 * m[i] + (1.f - beta1) * gi;
        const float vi = beta2 * v[i] + (1.f - beta2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        p[i] = pi;
        pbf[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void k_cast_bf16(const float *__restrict__ p, __nv_bfloat16 *__restrict__ q, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        q[i] = __float2bfloat16_rn(p[i]);
}

// ---------------------------------------------------------------------------
// Beam's-eye-view projection of structure masks (network input)
// ---------------------------------------------------------------------------
// For control point b and BEV pixel (py, px) of a side x side grid of pitch
// `pitch` at the isocentre plane (u = (px - (side-1)/2) pitch along e_u,
// v = (py - (side-1)/2) pitch along e_v), the ray from the source through
// iso + u e_u + v e_v is sampled every `step` mm of depth over +-reach around
// the isocentre plane; channel s is 1 if any sample's nearest voxel carries
// bit s of the mask volume.  Output BF16 [n_cp][side][side][3].
// The sample position decides an integer (the voxel index), so it is taken in
// FP32 with every operation rounded to nearest and in a fixed order (explicit
// _rn intrinsics: no contraction into FMAs), which a reference can reproduce
// bit for bit:
//   half = (side - 1) / 2; u = (px - half) * pitch; v = (py - half) * pitch
//   sxp = ix - sid * sn; syp = iy - sid * cs; szp = iz      (source)
//   dx = u * cs + sid * sn; dy = -(u * sn) + sid * cs; dz = v
//   w = -reach + q * step; t = (sid + w) / sid   (q = 0 .. n_steps - 1)
//   x = sxp + t * dx (likewise y, z); index = rint((x - ox) / sx), ties to even
// with n_steps = floor(2 reach / step) + 1 computed on the host in double and
// cs, sn = (float) cos / sin of (gantry_deg * pi / 180) in double.
struct BevGeo {
    int nx, ny, nz;
    float sx, sy, sz;
    float ox, oy, oz;      // voxel (0,0,0) centre, mm
    float ix, iy, iz;      // isocentre, mm
    float sid, pitch, reach, step;
    int side;
    int n_steps;
};

__device__ __forceinline__ int bev_index(float x, float o, float s)
{
    return __float2int_rn(__fdiv_rn(__fsub_rn(x, o), s));
}

__global__ void k_bev(const uint8_t *__restrict__ masks, BevGeo G, const float2 *__restrict__ cs_sn,
                      __nv_bfloat16 *__restrict__ out)
{
    const int b = blockIdx.y;
    const int pix = blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= G.side * G.side) return;
    const int py = pix / G.side, px = pix - py * G.side;
    const float cs = cs_sn[b].x, sn = cs_sn[b].y;
    const float half = 0.5f * (float)(G.side - 1);
    const float u = __fmul_rn(__fsub_rn((float)px, half), G.pitch);
    const float v = __fmul_rn(__fsub_rn((float)py, half), G.pitch);
    // e_w = (sn, cs, 0), e_u = (cs, -sn, 0), e_v = (0, 0, 1)
    const float sxp = __fsub_rn(G.ix, __fmul_rn(G.sid, sn));
    const float syp = __fsub_rn(G.iy, __fmul_rn(G.sid, cs));
    const float szp = G.iz;
    const float dx = __fadd_rn(__fmul_rn(u, cs), __fmul_rn(G.sid, sn));
    const float dy = __fadd_rn(-__fmul_rn(u, sn), __fmul_rn(G.sid, cs));
    const float dz = v;
    unsigned bits = 0u;
    for (int q = 0; q < G.n_steps; ++q) {
        const float w = __fadd_rn(-G.reach, __fmul_rn((float)q, G.step));   // depth beyond the isocentre plane
        const float t = __fdiv_rn(__fadd_rn(G.sid, w), G.sid);
        const int ix = bev_index(__fadd_rn(sxp, __fmul_rn(t, dx)), G.ox, G.sx);
        const int iy = bev_index(__fadd_rn(syp, __fmul_rn(t, dy)), G.oy, G.sy);
        const int iz = bev_index(__fadd_rn(szp, __fmul_rn(t, dz)), G.oz, G.sz);
        if (ix < 0 || ix >= G.nx || iy < 0 || iy >= G.ny || iz < 0 || iz >= G.nz) continue;
        bits |= masks[((long long)iz * G.ny + iy) * G.nx + ix];
    }
    __nv_bfloat16 *o = out + (((long long)b * G.side + py) * G.side + px) * 3;
#pragma unroll
    for (int s = 0; s < 3; ++s) o[s] = __float2bfloat16_rn((bits >> s) & 1u ? 1.f : 0.f);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
constexpr int kMaxSplits = 64;

// parameter offsets (floats) in the FP32 vector
constexpr long long kW1 = 0, kB1 = kW1 + 64 * 27, kW2 = kB1 + 64, kB2 = kW2 + 64 * 576,
                     kW3 = kB2 + 64, kB3 = kW3 + 64 * 576, kW4 = kB3 + 64, kB4 = kW4 + 64 * 576,
                     kW5 = kB4 + 64, kB5 = kW5 + 121LL * 1024, kParams = kB5 + 121;
constexpr long long kWOff[5] = {kW1, kW2, kW3, kW4, kW5};
constexpr long long kBOff[5] = {kB1, kB2, kB3, kB4, kB5};

}  // namespace cnn
}  // namespace pdrt

using namespace pdrt;
using namespace pdrt::cnn;

struct pdrt_cnn_s {
    int bmax = 0;
    int device = 0;
    int sm_count = 1;
    float *p = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *pbf = nullptr;                   // BF16 copy of the parameters
    __nv_bfloat16 *h[5] = {};                       // h0..h4
    __nv_bfloat16 *dz[5] = {};                      // dz1..dz4 (index = layer)
    __nv_bfloat16 *g5 = nullptr;                    // [bmax][128]
    float *out = nullptr;
    float *part = nullptr;                          // split-K / column-sum partials
    unsigned *flags = nullptr;
    int last_n = 0;
    long long step = 0;
    std::vector<void *> allocs;
};

namespace {

pdrt_status cnn_fail(pdrt_status st, const char *msg)
{
    internal_set_error(msg);
    return st;
}

pdrt_status cnn_cuda(cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    internal_set_error(m.c_str());
    return e == cudaErrorMemoryAllocation ? PDRT_ENOMEM : PDRT_ECUDA;
}

template <typename T>
cudaError_t cnn_alloc(pdrt_cnn_t net, T **p, size_t count)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) {
        net->allocs.push_back(q);
        *p = static_cast<T *>(q);
    }
    return e;
}

int side_of(int layer) { return PDRT_CNN_SIDE >> layer; }   // h_layer side
int ch_of(int layer) { return layer == 0 ? PDRT_CNN_IN_CH : 64; }

template <int NT>
constexpr int gemm_smem() { return 128 + 2 * (kBM * kBK * 2 + NT * kBK * 2); }

template <int MODE, int NT>
cudaError_t gemm_prepare()
{
    return cudaFuncSetAttribute(k_gemm<MODE, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                gemm_smem<NT>());
}

// shared-memory limits of every instantiation on the current device
cudaError_t gemm_prepare_all()
{
    cudaError_t e = gemm_prepare<G_CONV_FWD, 64>();
    if (e == cudaSuccess) e = gemm_prepare<G_DENSE_FWD, 128>();
    if (e == cudaSuccess) e = gemm_prepare<G_DENSE_WGRAD, 128>();
    if (e == cudaSuccess) e = gemm_prepare<G_DENSE_DGRAD, 128>();
    if (e == cudaSuccess) e = gemm_prepare<G_CONV_WGRAD, 64>();
    if (e == cudaSuccess) e = gemm_prepare<G_CONV_DGRAD, 64>();
    return e;
}

template <int MODE, int NT>
cudaError_t gemm_launch(const GemmArgs &g, int splits, cudaStream_t s)
{
    constexpr int smem = gemm_smem<NT>();
    dim3 grid((g.M + kBM - 1) / kBM, (g.N + NT - 1) / NT, splits);
    k_gemm<MODE, NT><<<grid, kGemmThreads, smem, s>>>(g);
    internal_count_launch();
    return cudaGetLastError();
}

// split-K factor: enough CTAs for about two per SM, at least 4 chunks each
int pick_splits(int M, int N, int NT, int K, int sm_count)
{
    const int tiles = ((M + kBM - 1) / kBM) * ((N + NT - 1) / NT);
    const int chunks = (K + kBK - 1) / kBK;
    int s = std::max(1, (2 * sm_count) / std::max(1, tiles));
    s = std::min(s, std::max(1, chunks / 4));
    return std::min(s, kMaxSplits);
}

GemmArgs base_args(pdrt_cnn_t net)
{
    GemmArgs g;
    memset(&g, 0, sizeof(g));
    g.flags = net->flags;
    return g;
}

cudaError_t reduce_parts(pdrt_cnn_t net, int splits, long long stride, long long count, float *dst,
                         cudaStream_t s)
{
    const long long blocks = std::min<long long>((count + 255) / 256, 4LL * net->sm_count);
    k_reduce_parts<<<(unsigned)std::max(1LL, blocks), 256, 0, s>>>(net->part, splits, stride, count, dst);
    internal_count_launch();
    return cudaGetLastError();
}

cudaError_t colsum(pdrt_cnn_t net, const __nv_bfloat16 *src, long long rows, int ld, int cols, float *dst,
                   cudaStream_t s)
{
    const int G = (int)std::max(1LL, std::min<long long>(kMaxSplits, rows / 64));
    k_colsum<<<G, 256, 0, s>>>(src, rows, ld, cols, net->part);
    internal_count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return reduce_parts(net, G, cols, cols, dst, s);
}

cudaError_t run_forward(pdrt_cnn_t net, int n, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    for (int l = 1; l <= 4 && e == cudaSuccess; ++l) {
        GemmArgs g = base_args(net);
        g.hin = side_of(l - 1);
        g.hout = side_of(l);
        g.cin = ch_of(l - 1);
        g.M = n * g.hout * g.hout;
        g.N = 64;
        g.K = 9 * g.cin;
        g.k_per_split = ((g.K + kBK - 1) / kBK) * kBK;
        g.a = net->h[l - 1];
        g.b = net->pbf + kWOff[l - 1];
        g.bias = net->p + kBOff[l - 1];
        g.out = l < 4 ? (void *)net->h[l] : (void *)net->h[4];
        e = gemm_launch<G_CONV_FWD, 64>(g, 1, s);
    }
    if (e != cudaSuccess) return e;
    GemmArgs g = base_args(net);
    g.M = n;
    g.N = PDRT_CNN_OUT;
    g.K = 1024;
    g.k_per_split = 1024;
    g.a = net->h[4];
    g.b = net->pbf + kW5;
    g.bias = net->p + kB5;
    g.out = net->out;
    return gemm_launch<G_DENSE_FWD, 128>(g, 1, s);
}

// backward from g5 (already packed) into net->grad
cudaError_t run_backward(pdrt_cnn_t net, int n, cudaStream_t s)
{
    cudaError_t e;
    {   // dense head: dW5, db5, dz4
        GemmArgs g = base_args(net);
        g.M = PDRT_CNN_OUT;
        g.N = 1024;
        g.K = n;
        const int splits = pick_splits(g.M, g.N, 128, g.K, net->sm_count);
        g.k_per_split = (((g.K + splits - 1) / splits + kBK - 1) / kBK) * kBK;
        const int used = (g.K + g.k_per_split - 1) / g.k_per_split;
        g.a = net->g5;
        g.b = net->h[4];
        g.part = net->part;
        g.part_stride = (long long)PDRT_CNN_OUT * 1024;
        if ((e = gemm_launch<G_DENSE_WGRAD, 128>(g, used, s)) != cudaSuccess) return e;
        if ((e = reduce_parts(net, used, g.part_stride, g.part_stride, net->grad + kW5, s)) != cudaSuccess)
            return e;
        if ((e = colsum(net, net->g5, n, 128, PDRT_CNN_OUT, net->grad + kB5, s)) != cudaSuccess) return e;
        GemmArgs d = base_args(net);
        d.M = n;
        d.N = 1024;
        d.K = PDRT_CNN_OUT;
        d.k_per_split = 128;
        d.a = net->g5;
        d.b = net->pbf + kW5;
        d.mask = net->h[4];
        d.out = net->dz[4];
        if ((e = gemm_launch<G_DENSE_DGRAD, 128>(d, 1, s)) != cudaSuccess) return e;
    }
    for (int l = 4; l >= 1; --l) {
        const int hin = side_of(l - 1), hout = side_of(l), cin = ch_of(l - 1);
        GemmArgs g = base_args(net);
        g.hin = hin;
        g.hout = hout;
        g.cin = cin;
        g.M = 9 * cin;
        g.N = 64;
        g.K = n * hout * hout;
        const int splits = pick_splits(g.M, g.N, 64, g.K, net->sm_count);
        g.k_per_split = (((g.K + splits - 1) / splits + kBK - 1) / kBK) * kBK;
        const int used = (g.K + g.k_per_split - 1) / g.k_per_split;
        g.a = net->h[l - 1];
        g.b = net->dz[l];
        g.part = net->part;
        g.part_stride = 64LL * 9 * cin;
        if ((e = gemm_launch<G_CONV_WGRAD, 64>(g, used, s)) != cudaSuccess) return e;
        if ((e = reduce_parts(net, used, g.part_stride, g.part_stride, net->grad + kWOff[l - 1], s)) !=
            cudaSuccess)
            return e;
        if ((e = colsum(net, net->dz[l], (long long)n * hout * hout, 64, 64, net->grad + kBOff[l - 1], s)) !=
            cudaSuccess)
            return e;
        if (l == 1) break;
        GemmArgs d = base_args(net);
        d.hin = hin;
        d.hout = hout;
        d.cin = cin;
        d.M = n * hin * hin;
        d.N = cin;
        d.K = 9 * 64;
        d.k_per_split = 9 * 64;
        d.a = net->dz[l];
        d.b = net->pbf + kWOff[l - 1];
        d.mask = net->h[l - 1];
        d.out = net->dz[l - 1];
        if ((e = gemm_launch<G_CONV_DGRAD, 64>(d, 1, s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

int64_t pdrt_cnn_param_count(void) { return kParams; }

void pdrt_cnn_destroy(pdrt_cnn_t net)
{
    if (!net) return;
    for (void *q : net->allocs) cudaFree(q);
    delete net;
}

pdrt_status pdrt_cnn_create(pdrt_cnn_t *out, int32_t batch_max, pdrt_stream_t stream)
{
    internal_set_error("");
    if (!out) return cnn_fail(PDRT_EINVAL, "NULL argument");
    *out = nullptr;
    if (batch_max < 1 || batch_max > 65536) return cnn_fail(PDRT_EINVAL, "batch_max must be in 1..65536");
    int dev = 0, major = 0, minor = 0, sms = 1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cnn_cuda(e, "cudaGetDevice");
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (major * 10 + minor != 103) return cnn_fail(PDRT_EDEVICE, "this library is built for sm_103a");
    if ((e = gemm_prepare_all()) != cudaSuccess) return cnn_cuda(e, "network kernel set-up");
    pdrt_cnn_t net = new pdrt_cnn_s();
    net->bmax = batch_max;
    net->device = dev;
    net->sm_count = sms;
    const size_t B = (size_t)batch_max;
    const size_t part = std::max<size_t>((size_t)kMaxSplits * PDRT_CNN_OUT * 1024, 0);
#define CNN_TRY(expr, what)                       \
    do {                                          \
        e = (expr);                               \
        if (e != cudaSuccess) {                   \
            pdrt_status st_ = cnn_cuda(e, what);  \
            pdrt_cnn_destroy(net);                \
            return st_;                           \
        }                                         \
    } while (0)
    CNN_TRY(cnn_alloc(net, &net->p, kParams), "cudaMalloc(parameters)");
    CNN_TRY(cnn_alloc(net, &net->grad, kParams), "cudaMalloc(gradients)");
    CNN_TRY(cnn_alloc(net, &net->m, kParams), "cudaMalloc(adam m)");
    CNN_TRY(cnn_alloc(net, &net->v, kParams), "cudaMalloc(adam v)");
    CNN_TRY(cnn_alloc(net, &net->pbf, kParams), "cudaMalloc(bf16 parameters)");
    for (int l = 0; l <= 4; ++l) {
        const size_t cnt = B * side_of(l) * side_of(l) * ch_of(l);
        CNN_TRY(cnn_alloc(net, &net->h[l], cnt), "cudaMalloc(activation)");
        if (l >= 1) CNN_TRY(cnn_alloc(net, &net->dz[l], cnt), "cudaMalloc(activation gradient)");
    }
    CNN_TRY(cnn_alloc(net, &net->g5, B * 128), "cudaMalloc(output gradient)");
    CNN_TRY(cnn_alloc(net, &net->out, B * PDRT_CNN_OUT), "cudaMalloc(output)");
    CNN_TRY(cnn_alloc(net, &net->part, part), "cudaMalloc(partials)");
    CNN_TRY(cnn_alloc(net, &net->flags, 1), "cudaMalloc(flags)");
    cudaStream_t s = (cudaStream_t)stream;
    CNN_TRY(cudaMemsetAsync(net->p, 0, sizeof(float) * kParams, s), "clear parameters");
    CNN_TRY(cudaMemsetAsync(net->m, 0, sizeof(float) * kParams, s), "clear adam m");
    CNN_TRY(cudaMemsetAsync(net->v, 0, sizeof(float) * kParams, s), "clear adam v");
    CNN_TRY(cudaMemsetAsync(net->pbf, 0, sizeof(__nv_bfloat16) * kParams, s), "clear bf16 parameters");
    CNN_TRY(cudaMemsetAsync(net->g5, 0, sizeof(__nv_bfloat16) * B * 128, s), "clear output gradient");
    CNN_TRY(cudaMemsetAsync(net->flags, 0, sizeof(unsigned), s), "clear flags");
#undef CNN_TRY
    *out = net;
    return PDRT_OK;
}

static pdrt_status check_net(pdrt_cnn_t net)
{
    internal_set_error("");
    if (!net) return cnn_fail(PDRT_EINVAL, "NULL network");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cnn_cuda(e, "cudaGetDevice");
    if (dev != net->device) return cnn_fail(PDRT_EINVAL, "current device differs from the network's");
    return PDRT_OK;
}

pdrt_status pdrt_cnn_set_params(pdrt_cnn_t net, const float *params_dev, pdrt_stream_t stream)
{
    pdrt_status st = check_net(net);
    if (st != PDRT_OK) return st;
    if (!params_dev) return cnn_fail(PDRT_EINVAL, "NULL parameters");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(net->p, params_dev, sizeof(float) * kParams, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(net->m, 0, sizeof(float) * kParams, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(net->v, 0, sizeof(float) * kParams, s);
    if (e != cudaSuccess) return cnn_cuda(e, "set parameters");
    k_cast_bf16<<<4 * net->sm_count, 256, 0, s>>>(net->p, net->pbf, kParams);
    internal_count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return cnn_cuda(e, "cast launch");
    net->step = 0;
    return PDRT_OK;
}

pdrt_status pdrt_cnn_get_params(pdrt_cnn_t net, float *params_dev, pdrt_stream_t stream)
{
    pdrt_status st = check_net(net);
    if (st != PDRT_OK) return st;
    if (!params_dev) return cnn_fail(PDRT_EINVAL, "NULL parameters");
    cudaError_t e = cudaMemcpyAsync(params_dev, net->p, sizeof(float) * kParams, cudaMemcpyDeviceToDevice,
                                    (cudaStream_t)stream);
    return e == cudaSuccess ? PDRT_OK : cnn_cuda(e, "get parameters");
}

pdrt_status pdrt_cnn_forward(pdrt_cnn_t net, const uint16_t *x_dev, int32_t n, float *y_dev,
                             pdrt_stream_t stream)
{
    pdrt_status st = check_net(net);
    if (st != PDRT_OK) return st;
    if (!x_dev || !y_dev) return cnn_fail(PDRT_EINVAL, "NULL buffer");
    if (n < 1 || n > net->bmax) return cnn_fail(PDRT_ESHAPE, "batch size outside 1..batch_max");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t xin = (size_t)n * PDRT_CNN_SIDE * PDRT_CNN_SIDE * PDRT_CNN_IN_CH;
    cudaError_t e = cudaMemcpyAsync(net->h[0], x_dev, xin * 2, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = run_forward(net, n, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(y_dev, net->out, sizeof(float) * n * PDRT_CNN_OUT, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cnn_cuda(e, "network forward");
    net->last_n = n;
    return PDRT_OK;
}

pdrt_status pdrt_cnn_backward(pdrt_cnn_t net, int32_t n, const float *dy_dev, float *grads_dev,
                              pdrt_stream_t stream)
{
    pdrt_status st = check_net(net);
    if (st != PDRT_OK) return st;
    if (!dy_dev) return cnn_fail(PDRT_EINVAL, "NULL upstream gradient");
    if (n != net->last_n || n < 1) return cnn_fail(PDRT_ESHAPE, "backward needs the batch of the last forward");
    cudaStream_t s = (cudaStream_t)stream;
    k_pack_g5<<<std::max(1, std::min(4 * net->sm_count, (n * PDRT_CNN_OUT + 255) / 256)), 256, 0, s>>>(
        dy_dev, n, net->g5);
    internal_count_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = run_backward(net, n, s);
    if (e == cudaSuccess && grads_dev)
        e = cudaMemcpyAsync(grads_dev, net->grad, sizeof(float) * kParams, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? PDRT_OK : cnn_cuda(e, "network backward");
}

pdrt_status pdrt_cnn_train_step(pdrt_cnn_t net, const uint16_t *x_dev, const float *target_dev,
                                int32_t n, float lr, float *loss_dev, pdrt_stream_t stream)
{
    pdrt_status st = check_net(net);
    if (st != PDRT_OK) return st;
    if (!x_dev || !target_dev) return cnn_fail(PDRT_EINVAL, "NULL buffer");
    if (n < 1 || n > net->bmax) return cnn_fail(PDRT_ESHAPE, "batch size outside 1..batch_max");
    if (!(lr > 0.f) || !std::isfinite(lr)) return cnn_fail(PDRT_EINVAL, "learning rate must be positive");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t xin = (size_t)n * PDRT_CNN_SIDE * PDRT_CNN_SIDE * PDRT_CNN_IN_CH;
    cudaError_t e = cudaMemcpyAsync(net->h[0], x_dev, xin * 2, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = run_forward(net, n, s);
    if (e == cudaSuccess) {
        k_mse<<<1, kLossThreads, 0, s>>>(net->out, target_dev, n, net->g5, loss_dev);
        internal_count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = run_backward(net, n, s);
    if (e == cudaSuccess) {
        net->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float bc1 = (float)(1.0 - pow(0.9, (double)net->step));
        const float bc2 = (float)(1.0 - pow(0.999, (double)net->step));
        k_adam<<<4 * net->sm_count, 256, 0, s>>>(net->p, net->grad, net->m, net->v, net->pbf, kParams, lr,
                                                 b1, b2, 1e-8f, bc1, bc2);
        internal_count_launch();
        e = cudaGetLastError();
    }
    net->last_n = n;
    return e == cudaSuccess ? PDRT_OK : cnn_cuda(e, "training step");
}

pdrt_status pdrt_cnn_read_activation(pdrt_cnn_t net, int32_t layer, int32_t n, void *dst_dev,
                                     pdrt_stream_t stream)
{
    pdrt_status st = check_net(net);
    if (st != PDRT_OK) return st;
    if (!dst_dev) return cnn_fail(PDRT_EINVAL, "NULL destination");
    if (layer < 0 || layer > 5) return cnn_fail(PDRT_EINVAL, "layer must be in 0..5");
    if (n != net->last_n || n < 1) return cnn_fail(PDRT_ESHAPE, "n must be the last forward's batch");
    const void *src = layer <= 4 ? (const void *)net->h[layer] : (const void *)net->out;
    const size_t bytes = layer <= 4 ? (size_t)n * side_of(layer) * side_of(layer) * ch_of(layer) * 2
                                    : (size_t)n * PDRT_CNN_OUT * sizeof(float);
    cudaError_t e = cudaMemcpyAsync(dst_dev, src, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    return e == cudaSuccess ? PDRT_OK : cnn_cuda(e, "read activation");
}

pdrt_status pdrt_cnn_status(pdrt_cnn_t net, pdrt_stream_t stream, uint32_t *flags)
{
    pdrt_status st = check_net(net);
    if (st != PDRT_OK) return st;
    if (!flags) return cnn_fail(PDRT_EINVAL, "NULL flags");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    unsigned f = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&f, net->flags, sizeof(f), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(net->flags, 0, sizeof(f));
    if (e != cudaSuccess) return cnn_cuda(e, "read flags");
    *flags = f;
    return PDRT_OK;
}

pdrt_status pdrt_bev_project(const uint8_t *masks_dev, int32_t nx, int32_t ny, int32_t nz,
                             double sx, double sy, double sz, const double origin_mm[3],
                             const double iso_mm[3], double sid_mm, int32_t n_cp,
                             const double *gantry_deg, int32_t side, double pitch_mm,
                             double reach_mm, double step_mm, uint16_t *out_dev,
                             pdrt_stream_t stream)
{
    internal_set_error("");
    if (!masks_dev || !origin_mm || !iso_mm || !gantry_deg || !out_dev)
        return cnn_fail(PDRT_EINVAL, "NULL argument");
    if (nx < 1 || ny < 1 || nz < 1 || n_cp < 1 || n_cp > 65535 || side < 1 || side > 4096)
        return cnn_fail(PDRT_EINVAL, "sizes out of range");
    if (!(sx > 0) || !(sy > 0) || !(sz > 0) || !(pitch_mm > 0) || !(step_mm > 0) || !(reach_mm >= 0) ||
        !(sid_mm > reach_mm))
        return cnn_fail(PDRT_EINVAL, "spacings must be positive and the reach inside the source distance");
    if (2.0 * reach_mm / step_mm > 1e6) return cnn_fail(PDRT_EINVAL, "too many samples per ray");
    BevGeo G;
    G.nx = nx; G.ny = ny; G.nz = nz;
    G.sx = (float)sx; G.sy = (float)sy; G.sz = (float)sz;
    G.ox = (float)origin_mm[0]; G.oy = (float)origin_mm[1]; G.oz = (float)origin_mm[2];
    G.ix = (float)iso_mm[0]; G.iy = (float)iso_mm[1]; G.iz = (float)iso_mm[2];
    G.sid = (float)sid_mm; G.pitch = (float)pitch_mm; G.reach = (float)reach_mm; G.step = (float)step_mm;
    G.side = side;
    G.n_steps = (int)floor(2.0 * reach_mm / step_mm) + 1;
    std::vector<float2> h(n_cp);
    for (int b = 0; b < n_cp; ++b) {
        const double g = gantry_deg[b] * M_PI / 180.0;
        h[b] = make_float2((float)cos(g), (float)sin(g));
    }
    cudaStream_t s = (cudaStream_t)stream;
    float2 *d = nullptr;
    // a small per-call table (n_cp entries) in stream-ordered memory
    cudaError_t e = cudaMallocAsync(&d, sizeof(float2) * n_cp, s);
    if (e != cudaSuccess) return cnn_cuda(e, "cudaMallocAsync(angles)");
    e = cudaMemcpyAsync(d, h.data(), sizeof(float2) * n_cp, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        dim3 grid((side * side + 255) / 256, n_cp);
        k_bev<<<grid, 256, 0, s>>>(masks_dev, G, d, reinterpret_cast<__nv_bfloat16 *>(out_dev));
        internal_count_launch();
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host table goes out of scope
    return e == cudaSuccess ? PDRT_OK : cnn_cuda(e, "beam's-eye-view projection");
}

}  // extern "C"
