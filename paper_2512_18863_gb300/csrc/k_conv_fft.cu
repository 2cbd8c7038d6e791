// Per-slice lateral convolution (Sec. 2.2.6) by FFT, FP32 on the CUDA cores.
//
// For one beam slice with input box I (forward: the non-zero fluence volume;
// adjoint: the gathered gradient on the forward's output box) and output box
// O, out(i, j) = scale * sum_p sum_q in(i - p, j - q) K(|p|, |q|) for
// |p|, |q| <= R (K is even in p and in q, so the adjoint is the same sum).
// It is a linear convolution, computed as a circular one of period (Pu, Pv)
// in (u, v) with every input point placed at its offset from the box corner:
// Pu = the smallest supported size >= max(O.i1 - 1 - I.i0, I.i1 - 1 - O.i0)
// + R + 1 (likewise Pv), so no tap within R wraps onto an output and no tap
// beyond R reaches one.  Per slice, in one CTA:
//   1. kernel spectrum.  K is real and even, so its DFT is real and
//      separable into cosine sums over the quadrant p, q in [0, R]:
//        A(p, kv)  = sum_q c_q K(p, q) cos(2 pi kv q / Pv)
//        Kf(ku, kv) = sum_p c_p cos(2 pi ku p / Pu) A(p, kv),  c_0 = 1, c_>0 = 2,
//      for ku <= Pu/2 and kv <= Pv/2 (Kf is even in kv), scaled by
//      scale / (Pu Pv);
//   2. real FFT along u of every input row: the row's Pu reals packed as
//      Pu/2 complex pairs, a complex FFT of length Pu/2 and the standard
//      split into the Pu/2 + 1 non-redundant frequencies;
//   3. complex FFT along v of those Pu/2 + 1 columns;
//   4. product with Kf, inverse FFT along v, inverse real FFT along u of the
//      output rows, and the output box written out.
// The complex FFTs are in place in shared memory: mixed-radix (2, 3, 4, 5,
// 8, 9, 16) decimation in frequency forward, leaving the spectrum in
// digit-reversed order, and decimation in time backward, which takes that
// order and returns natural order, so no reordering pass exists; every
// element belongs to one butterfly per pass and one barrier separates the
// passes.  Twiddles come from per-size tables (sincospif), the index maps of
// the digit reversal from small tables.
// Slices whose sizes exceed the plan's limit (the shared memory was sized
// for it) are appended to an overflow list that the tensor-core kernel
// takes next.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "pdrt_impl.cuh"

namespace pdrt {

namespace {

constexpr int kFftThreads = 256;
constexpr int kNumFftSizes = 16;

struct Radices {
    int np;
    int r[3];
};

// radix passes of a complex transform length (first pass first): every
// supported length in at most two passes
__host__ __device__ inline Radices radices_of(int n)
{
    switch (n) {
    case 16: return {1, {16, 1, 1}};
    case 20: return {2, {4, 5, 1}};
    case 24: return {2, {8, 3, 1}};
    case 30: return {2, {6, 5, 1}};
    case 32: return {2, {8, 4, 1}};
    case 36: return {2, {6, 6, 1}};
    case 40: return {2, {8, 5, 1}};
    case 45: return {2, {9, 5, 1}};
    case 48: return {2, {16, 3, 1}};
    case 50: return {2, {10, 5, 1}};
    case 54: return {2, {6, 9, 1}};
    case 60: return {2, {12, 5, 1}};
    case 64: return {2, {8, 8, 1}};
    case 72: return {2, {8, 9, 1}};
    case 80: return {2, {16, 5, 1}};
    case 90: return {2, {10, 9, 1}};
    case 96: return {2, {16, 6, 1}};
    case 100: return {2, {10, 10, 1}};
    case 108: return {2, {12, 9, 1}};
    case 120: return {2, {12, 10, 1}};
    case 128: return {2, {16, 8, 1}};
    case 144: return {2, {16, 9, 1}};
    case 160: return {2, {16, 10, 1}};
    case 192: return {2, {16, 12, 1}};
    default: return {0, {1, 1, 1}};
    }
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// small DFTs in registers: y_q = sum_m v_m exp(S 2 pi i m q / R), S = +-1
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// S i a
template <int S>
__device__ __forceinline__ float2 mul_si(float2 a)
{
    return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <int S>
__device__ __forceinline__ void dft2(float2 &a, float2 &b)
{
    const float2 t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <int S>
__device__ __forceinline__ void dft4(float2 &v0, float2 &v1, float2 &v2, float2 &v3)
{
    const float2 a0 = cadd(v0, v2), a1 = csub(v0, v2), a2 = cadd(v1, v3), a3 = mul_si<S>(csub(v1, v3));
    v0 = cadd(a0, a2);
    v2 = csub(a0, a2);
    v1 = cadd(a1, a3);
    v3 = csub(a1, a3);
}

template <int S>
__device__ __forceinline__ void dft8(float2 *v)
{
    // even and odd halves, then the radix-2 combination with W8^q
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<S>(e0, e1, e2, e3);
    dft4<S>(o0, o1, o2, o3);
    const float h = 0.70710678118654752f;
    const float2 t1 = make_float2(h * (o1.x - S * o1.y), h * (o1.y + S * o1.x));    // W8^1 o1
    const float2 t2 = mul_si<S>(o2);                                                 // W8^2 o2
    const float2 t3 = make_float2(-h * (o3.x + S * o3.y), h * (S * o3.x - o3.y));   // W8^3 o3
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, t1); v[5] = csub(e1, t1);
    v[2] = cadd(e2, t2); v[6] = csub(e2, t2);
    v[3] = cadd(e3, t3); v[7] = csub(e3, t3);
}

template <int S>
__device__ __forceinline__ void dft16(float2 *v)
{
    float2 e[8], o[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        e[m] = v[2 * m];
        o[m] = v[2 * m + 1];
    }
    dft8<S>(e);
    dft8<S>(o);
    // W16^q = cos(q pi / 8) + S i sin(q pi / 8), q = 0..7
    const float c[8] = {1.f, 0.92387953251128676f, 0.70710678118654752f, 0.38268343236508977f,
                        0.f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128676f};
    const float s[8] = {0.f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128676f,
                        1.f, 0.92387953251128676f, 0.70710678118654752f, 0.38268343236508977f};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float2 w = make_float2(c[q], S * s[q]);
        const float2 t = cmul(w, o[q]);
        v[q] = cadd(e[q], t);
        v[q + 8] = csub(e[q], t);
    }
}

template <int S>
__device__ __forceinline__ void dft3(float2 &v0, float2 &v1, float2 &v2)
{
    const float h = 0.86602540378443865f;   // sin(2 pi / 3)
    const float2 t = cadd(v1, v2);
    const float2 d = mul_si<S>(cscale(csub(v1, v2), h));
    const float2 a = make_float2(v0.x - 0.5f * t.x, v0.y - 0.5f * t.y);
    v0 = cadd(v0, t);
    v1 = cadd(a, d);
    v2 = csub(a, d);
}

template <int S>
__device__ __forceinline__ void dft5(float2 *v)
{
    const float c1 = 0.30901699437494742f, c2 = -0.80901699437494742f;   // cos(2 pi / 5), cos(4 pi / 5)
    const float s1 = 0.95105651629515357f, s2 = 0.58778525229247313f;    // sin(2 pi / 5), sin(4 pi / 5)
    const float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    const float2 d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
    const float2 a1 = make_float2(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
    const float2 a2 = make_float2(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
    const float2 b1 = mul_si<S>(make_float2(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y));
    const float2 b2 = mul_si<S>(make_float2(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y));
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = cadd(a1, b1);
    v[4] = csub(a1, b1);
    v[2] = cadd(a2, b2);
    v[3] = csub(a2, b2);
}

template <int R, int S>
__device__ __forceinline__ void dft(float2 *v);

// Composite length A B (Cooley-Tukey in registers): with n = B n1 + n2 and
// k = k1 + A k2, a DFT of length A over n1 for every n2, the twiddle
// exp(S 2 pi i n2 k1 / (A B)), then a DFT of length B over n2 for every k1.
// w[n2 * A + k1] holds that twiddle (cos, sin of 2 pi n2 k1 / (A B)).
template <int A, int B, int S>
__device__ __forceinline__ void dft_ct(float2 *v, const float (*w)[2])
{
    float2 u[B][A];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) {
#pragma unroll
        for (int n1 = 0; n1 < A; ++n1) u[n2][n1] = v[B * n1 + n2];
        dft<A, S>(u[n2]);
#pragma unroll
        for (int k1 = 1; k1 < A; ++k1)
            if (n2 > 0) u[n2][k1] = cmul(u[n2][k1], make_float2(w[n2 * A + k1][0], S * w[n2 * A + k1][1]));
    }
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
        float2 c[B];
#pragma unroll
        for (int n2 = 0; n2 < B; ++n2) c[n2] = u[n2][k1];
        dft<B, S>(c);
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = c[k2];
    }
}

template <int R, int S>
__device__ __forceinline__ void dft(float2 *v)
{
    if constexpr (R == 2) dft2<S>(v[0], v[1]);
    else if constexpr (R == 3) dft3<S>(v[0], v[1], v[2]);
    else if constexpr (R == 4) dft4<S>(v[0], v[1], v[2], v[3]);
    else if constexpr (R == 5) dft5<S>(v);
    else if constexpr (R == 6) {
        // A = 2, B = 3: twiddles 2 pi n2 / 6 for k1 = 1
        const float w[6][2] = {{1.f, 0.f}, {1.f, 0.f}, {1.f, 0.f}, {0.5f, 0.86602540378443865f},
                               {1.f, 0.f}, {-0.5f, 0.86602540378443865f}};
        dft_ct<2, 3, S>(v, w);
    } else if constexpr (R == 8) dft8<S>(v);
    else if constexpr (R == 9) {
        // A = 3, B = 3: twiddles 2 pi n2 k1 / 9
        const float c40 = 0.76604444311897804f, s40 = 0.64278760968653933f;
        const float c80 = 0.17364817766693035f, s80 = 0.98480775301220806f;
        const float c160 = -0.93969262078590838f, s160 = 0.34202014332566873f;
        const float w[9][2] = {{1.f, 0.f}, {1.f, 0.f}, {1.f, 0.f},
                               {1.f, 0.f}, {c40, s40}, {c80, s80},
                               {1.f, 0.f}, {c80, s80}, {c160, s160}};
        dft_ct<3, 3, S>(v, w);
    }
    else if constexpr (R == 10) {
        // A = 2, B = 5: twiddles 2 pi n2 / 10 for k1 = 1
        const float w[10][2] = {{1.f, 0.f}, {1.f, 0.f},
                                {1.f, 0.f}, {0.80901699437494742f, 0.58778525229247313f},
                                {1.f, 0.f}, {0.30901699437494742f, 0.95105651629515357f},
                                {1.f, 0.f}, {-0.30901699437494742f, 0.95105651629515357f},
                                {1.f, 0.f}, {-0.80901699437494742f, 0.58778525229247313f}};
        dft_ct<2, 5, S>(v, w);
    } else if constexpr (R == 12) {
        // A = 4, B = 3: twiddles 2 pi n2 k1 / 12
        const float c30 = 0.86602540378443865f;
        const float w[12][2] = {{1.f, 0.f}, {1.f, 0.f}, {1.f, 0.f}, {1.f, 0.f},
                                {1.f, 0.f}, {c30, 0.5f}, {0.5f, c30}, {0.f, 1.f},
                                {1.f, 0.f}, {0.5f, c30}, {-0.5f, c30}, {-1.f, 0.f}};
        dft_ct<4, 3, S>(v, w);
    } else dft16<S>(v);
}

// Per-slice geometry of the transforms, shared by all threads of the CTA.
struct FftGeom {
    int pu, pv, hu;          // padded sizes, hu = pu / 2
    int pitch;               // complex elements per S row (hu + 1)
    int n_rows_in;           // input rows (rows 0..n_rows_in-1 of S)
    int out_row0, n_rows_out;// output rows: S rows (out_row0 + t) % pv
};

// Division by a small positive divisor d (< 2^16) of x < 2^16 by a multiply
// high: with m = ceil(2^32 / d), floor(x m / 2^32) = floor(x / d) because the
// error term x (m - 2^32 / d) / 2^32 < 2^-16 < 1 / d cannot reach the next
// integer.  The multipliers of d <= kFdivMax (every divisor of the
// transforms: lengths, counts and strides of at most 97) come from a
// constant table, so a divisor costs one broadcast load instead of a
// division per thread.
struct FastDiv {
    unsigned m;
    int d;
};
constexpr int kFdivMax = 255;
__constant__ unsigned g_fft_mh[kFdivMax + 1];   // m(d) = floor((2^32 - 1) / d) + 1, m(0) = m(1) = 0
__host__ __device__ inline unsigned fast_div_mult(int d)
{
    return d > 1 ? (unsigned)(0xFFFFFFFFull / (unsigned)d) + 1u : 0u;
}
__device__ __forceinline__ FastDiv fast_div(int d)
{
    FastDiv f;
    f.d = d;
    f.m = d <= kFdivMax ? g_fft_mh[d] : fast_div_mult(d);
    return f;
}
__device__ __forceinline__ int operator/(int x, const FastDiv &f)
{
    return f.d == 1 ? x : (int)__umulhi((unsigned)x, f.m);
}

// v[q] *= w^q for q = 1 .. R-1, the powers by a balanced product tree
// (w^q = w^h w^(q-h), h the largest power of two below q; w^(2h) = (w^h)^2):
// depth log2 R instead of the R - 2 steps of a recurrence, so the
// butterfly's critical path is short and the rounding error grows with the
// depth (<= 4 products) only
template <int R>
__device__ __forceinline__ void twiddle_powers(float2 *v, float2 w)
{
    float2 p[R];
    p[1] = w;
#pragma unroll
    for (int q = 2; q < R; ++q) {
        int h = 1;
        while (2 * h < q) h *= 2;
        p[q] = (2 * h == q) ? cmul(p[h], p[h]) : cmul(p[h], p[q - h]);
    }
#pragma unroll
    for (int q = 1; q < R; ++q) v[q] = cmul(v[q], p[q]);
}

// One radix-R pass over a batch of transforms.
//   COLS = false: transforms are S rows row(t) = (row0 + t) % pv, t < n_tr,
//                 length hu, elements contiguous;
//   COLS = true : transforms are the hu + 1 columns, length pv, stride pitch.
//   INV  = false: decimation in frequency (DFT then twiddle W_L^{jq});
//   INV  = true : decimation in time (conjugate twiddle W_L^{-jm}, then DFT).
// L is the pass's block size and nl = N / L; the twiddle W_L^e =
// T[e nl tmul] with T the table of exp(-2 pi i t / (N tmul)).  MUL (first
// inverse column pass): every element read is first multiplied by the
// kernel spectrum.
// Output of the last inverse row pass, written straight to the region: real
// sample n of row tr is output u = in_i0 + n (or n - pu) of output row tr.
struct OutCtx {
    float *dst;
    int out_w, in_i0, out_i0, out_i1, pu;
};

template <int R, bool COLS, bool INV, bool MUL, bool OUT = false>
__device__ __forceinline__ void fft_pass(float2 *__restrict__ S, const FftGeom &G, int n_tr, int row0, int N,
                                         int L, int nl, const float2 *__restrict__ T, int tmul,
                                         const float *__restrict__ Kf, const short *__restrict__ kv_of,
                                         const short *__restrict__ ku_of, int valid = 1 << 30,
                                         const OutCtx *oc = nullptr)
{
    const int M = L / R;
    const int per_tr = N / R;
    const int total = n_tr * per_tr;
    const int tstep = nl * tmul;
    const FastDiv div_tr = fast_div(COLS ? n_tr : per_tr), div_m = fast_div(M);
    for (int b = threadIdx.x; b < total; b += kFftThreads) {
        const int q0 = b / div_tr;
        int tr, t;
        if (COLS) {
            t = q0;
            tr = b - q0 * n_tr;
        } else {
            tr = q0;
            t = b - q0 * per_tr;
        }
        const int blk = t / div_m, j = t - blk * M;
        const int e0 = blk * L + j;
        float2 *base;
        int es;
        if (COLS) {
            base = S + tr;
            es = G.pitch;
        } else {
            int row = row0 + tr;
            if (row >= G.pv) row -= G.pv;
            base = S + row * G.pitch;
            es = 1;
        }
        float2 v[R];
#pragma unroll
        for (int m = 0; m < R; ++m)
            v[m] = (e0 + m * M < valid) ? base[(e0 + m * M) * es] : make_float2(0.f, 0.f);
        if (MUL) {
            const int ku = __ldg(ku_of + tr);
#pragma unroll
            for (int m = 0; m < R; ++m) v[m] = cscale(v[m], Kf[__ldg(kv_of + e0 + m * M) * G.pitch + ku]);
        }
        // twiddles W_L^{j q}, q = 1..R-1, from one table read
        if (INV) {
            if (j) twiddle_powers<R>(v, cconj(__ldg(T + j * tstep)));
            dft<R, 1>(v);
        } else {
            dft<R, -1>(v);
            if (j) twiddle_powers<R>(v, __ldg(T + j * tstep));
        }
        if (OUT) {
            // natural order: complex element e0 + q M holds reals 2 (e0 + q M) and + 1
            float *drow = oc->dst + (long long)tr * oc->out_w;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                int u = oc->in_i0 + 2 * (e0 + q * M);
                if (u >= oc->out_i1) u -= oc->pu;
                if (u >= oc->out_i0 && u < oc->out_i1) drow[u - oc->out_i0] = v[q].x;
                int u1 = oc->in_i0 + 2 * (e0 + q * M) + 1;
                if (u1 >= oc->out_i1) u1 -= oc->pu;
                if (u1 >= oc->out_i0 && u1 < oc->out_i1) drow[u1 - oc->out_i0] = v[q].y;
            }
        } else {
#pragma unroll
            for (int m = 0; m < R; ++m) base[(e0 + m * M) * es] = v[m];
        }
    }
}

template <bool COLS, bool INV, bool MUL, bool OUT = false>
__device__ __forceinline__ void fft_pass_r(int R, float2 *S, const FftGeom &G, int n_tr, int row0, int N, int L,
                                           int nl, const float2 *T, int tmul, const float *Kf, const short *kv_of,
                                           const short *ku_of, int valid = 1 << 30, const OutCtx *oc = nullptr)
{
#define PDRT_FFT_PASS(RR) \
    fft_pass<RR, COLS, INV, MUL, OUT>(S, G, n_tr, row0, N, L, nl, T, tmul, Kf, kv_of, ku_of, valid, oc)
    switch (R) {
    case 3: PDRT_FFT_PASS(3); break;
    case 4: PDRT_FFT_PASS(4); break;
    case 5: PDRT_FFT_PASS(5); break;
    case 6: PDRT_FFT_PASS(6); break;
    case 8: PDRT_FFT_PASS(8); break;
    case 9: PDRT_FFT_PASS(9); break;
    case 10: PDRT_FFT_PASS(10); break;
    case 12: PDRT_FFT_PASS(12); break;
    default: PDRT_FFT_PASS(16); break;
    }
#undef PDRT_FFT_PASS
}

// Whole transform of length N over a batch: forward (DIF, natural in,
// digit-reversed out; rows at or past `valid` of a column read as zero in the
// first pass) or inverse (DIT, digit-reversed in, natural out; the first
// inverse column pass applies the kernel spectrum; with an output context the
// last inverse row pass writes the output box instead of S).
template <bool COLS, bool INV>
__device__ void fft_run(float2 *S, const FftGeom &G, int n_tr, int row0, int N, const float2 *T, int tmul,
                        const float *Kf, const short *kv_of, const short *ku_of, int valid = 1 << 30,
                        const OutCtx *oc = nullptr)
{
    const Radices rd = radices_of(N);
    const int r0 = rd.r[0], L1 = N / r0;
    if (!INV) {
        fft_pass_r<COLS, false, false>(r0, S, G, n_tr, row0, N, N, 1, T, tmul, Kf, kv_of, ku_of, valid);
        __syncthreads();
        if (rd.np > 1) {
            fft_pass_r<COLS, false, false>(rd.r[1], S, G, n_tr, row0, N, L1, r0, T, tmul, Kf, kv_of, ku_of);
            __syncthreads();
        }
    } else {
        if (rd.np > 1) {
            fft_pass_r<COLS, true, COLS>(rd.r[1], S, G, n_tr, row0, N, L1, r0, T, tmul, Kf, kv_of, ku_of);
            __syncthreads();
        }
        if (!COLS && oc) {
            fft_pass_r<false, true, false, true>(r0, S, G, n_tr, row0, N, N, 1, T, tmul, Kf, kv_of, ku_of, 1 << 30,
                                                 oc);
        } else if (rd.np > 1) {
            fft_pass_r<COLS, true, false>(r0, S, G, n_tr, row0, N, N, 1, T, tmul, Kf, kv_of, ku_of);
        } else {
            fft_pass_r<COLS, true, COLS>(r0, S, G, n_tr, row0, N, N, 1, T, tmul, Kf, kv_of, ku_of);
        }
        __syncthreads();
    }
}

// position of frequency k in the forward (DIF) output of length N, and the
// frequency held at position p
__host__ __device__ inline int dif_pos(int k, int N)
{
    const Radices rd = radices_of(N);
    int p = 0, L = N;
    for (int s = 0; s < rd.np; ++s) {
        const int q = k % rd.r[s];
        k /= rd.r[s];
        L /= rd.r[s];
        p += q * L;
    }
    return p;
}

__host__ __device__ inline int dif_freq(int p, int N)
{
    const Radices rd = radices_of(N);
    int k = 0, L = N, mul = 1;
    for (int s = 0; s < rd.np; ++s) {
        L /= rd.r[s];
        const int q = p / L;
        p -= q * L;
        k += q * mul;
        mul *= rd.r[s];
    }
    return k;
}

// Tables of every supported padded size P, laid out one size after another:
//   twiddles exp(-2 pi i t / P), t < P                          (sum P entries)
//   pos: position of frequency k in the DIF of length P/2, k < P/2
//   ku : frequency held at position c of that DIF (c < P/2), P/2 at c = P/2
//   kv : min(f, P - f), f the frequency at position e of the DIF of length P
// Constant, uploaded once per device (computed on the host in double).
constexpr int kSizes[kNumFftSizes] = {32, 40, 48, 60, 64, 72, 80, 90, 96, 100, 108, 120, 128, 144, 160, 192};
constexpr int kTwTotal = 1534, kPosTotal = 767, kKuTotal = 783, kKvTotal = 1534;
__device__ float2 g_fft_tw[kTwTotal];
__device__ short g_fft_pos[kPosTotal];
__device__ short g_fft_ku[kKuTotal];
__device__ short g_fft_kv[kKvTotal];

struct SizeOff {
    int tw, pos, ku, kv, cos;
};

// offsets of size P in the tables; cos: offset in the plan's cosine table
// (rows of (P/2 + 1) rounded up to 4 floats, R + 1 rows per size)
__host__ __device__ inline SizeOff size_offsets(int P, int R)
{
    const int sizes[kNumFftSizes] = {32, 40, 48, 60, 64, 72, 80, 90, 96, 100, 108, 120, 128, 144, 160, 192};
    SizeOff o = {0, 0, 0, 0, 0};
    for (int i = 0; i < kNumFftSizes && sizes[i] < P; ++i) {
        const int q = sizes[i];
        o.tw += q;
        o.pos += q / 2;
        o.ku += q / 2 + 1;
        o.kv += q;
        o.cos += (R + 1) * (((q / 2 + 1) + 3) & ~3);
    }
    return o;
}

}  // namespace

int conv_fft_cos_floats(int R) { return size_offsets(1 << 20, R).cos; }

// c_p cos(2 pi k p / P) for p <= R and k <= P/2 (0 in the row padding), c_0 = 1,
// c_{p>0} = 2, every supported P: the cosine sums of the kernel spectrum
void conv_fft_cos_table(int R, float *out)
{
    for (int i = 0; i < kNumFftSizes; ++i) {
        const int P = kSizes[i], w4 = ((P / 2 + 1) + 3) & ~3;
        float *t = out + size_offsets(P, R).cos;
        for (int pp = 0; pp <= R; ++pp)
            for (int k = 0; k < w4; ++k) {
                const long long e = ((long long)k * pp) % P;
                t[pp * w4 + k] = k <= P / 2 ? (float)((pp ? 2.0 : 1.0) * cos(2.0 * M_PI * (double)e / P)) : 0.f;
            }
    }
}

// uploads the size tables to the current device (once per device)
cudaError_t conv_fft_tables_upload()
{
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    std::vector<float2> tw(kTwTotal);
    std::vector<short> pos(kPosTotal), ku(kKuTotal), kv(kKvTotal);
    for (int i = 0; i < kNumFftSizes; ++i) {
        const int P = kSizes[i], H = P / 2;
        const SizeOff o = size_offsets(P, 0);
        for (int t = 0; t < P; ++t)
            tw[o.tw + t] = make_float2((float)cos(2.0 * M_PI * t / P), (float)-sin(2.0 * M_PI * t / P));
        for (int k = 0; k < H; ++k) pos[o.pos + k] = (short)dif_pos(k, H);
        for (int c = 0; c <= H; ++c) ku[o.ku + c] = (short)(c == H ? H : dif_freq(c, H));
        for (int q = 0; q < P; ++q) {
            const int f = dif_freq(q, P);
            kv[o.kv + q] = (short)std::min(f, P - f);
        }
    }
    if ((e = cudaMemcpyToSymbol(g_fft_tw, tw.data(), sizeof(float2) * kTwTotal)) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(g_fft_pos, pos.data(), sizeof(short) * kPosTotal)) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(g_fft_ku, ku.data(), sizeof(short) * kKuTotal)) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(g_fft_kv, kv.data(), sizeof(short) * kKvTotal)) != cudaSuccess) return e;
    unsigned mh[kFdivMax + 1];
    for (int d = 0; d <= kFdivMax; ++d) mh[d] = fast_div_mult(d);
    if ((e = cudaMemcpyToSymbol(g_fft_mh, mh, sizeof(mh))) != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) done[dev] = true;
    return cudaSuccess;
}

// shared memory of k_conv_fft for a size limit pmax and kernel half-width R:
// header, kernel spectrum, forward fill tables and the complex work array
// (which first holds the spectrum's scratch K [R+1][R+1] and A [R+1][P/2+1])
int conv_fft_smem_bytes(int pmax, int R)
{
    const int hu = pmax / 2, r1 = R + 1, w4 = ((hu + 1) + 3) & ~3;
    const int kf = (pmax / 2 + 1) * (hu + 1) * 4;               // Kf [kv'][ku]
    const int ft = 4 * pmax * 8;                                // forward fill tables
    const int scratch = (r1 * ((r1 + 3) & ~3) + ((r1 + 3) & ~3) * w4) * 4;
    const int s = std::max(pmax * (hu + 1) * 8, scratch);       // S [pv][hu + 1] complex
    auto al = [](int x) { return (x + 15) & ~15; };
    return 64 + al(kf) + ft + al(s);
}

// MINB: resident CTAs per SM the register budget is sized for (launch
// bounds); the launcher picks the instantiation that matches what the size
// limit's shared memory allows (fewer resident CTAs leave more registers).
// Shared-memory carve-up of k_conv_fft for a size limit pmax: the kernel
// spectrum, the forward fill tables and the complex work array (which also
// holds the spectrum's scratch before the fill).
struct FftSmem {
    float *Kf;
    int2 *fu_idx;
    float2 *fu_w;
    int2 *fv_idx;
    float2 *fv_w;
    float2 *S;
};

__device__ __forceinline__ FftSmem fft_smem(unsigned char *smem, int pmax)
{
    auto al = [](int x) { return (x + 15) & ~15; };
    const int hmax = pmax / 2;
    FftSmem m;
    unsigned char *p = smem + 64;
    m.Kf = reinterpret_cast<float *>(p);
    p += al((pmax / 2 + 1) * (hmax + 1) * 4);
    m.fu_idx = reinterpret_cast<int2 *>(p);
    m.fu_w = reinterpret_cast<float2 *>(m.fu_idx + pmax);
    m.fv_idx = reinterpret_cast<int2 *>(m.fu_w + pmax);
    m.fv_w = reinterpret_cast<float2 *>(m.fv_idx + pmax);
    p += 4 * pmax * 8;
    m.S = reinterpret_cast<float2 *>(p);
    return m;
}

// Kernel spectrum of one slice into Kf[kv'][ku] (kv' < pv/2 + 1, ku <= pu/2,
// rows of pitch floats; shared or global memory) by the NT threads of the
// CTA: K(p, q) (the expressions of the other convolution kernels), A = K Cv,
// Kf = scale / (pu pv) Cu^T A.  KT and A are shared scratch ([R1][R1p] and
// [R1][nkv4] floats).  Starts between barriers; ends after the Kf stores,
// before the barrier that must follow them.
template <int NT, class PL>
__device__ __forceinline__ void slice_spectrum(const PL &P, const SliceTab &st, int R, int pu, int pv,
                                               float *__restrict__ KT, float *__restrict__ A,
                                               float *__restrict__ Kf, int pitch)
{
    const Lattice &L = P.lat;
    const int R1 = R + 1, R1p = (R1 + 3) & ~3, tid = threadIdx.x;
    const bool sym = L.du == L.dv;                   // K(p, q) = K(q, p)
    const int hu = pu / 2, nkv = pv / 2 + 1, nkv4 = (nkv + 3) & ~3, hu4 = (hu + 1 + 3) & ~3;
    const SizeOff ou = size_offsets(pu, R), ov = size_offsets(pv, R);
    const float *Cv = P.fft_cos + ov.cos;        // [q][kv'], c_q folded in
    const float *Cu = P.fft_cos + ou.cos;        // [p][ku], c_p folded in
    // Kernel spectrum: K(p, q) (the expressions of the other convolution
    // kernels), A = K Cv, Kf[kv'][ku] = scale / (pu pv) sum_p Cu[p][ku] A[p][kv'].
    // K is stored transposed, KT[q][p] (rows of R1p = R1 rounded up to 4),
    // so that both products read 4-wide vectors of each operand.
    for (int idx = tid; idx < R1 * R1; idx += NT) {
        const int pp = idx / R1, q = idx - pp * R1;
        if (sym && pp > q) continue;
        const float pu_mm = pp * L.du, qv = q * L.dv;
        const float r = sqrtf(pu_mm * pu_mm + qv * qv);
        const float kv = st.wn[0] * expf(-st.a[0] * r) + st.wn[1] * expf(-st.a[1] * r) +
                         st.wn[2] * expf(-st.a[2] * r);
        KT[q * R1p + pp] = kv;
        if (sym) KT[pp * R1p + q] = kv;
    }
    for (int idx = tid; idx < R1 * (R1p - R1); idx += NT) {   // zero padding columns
        const int q = idx / (R1p - R1);
        KT[q * R1p + R1 + (idx - q * (R1p - R1))] = 0.f;
    }
    __syncthreads();
    // A[4 p4 .. +3][4 g .. +3] per item
    {
        const int G4 = nkv4 / 4, P4 = R1p / 4;
        const FastDiv dg = fast_div(G4);
        for (int idx = tid; idx < P4 * G4; idx += NT) {
            const int p4 = idx / dg, g = idx - p4 * G4;
            float4 acc[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) acc[a] = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 *kt = reinterpret_cast<const float4 *>(KT) + p4;
            const float4 *cv = reinterpret_cast<const float4 *>(Cv) + g;
            for (int q = 0; q < R1; ++q) {
                const float4 kk = kt[q * P4];
                const float4 c = __ldg(cv + q * G4);
                const float k4[4] = {kk.x, kk.y, kk.z, kk.w};
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    acc[a].x = fmaf(k4[a], c.x, acc[a].x);
                    acc[a].y = fmaf(k4[a], c.y, acc[a].y);
                    acc[a].z = fmaf(k4[a], c.z, acc[a].z);
                    acc[a].w = fmaf(k4[a], c.w, acc[a].w);
                }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
                if (4 * p4 + a < R1) reinterpret_cast<float4 *>(A)[(4 * p4 + a) * G4 + g] = acc[a];
        }
    }
    __syncthreads();
    // Kf[4 i4 .. +3][4 g .. +3] per item
    {
        const float kscale = st.tdd * st.c2 / ((float)pu * (float)pv);
        const int U4 = hu4 / 4, V4 = nkv4 / 4;
        const FastDiv du4 = fast_div(U4);
        for (int idx = tid; idx < V4 * U4; idx += NT) {
            const int i4 = idx / du4, g = idx - i4 * U4;
            float4 acc[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) acc[a] = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 *av = reinterpret_cast<const float4 *>(A) + i4;
            const float4 *cu = reinterpret_cast<const float4 *>(Cu) + g;
            for (int pp = 0; pp < R1; ++pp) {
                const float4 aa = av[pp * V4];
                const float4 c = __ldg(cu + pp * U4);
                const float a4[4] = {aa.x, aa.y, aa.z, aa.w};
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    acc[a].x = fmaf(a4[a], c.x, acc[a].x);
                    acc[a].y = fmaf(a4[a], c.y, acc[a].y);
                    acc[a].z = fmaf(a4[a], c.z, acc[a].z);
                    acc[a].w = fmaf(a4[a], c.w, acc[a].w);
                }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int kv = 4 * i4 + a;
                if (kv >= nkv) continue;
                const float r4[4] = {acc[a].x, acc[a].y, acc[a].z, acc[a].w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (4 * g + e <= hu) Kf[kv * pitch + 4 * g + e] = r4[e] * kscale;
            }
        }
    }
}

// Convolution of one (control point, slice) item of the chunk starting at
// control point b0, by the whole CTA; a slice beyond the size limit pmax is
// appended to the overflow list instead.  Every thread calls it with the
// same arguments; it starts and ends between barriers.
template <bool ADJ, class PL>
__device__ __forceinline__ void fft_slice(const PL &P, int R, int b0, int nb, int item, int pmax,
                                          int *__restrict__ over_list, unsigned int *__restrict__ over_count,
                                          const FftSmem &sm)
{
    const Lattice &L = P.lat;
    const int R1 = R + 1;
    float *Kf = sm.Kf;
    int2 *fu_idx = sm.fu_idx;
    float2 *fu_w = sm.fu_w;
    int2 *fv_idx = sm.fv_idx;
    float2 *fv_w = sm.fv_w;
    float2 *S = sm.S;
    const int R1p = (R1 + 3) & ~3;
    float *KT = reinterpret_cast<float *>(S);        // spectrum scratch before the fill: [q][p]
    float *A = KT + R1 * R1p;                        // [p][kv'] (16-byte aligned rows)
    const int tid = threadIdx.x;
    // items in slice-major order: the CTAs in flight work on neighbouring
    // depths of every control point, whose padded sizes mostly agree
    const int k = item / nb, bl = item - k * nb, b = b0 + bl;
    const SliceTab st = P.slices[(long long)b * L.nw + k];
    int pu, pv;
    fft_slice_sizes(st, ADJ, R, pu, pv);
    if (pu == 0) return;                     // no work in this slice
    if (pu > pmax || pv > pmax) {              // too large: the tensor-core kernel takes it
        if (tid == 0) over_list[atomicAdd(over_count, 1u)] = bl * L.nw + k;   // control-point-major
        return;
    }
    const TcBoxes bx = tc_boxes(st, ADJ, R);
    const int hu = pu / 2;
    FftGeom G;
    G.pu = pu; G.pv = pv; G.hu = hu; G.pitch = hu + 1;
    G.n_rows_in = bx.in_j1 - bx.in_j0;
    G.n_rows_out = bx.out_j1 - bx.out_j0;
    G.out_row0 = ((bx.out_j0 - bx.in_j0) % pv + pv) % pv;
    const int wi = bx.in_i1 - bx.in_i0;
    const SizeOff ou = size_offsets(pu, R), ov = size_offsets(pv, R);
    const float2 *Tu = g_fft_tw + ou.tw, *Tv = g_fft_tw + ov.tw;
    const short *pos_u = g_fft_pos + ou.pos, *ku_of = g_fft_ku + ou.ku, *kv_of = g_fft_kv + ov.kv;
    const int nkv = pv / 2 + 1;
    // memoised spectrum of this slice: it depends on the slice's depth,
    // kernel and magnification (fixed by the plan) and on (pu, pv) only, so
    // an entry tagged with the same sizes holds exactly what slice_spectrum
    // would compute (every thread reads the same tag: no CTA of this launch
    // writes it)
    const long long ce = (long long)b * L.nw + k;
    const bool memo = P.kf_memo != nullptr && pu <= P.kf_pmax && pv <= P.kf_pmax;
    const int ktag = (pu << 16) | pv;
    const bool hit = memo && P.kf_tag[ce] == ktag;
    const int nkf4 = (nkv * G.pitch + 3) >> 2;   // Kf as float4 (the rows are contiguous)
    float4 *memo4 = memo ? reinterpret_cast<float4 *>(P.kf_memo + ce * P.kf_stride) : nullptr;

    if (!hit) {
        slice_spectrum<kFftThreads>(P, st, R, pu, pv, KT, A, Kf, G.pitch);
    } else {
        for (int t = tid; t < nkf4; t += kFftThreads) reinterpret_cast<float4 *>(Kf)[t] = __ldg(memo4 + t);
    }
    // fill tables (forward): per input column n the two fluence rows a of
    // its bilinear stencil (clamped into the support box) with their
    // weights (zero outside the box), likewise per input row j
    if (!ADJ) {
        const CpTab &ct = P.cptab[b];
        for (int t = tid; t < wi + G.n_rows_in; t += kFftThreads) {
            const bool col = t < wi;
            const int lo = col ? ct.fa0 : ct.fc0, hi = col ? ct.fa1 : ct.fc1;
            const int idx0 = col ? bx.in_i0 + t : bx.in_j0 + (t - wi);
            const float f = col ? mag_coord(st.m, idx0, L.cu) : mag_coord(st.m, idx0, L.cv);
            const float fl = floorf(f);
            const int a0 = (int)fl;
            const float tw = f - fl;
            const bool ok0 = a0 >= lo && a0 < hi, ok1 = a0 + 1 >= lo && a0 + 1 < hi;
            const int i0 = min(max(a0 - lo, 0), hi - lo - 1), i1 = min(max(a0 + 1 - lo, 0), hi - lo - 1);
            const float w0 = ok0 ? 1.f - tw : 0.f, w1 = ok1 ? tw : 0.f;
            if (col) {
                fu_idx[t] = make_int2(i0, i1);
                fu_w[t] = make_float2(w0, w1);
            } else {
                fv_idx[t - wi] = make_int2(i0, i1);
                fv_w[t - wi] = make_float2(w0, w1);
            }
        }
    }
    __syncthreads();

    // fill the input rows (j = v offset from the input box), packed
    // (x[2m], x[2m+1]) along u; the rows past them are never written: the
    // first column pass reads them as zero
    {
        const int n_fill = G.n_rows_in * hu;
        const FastDiv dh = fast_div(hu);
        const float *fmap = P.fbuf + (long long)b * L.nu * L.nv;
        const int Fc = P.cptab[b].fc1 - P.cptab[b].fc0;
        const float *hsrc = P.region + (long long)bl * P.cap_o + st.off_o;
        const int h_w = st.oi1 - st.oi0;
        for (int idx = tid; idx < n_fill; idx += kFftThreads) {
            const int j = idx / dh, m = idx - j * hu;
            float x[2] = {0.f, 0.f};
            int2 ci = make_int2(0, 0);
            float2 cw = make_float2(0.f, 0.f);
            if (!ADJ) {
                ci = fv_idx[j];
                cw = fv_w[j];
            }
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int n = 2 * m + e;
                if (n >= wi) continue;
                if (ADJ) {
                    x[e] = hsrc[(long long)(bx.in_j0 + j - st.oj0) * h_w + (bx.in_i0 + n - st.oi0)];
                } else {
                    const int2 ai = fu_idx[n];
                    const float2 aw = fu_w[n];
                    const float *r0 = fmap + (long long)ai.x * Fc, *r1 = fmap + (long long)ai.y * Fc;
                    x[e] = aw.x * (cw.x * __ldg(r0 + ci.x) + cw.y * __ldg(r0 + ci.y)) +
                           aw.y * (cw.x * __ldg(r1 + ci.x) + cw.y * __ldg(r1 + ci.y));
                }
            }
            S[j * G.pitch + m] = make_float2(x[0], x[1]);
        }
    }
    if (memo && !hit) {   // store the spectrum just computed
        for (int t = tid; t < nkf4; t += kFftThreads) memo4[t] = reinterpret_cast<const float4 *>(Kf)[t];
        if (tid == 0) P.kf_tag[ce] = ktag;
    }
    __syncthreads();
    // rows: complex FFT of length hu over the input rows
    fft_run<false, false>(S, G, G.n_rows_in, 0, hu, Tu, 2, Kf, kv_of, ku_of);
    // real-FFT split: X[k] = E_k + W^k O_k and X[hu - k] = conj(E_k - W^k O_k),
    // E_k = (Z_k + conj Z_{hu-k}) / 2, O_k = (Z_k - conj Z_{hu-k}) / (2i),
    // W = exp(-2 pi i / pu); X[hu] goes to column hu
    {
        const int half = hu / 2 + 1;
        const FastDiv dhf = fast_div(half);
        for (int idx = tid; idx < G.n_rows_in * half; idx += kFftThreads) {
            const int j = idx / dhf, kk = idx - j * half;
            float2 *row = S + j * G.pitch;
            if (kk == 0) {
                const int p0 = __ldg(pos_u);
                const float2 z = row[p0];
                row[p0] = make_float2(z.x + z.y, 0.f);
                row[hu] = make_float2(z.x - z.y, 0.f);
                continue;
            }
            const int pk = __ldg(pos_u + kk), pc = __ldg(pos_u + hu - kk);
            const float2 zk = row[pk], zc = cconj(row[pc]);
            const float2 E = cscale(cadd(zk, zc), 0.5f);
            const float2 d = cscale(csub(zk, zc), 0.5f);
            const float2 O = make_float2(d.y, -d.x);   // d / i
            const float2 WO = cmul(__ldg(Tu + kk), O);
            row[pk] = cadd(E, WO);
            if (pc != pk) row[pc] = cconj(csub(E, WO));
        }
    }
    __syncthreads();
    // columns: forward FFT of length pv (rows past the input read as
    // zero), then product and inverse
    fft_run<true, false>(S, G, hu + 1, 0, pv, Tv, 1, Kf, kv_of, ku_of, G.n_rows_in);
    fft_run<true, true>(S, G, hu + 1, 0, pv, Tv, 1, Kf, kv_of, ku_of);
    // inverse real FFT of the output rows: Z[k] = (X_k + conj X_{hu-k})
    // + i exp(2 pi i k / pu) (X_k - conj X_{hu-k}), stored at pos_u(k)
    {
        const int half = hu / 2 + 1;
        const FastDiv dhf = fast_div(half);
        for (int idx = tid; idx < G.n_rows_out * half; idx += kFftThreads) {
            const int rr = idx / dhf, kk = idx - rr * half;
            int row_i = G.out_row0 + rr;
            if (row_i >= pv) row_i -= pv;
            float2 *row = S + row_i * G.pitch;
            const int pk = __ldg(pos_u + kk);
            const int pc = kk == 0 ? hu : __ldg(pos_u + hu - kk);
            const float2 xk = row[pk];
            const float2 xc = cconj(row[pc]);
            const float2 sum = cadd(xk, xc), dif = csub(xk, xc);
            const float2 w = __ldg(Tu + kk);
            const float2 wd = cmul(cconj(w), dif);
            row[pk] = make_float2(sum.x - wd.y, sum.y + wd.x);   // sum + i wd
            if (kk > 0 && 2 * kk != hu) {
                // Z[hu - k] = (X_{hu-k} + conj X_k) - i exp(-2 pi i k / pu) (X_{hu-k} - conj X_k)
                const float2 yk = cconj(xc), yc = cconj(xk);   // X_{hu-k}, conj X_k
                const float2 s2 = cadd(yk, yc), d2 = csub(yk, yc);
                const float2 w2 = cmul(w, d2);
                row[pc] = make_float2(s2.x + w2.y, s2.y - w2.x);   // s2 - i w2
            }
        }
    }
    __syncthreads();
    // inverse rows; the last pass writes the output box:
    // (u, v) holds real sample (u - in_i0) mod pu of row (v - in_j0) mod pv
    OutCtx oc;
    oc.dst = ADJ ? P.adjbuf + (long long)bl * P.cap_a + st.off_a
                 : P.region + (long long)bl * P.cap_o + st.off_o;
    oc.out_w = bx.out_i1 - bx.out_i0;
    oc.in_i0 = bx.in_i0;
    oc.out_i0 = bx.out_i0;
    oc.out_i1 = bx.out_i1;
    oc.pu = pu;
    fft_run<false, true>(S, G, G.n_rows_out, G.out_row0, hu, Tu, 2, Kf, kv_of, ku_of, 1 << 30, &oc);
}

template <bool ADJ, int MINB>
__global__ void __launch_bounds__(kFftThreads, MINB) k_conv_fft(PlanDev P, int b0, int nb, int pmax,
                                                            unsigned int *__restrict__ counter,
                                                            int *__restrict__ over_list,
                                                            unsigned int *__restrict__ over_count)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int *s_item = reinterpret_cast<int *>(smem);
    const FftSmem sm = fft_smem(smem, pmax);
    const int n_items = nb * P.lat.nw;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) *s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int item = *s_item;
        if (item >= n_items) break;
        fft_slice<ADJ>(P, P.mach.R, b0, nb, item, pmax, over_list, over_count, sm);
    }
}

// Batched form: one persistent launch over the items of several plans'
// passes.  Entry e is pass round[e].w (control points round[e].x ..
// + round[e].y) of plan plan[e]; its items follow those of the entries
// before it.  Each slice goes by its own plan's size limit and overflow list;
// the shared memory is laid out for the largest limit pmax.  The entries sit
// in the kernel parameters (grid constant), so an entry's fields are read
// through the constant cache as in k_conv_fft.
struct FftBatchArgs {
    FftPlan plan[kFftBatchMax];
    int4 round[kFftBatchMax];   // {b0, nb, first item, pass}
    int n_ent, n_items;
};
static_assert(sizeof(FftBatchArgs) + 2 * sizeof(void *) <= 32764, "kernel parameters above 32 KB");

template <bool ADJ, int MINB>
__global__ void __launch_bounds__(kFftThreads, MINB)
k_conv_fft_multi(const __grid_constant__ FftBatchArgs A, int pmax, unsigned int *__restrict__ counter)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int *s_item = reinterpret_cast<int *>(smem);
    const FftSmem sm = fft_smem(smem, pmax);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) *s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int item = *s_item;
        if (item >= A.n_items) break;
        int e = 0;
        while (e + 1 < A.n_ent && A.round[e + 1].z <= item) ++e;
        const FftPlan &P = A.plan[e];
        const int4 r = A.round[e];
        unsigned int *ctr = P.fft_ctr + 4 * r.w + (ADJ ? 2 : 0);
        fft_slice<ADJ>(P, P.R, r.x, r.y, item - r.z, P.fft_pmax, P.fft_over, ctr + 1, sm);
    }
}

// Spectra of one pass's slices into the kernel-spectrum memo, ahead of the
// FFT convolution (which then takes them from the memo): one CTA of
// kSpecThreads per (control point, slice) item; items without FFT work, with
// sizes beyond the memo or the size limit, or whose entry already holds
// their sizes, return at once.  The spectrum is the FFT kernel's own
// (slice_spectrum), so the memo holds the same bytes either way.
constexpr int kSpecThreads = 128;

__global__ void __launch_bounds__(kSpecThreads) k_spectrum(PlanDev P, int b0, int nb, int pmax, int adjoint)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Lattice &L = P.lat;
    const int bl = (int)blockIdx.x / L.nw, k = (int)blockIdx.x - bl * L.nw, b = b0 + bl;
    if (bl >= nb) return;
    const int R = P.mach.R;
    const SliceTab st = P.slices[(long long)b * L.nw + k];
    int pu, pv;
    fft_slice_sizes(st, adjoint != 0, R, pu, pv);
    if (pu == 0 || pu > pmax || pv > pmax || pu > P.kf_pmax || pv > P.kf_pmax) return;
    const long long ce = (long long)b * L.nw + k;
    const int ktag = (pu << 16) | pv;
    if (P.kf_tag[ce] == ktag) return;
    const int R1 = R + 1, R1p = (R1 + 3) & ~3;
    float *KT = reinterpret_cast<float *>(smem);
    float *A = KT + R1 * R1p;
    slice_spectrum<kSpecThreads>(P, st, R, pu, pv, KT, A, P.kf_memo + ce * P.kf_stride, pu / 2 + 1);
    if (threadIdx.x == 0) P.kf_tag[ce] = ktag;
}

cudaError_t launch_spectrum(const PlanDev &P, int b0, int nb, bool adjoint, int pmax, cudaStream_t s)
{
    if (!P.kf_memo || !pmax || nb < 1) return cudaSuccess;
    const int R1 = P.mach.R + 1, R1p = (R1 + 3) & ~3, w4 = ((P.kf_pmax / 2 + 1) + 3) & ~3;
    const int smem = (R1 * R1p + R1 * w4) * (int)sizeof(float);
    k_spectrum<<<(unsigned)(nb * P.lat.nw), kSpecThreads, smem, s>>>(P, b0, nb, pmax, adjoint ? 1 : 0);
    internal_count_launch();
    return cudaGetLastError();
}

namespace {

// resident CTAs per SM that the shared memory of a size limit allows
int fft_ctas_by_smem(int pmax, int R, int smem_sm, int resv)
{
    return smem_sm / (conv_fft_smem_bytes(pmax, R) + resv);
}

template <bool ADJ>
const void *fft_kernel_for(int minb)
{
    if (minb >= 4) return (const void *)k_conv_fft<ADJ, 4>;
    if (minb == 3) return (const void *)k_conv_fft<ADJ, 3>;
    return (const void *)k_conv_fft<ADJ, 2>;
}

template <bool ADJ>
const void *fft_multi_kernel_for(int minb)
{
    if (minb >= 4) return (const void *)k_conv_fft_multi<ADJ, 4>;
    if (minb == 3) return (const void *)k_conv_fft_multi<ADJ, 3>;
    return (const void *)k_conv_fft_multi<ADJ, 2>;
}

struct SmemLimits {
    int smem_sm, resv, regs_sm, optin;
};

cudaError_t smem_limits(SmemLimits &l)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l.smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l.resv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l.regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l.optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return e;
}

}  // namespace

cudaError_t launch_conv_fft(const PlanDev &P, int b0, int nb, bool adjoint, int pmax, unsigned int *counter,
                            int *over_list, unsigned int *over_count, int grid_blocks, cudaStream_t s)
{
    const int smem = conv_fft_smem_bytes(pmax, P.mach.R);
    // the grid is (CTAs per SM) x SMs; the instantiation for that many CTAs
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int minb = grid_blocks / (sms > 0 ? sms : 1);
    const void *k = adjoint ? fft_kernel_for<true>(minb) : fft_kernel_for<false>(minb);
    void *args[] = {(void *)&P, (void *)&b0, (void *)&nb, (void *)&pmax, (void *)&counter, (void *)&over_list,
                    (void *)&over_count};
    return cudaLaunchKernel(k, dim3(grid_blocks), dim3(kFftThreads), args, smem, s);
}

cudaError_t launch_conv_fft_multi(const FftPlan *plans, const int4 *round, int n_ent, int pmax, int smem,
                                  int grid_blocks, bool adjoint, unsigned int *counters, cudaStream_t s)
{
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int minb = grid_blocks / (sms > 0 ? sms : 1);
    const void *k = adjoint ? fft_multi_kernel_for<true>(minb) : fft_multi_kernel_for<false>(minb);
    static thread_local FftBatchArgs A;   // 22 KB: not on the stack
    for (int g = 0; g * kFftBatchMax < n_ent; ++g) {
        const int e0 = g * kFftBatchMax, ne = std::min(kFftBatchMax, n_ent - e0);
        A.n_ent = ne;
        A.n_items = 0;
        for (int e = 0; e < ne; ++e) {
            A.plan[e] = plans[e0 + e];
            A.round[e] = make_int4(round[e0 + e].x, round[e0 + e].y, A.n_items, round[e0 + e].w);
            A.n_items += round[e0 + e].y * plans[e0 + e].lat.nw;
        }
        unsigned int *ctr = counters + g;
        void *args[] = {(void *)&A, (void *)&pmax, (void *)&ctr};
        const cudaError_t e = cudaLaunchKernel(k, dim3(grid_blocks), dim3(kFftThreads), args, smem, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// CTAs of one direction per SM at a size limit: the shared memory decides
// how many fit, the register-bound instantiation for that count (2, 3 or 4)
// must also fit; also uploads the size tables to the current device
cudaError_t conv_fft_ctas(int pmax, int R, bool adjoint, int *ctas)
{
    *ctas = 0;
    if (!fft_size_for(pmax) || fft_size_for(pmax) != pmax || pmax < 2 * R + 2) return cudaSuccess;
    cudaError_t e = conv_fft_tables_upload();
    if (e != cudaSuccess) return e;
    SmemLimits l;
    if ((e = smem_limits(l)) != cudaSuccess) return e;
    const int smem = conv_fft_smem_bytes(pmax, R);
    if (smem > l.optin) return cudaSuccess;
    const int want = std::min(4, fft_ctas_by_smem(pmax, R, l.smem_sm, l.resv));
    if (want < 1) return cudaSuccess;
    // every instantiation may be launched (the launchers pick by CTAs per SM)
    for (int q = 0; q < 6 && e == cudaSuccess; ++q) {
        const int mb = 2 + q % 3;
        const void *km = q < 3 ? (adjoint ? fft_kernel_for<true>(mb) : fft_kernel_for<false>(mb))
                               : (adjoint ? fft_multi_kernel_for<true>(mb) : fft_multi_kernel_for<false>(mb));
        cudaFuncAttributes fm;
        e = cudaFuncGetAttributes(&fm, km);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(km, cudaFuncAttributeMaxDynamicSharedMemorySize, l.optin - (int)fm.sharedSizeBytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(km, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
    }
    if (e != cudaSuccess) return e;
    const void *k = adjoint ? fft_kernel_for<true>(want) : fft_kernel_for<false>(want);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k);
    if (e != cudaSuccess) return e;
    const int by_smem = l.smem_sm / (smem + (int)fa.sharedSizeBytes + l.resv);
    const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
    const int by_regs = l.regs_sm / (regs_warp * (kFftThreads / 32));
    *ctas = std::max(1, std::min(want, std::min(by_smem, by_regs)));
    return cudaSuccess;
}

}  // namespace pdrt
