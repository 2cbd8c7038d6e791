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
// 8, 16) decimation in frequency forward, leaving the spectrum in
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

#include "pdrt_impl.cuh"

namespace pdrt {

namespace {

constexpr int kFftThreads = 256;

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
    case 32: return {2, {8, 4, 1}};
    case 40: return {2, {8, 5, 1}};
    case 48: return {2, {16, 3, 1}};
    case 60: return {2, {12, 5, 1}};
    case 64: return {2, {8, 8, 1}};
    case 80: return {2, {16, 5, 1}};
    case 96: return {2, {16, 6, 1}};
    case 120: return {2, {12, 10, 1}};
    case 128: return {2, {16, 8, 1}};
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
// integer.
struct FastDiv {
    unsigned m;
    int d;
};
__device__ __forceinline__ FastDiv fast_div(int d)
{
    FastDiv f;
    f.d = d;
    f.m = d > 1 ? (unsigned)(0xFFFFFFFFull / (unsigned)d) + 1u : 0u;
    return f;
}
__device__ __forceinline__ int operator/(int x, const FastDiv &f)
{
    return f.d == 1 ? x : (int)__umulhi((unsigned)x, f.m);
}

// One radix-R pass over a batch of transforms.
//   COLS = false: transforms are S rows row(t) = (row0 + t) % pv, t < n_tr,
//                 length hu, elements contiguous;
//   COLS = true : transforms are the hu + 1 columns, length pv, stride pitch.
//   INV  = false: decimation in frequency (DFT then twiddle W_L^{jq});
//   INV  = true : decimation in time (conjugate twiddle W_L^{-jm}, then DFT).
// L is the pass's block size; the twiddle W_L^e = T[e (N / L) tmul] with T
// the table of exp(-2 pi i t / (N tmul)).  MUL (first inverse column pass):
// every element read is first multiplied by the kernel spectrum.
template <int R, bool COLS, bool INV, bool MUL>
__device__ __forceinline__ void fft_pass(float2 *__restrict__ S, const FftGeom &G, int n_tr, int row0, int N,
                                         int L, const float2 *__restrict__ T, int tmul,
                                         const float *__restrict__ Kf, const short *__restrict__ kv_of,
                                         const short *__restrict__ ku_of)
{
    const int M = L / R;
    const int per_tr = N / R;
    const int total = n_tr * per_tr;
    const int tstep = (N / L) * tmul;
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
        for (int m = 0; m < R; ++m) v[m] = base[(e0 + m * M) * es];
        if (MUL) {
            const int ku = ku_of[tr];
#pragma unroll
            for (int m = 0; m < R; ++m) v[m] = cscale(v[m], Kf[kv_of[e0 + m * M] * G.pitch + ku]);
        }
        if (INV) {
#pragma unroll
            for (int m = 1; m < R; ++m) v[m] = cmul(v[m], cconj(T[j * m * tstep]));
            dft<R, 1>(v);
        } else {
            dft<R, -1>(v);
#pragma unroll
            for (int q = 1; q < R; ++q) v[q] = cmul(v[q], T[j * q * tstep]);
        }
#pragma unroll
        for (int m = 0; m < R; ++m) base[(e0 + m * M) * es] = v[m];
    }
}

template <bool COLS, bool INV, bool MUL>
__device__ __forceinline__ void fft_pass_r(int R, float2 *S, const FftGeom &G, int n_tr, int row0, int N, int L,
                                           const float2 *T, int tmul, const float *Kf, const short *kv_of,
                                           const short *ku_of)
{
    switch (R) {
    case 3: fft_pass<3, COLS, INV, MUL>(S, G, n_tr, row0, N, L, T, tmul, Kf, kv_of, ku_of); break;
    case 4: fft_pass<4, COLS, INV, MUL>(S, G, n_tr, row0, N, L, T, tmul, Kf, kv_of, ku_of); break;
    case 5: fft_pass<5, COLS, INV, MUL>(S, G, n_tr, row0, N, L, T, tmul, Kf, kv_of, ku_of); break;
    case 6: fft_pass<6, COLS, INV, MUL>(S, G, n_tr, row0, N, L, T, tmul, Kf, kv_of, ku_of); break;
    case 8: fft_pass<8, COLS, INV, MUL>(S, G, n_tr, row0, N, L, T, tmul, Kf, kv_of, ku_of); break;
    case 10: fft_pass<10, COLS, INV, MUL>(S, G, n_tr, row0, N, L, T, tmul, Kf, kv_of, ku_of); break;
    case 12: fft_pass<12, COLS, INV, MUL>(S, G, n_tr, row0, N, L, T, tmul, Kf, kv_of, ku_of); break;
    default: fft_pass<16, COLS, INV, MUL>(S, G, n_tr, row0, N, L, T, tmul, Kf, kv_of, ku_of); break;
    }
}

// Whole transform of length N over a batch: forward (DIF, natural in,
// digit-reversed out) or inverse (DIT, digit-reversed in, natural out; the
// first inverse column pass applies the kernel spectrum).
template <bool COLS, bool INV>
__device__ void fft_run(float2 *S, const FftGeom &G, int n_tr, int row0, int N, const float2 *T, int tmul,
                        const float *Kf, const short *kv_of, const short *ku_of)
{
    const Radices rd = radices_of(N);
    const int r0 = rd.r[0], L1 = N / r0;
    if (!INV) {
        fft_pass_r<COLS, false, false>(r0, S, G, n_tr, row0, N, N, T, tmul, Kf, kv_of, ku_of);
        __syncthreads();
        if (rd.np > 1) {
            fft_pass_r<COLS, false, false>(rd.r[1], S, G, n_tr, row0, N, L1, T, tmul, Kf, kv_of, ku_of);
            __syncthreads();
        }
    } else {
        if (rd.np > 1) {
            fft_pass_r<COLS, true, COLS>(rd.r[1], S, G, n_tr, row0, N, L1, T, tmul, Kf, kv_of, ku_of);
            __syncthreads();
            fft_pass_r<COLS, true, false>(r0, S, G, n_tr, row0, N, N, T, tmul, Kf, kv_of, ku_of);
        } else {
            fft_pass_r<COLS, true, COLS>(r0, S, G, n_tr, row0, N, N, T, tmul, Kf, kv_of, ku_of);
        }
        __syncthreads();
    }
}

// position of frequency k in the forward (DIF) output of length N, and the
// frequency held at position p
__device__ __forceinline__ int dif_pos(int k, int N)
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

__device__ __forceinline__ int dif_freq(int p, int N)
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

}  // namespace

// shared memory of k_conv_fft for a size limit pmax: header, twiddle tables,
// index tables, kernel spectrum and the complex work array
int conv_fft_smem_bytes(int pmax)
{
    const int hu = pmax / 2;
    const int tw = 2 * pmax * 8;                               // Tu, Tv
    const int idx = (3 * pmax + 8) * 2;                         // pos_u, ku_of, kv_of (short)
    const int kf = (pmax / 2 + 1) * (hu + 1) * 4;               // Kf [kv'][ku]
    const int ft = 4 * pmax * 8;                                // forward fill tables
    // S [pv][hu + 1] complex; it also holds the kernel-spectrum scratch
    // K, Cv, Cu, A for a kernel half-width up to pmax / 2 - 1
    const int r1 = hu, w4 = ((hu + 1) + 3) & ~3;
    const int scratch = (r1 * (r1 + 3 * w4) + 4) * 4;
    const int s = std::max(pmax * (hu + 1) * 8, scratch);
    auto al = [](int x) { return (x + 15) & ~15; };
    return 64 + al(tw) + al(idx) + al(kf) + ft + al(s);
}

template <bool ADJ>
__global__ void __launch_bounds__(kFftThreads, 3) k_conv_fft(PlanDev P, int b0, int nb, int pmax,
                                                            unsigned int *__restrict__ counter,
                                                            int *__restrict__ over_list,
                                                            unsigned int *__restrict__ over_count)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Lattice &L = P.lat;
    const int R = P.mach.R;
    const int hmax = pmax / 2;
    auto al = [](int x) { return (x + 15) & ~15; };
    int *s_item = reinterpret_cast<int *>(smem);
    int *s_sizes = reinterpret_cast<int *>(smem + 16);   // current table sizes (pu, pv)
    unsigned char *p = smem + 64;
    float2 *Tu = reinterpret_cast<float2 *>(p);
    float2 *Tv = Tu + pmax;
    p += al(2 * pmax * 8);
    short *pos_u = reinterpret_cast<short *>(p);
    short *ku_of = pos_u + hmax;
    short *kv_of = ku_of + hmax + 4;
    p += al((3 * pmax + 8) * 2);
    float *Kf = reinterpret_cast<float *>(p);
    p += al((pmax / 2 + 1) * (hmax + 1) * 4);
    int2 *fu_idx = reinterpret_cast<int2 *>(p);   // forward fill tables, [pmax] each
    float2 *fu_w = reinterpret_cast<float2 *>(fu_idx + pmax);
    int2 *fv_idx = reinterpret_cast<int2 *>(fu_w + pmax);
    float2 *fv_w = reinterpret_cast<float2 *>(fv_idx + pmax);
    p += 4 * pmax * 8;
    float2 *S = reinterpret_cast<float2 *>(p);
    float *scratch = reinterpret_cast<float *>(S);   // kernel rows and A before the fill
    const int tid = threadIdx.x;
    const int n_items = nb * L.nw;
    if (tid == 0) s_sizes[0] = s_sizes[1] = 0;

    for (;;) {
        __syncthreads();
        if (tid == 0) *s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int item = *s_item;
        if (item >= n_items) break;
        const int bl = item / L.nw, k = item - bl * L.nw, b = b0 + bl;
        const SliceTab st = P.slices[(long long)b * L.nw + k];
        int pu, pv;
        fft_slice_sizes(st, ADJ, R, pu, pv);
        if (pu == 0) continue;                     // no work in this slice
        if (pu > pmax || pv > pmax) {              // too large: the tensor-core kernel takes it
            if (tid == 0) over_list[atomicAdd(over_count, 1u)] = item;
            continue;
        }
        const TcBoxes bx = tc_boxes(st, ADJ, R);
        const int hu = pu / 2;
        FftGeom G;
        G.pu = pu; G.pv = pv; G.hu = hu; G.pitch = hu + 1;
        G.n_rows_in = bx.in_j1 - bx.in_j0;
        G.n_rows_out = bx.out_j1 - bx.out_j0;
        G.out_row0 = ((bx.out_j0 - bx.in_j0) % pv + pv) % pv;
        const int wi = bx.in_i1 - bx.in_i0;

        // twiddle and index tables when the sizes change (all threads read
        // s_sizes before any thread rewrites it: the barrier after the item)
        const bool new_sizes = (s_sizes[0] != pu || s_sizes[1] != pv);
        if (new_sizes) {
            for (int t = tid; t < pu + pv; t += kFftThreads) {
                const int n = t < pu ? pu : pv, e = t < pu ? t : t - pu;
                float sn, cs;
                sincospif(2.0f * (float)e / (float)n, &sn, &cs);
                (t < pu ? Tu : Tv)[e] = make_float2(cs, -sn);
            }
            for (int t = tid; t < hu + 1 + pv + hu; t += kFftThreads) {
                if (t < hu + 1) {
                    ku_of[t] = (short)(t == hu ? hu : dif_freq(t, hu));
                } else if (t < hu + 1 + pv) {
                    const int e = t - hu - 1, kv = dif_freq(e, pv);
                    kv_of[e] = (short)min(kv, pv - kv);
                } else {
                    const int e = t - hu - 1 - pv;
                    pos_u[e] = (short)dif_pos(e, hu);
                }
            }
        }
        // Kernel spectrum.  Scratch in S: K(p, q) [R1][R1]; cosine tables
        // Cv[q][kv'] = c_q cos(2 pi kv' q / pv) and Cu[p][ku] = c_p cos(2 pi ku p / pu)
        // (rows padded to multiples of 4); A = K Cv [R1][nkv4]; then
        // Kf[kv'][ku] = scale / (pu pv) sum_p Cu[p][ku] A[p][kv'].
        const int R1 = R + 1;
        const int nkv = pv / 2 + 1, nkv4 = (nkv + 3) & ~3, hu4 = (hu + 1 + 3) & ~3;
        float *Kq = scratch;                   // [p][q]
        float *Cv = Kq + ((R1 * R1 + 3) & ~3); // [q][kv'] (16-byte aligned rows)
        float *Cu = Cv + R1 * nkv4;            // [p][ku]
        float *A = Cu + R1 * hu4;              // [p][kv']
        for (int idx = tid; idx < R1 * R1; idx += kFftThreads) {
            const int pp = idx / R1, q = idx - pp * R1;
            const float pu_mm = pp * L.du, qv = q * L.dv;
            const float r = sqrtf(pu_mm * pu_mm + qv * qv);
            Kq[idx] = st.wn[0] * expf(-st.a[0] * r) + st.wn[1] * expf(-st.a[1] * r) +
                      st.wn[2] * expf(-st.a[2] * r);
        }
        __syncthreads();
        // every thread has read s_sizes (before the barrier above)
        if (tid == 0) {
            s_sizes[0] = pu;
            s_sizes[1] = pv;
        }
        {
            const FastDiv dv = fast_div(pv), du = fast_div(pu), d4v = fast_div(nkv4), d4u = fast_div(hu4);
            for (int idx = tid; idx < R1 * (nkv4 + hu4); idx += kFftThreads) {
                if (idx < R1 * nkv4) {
                    const int q = idx / d4v, kv = idx - q * nkv4;
                    const int e = kv * q - ((kv * q) / dv) * pv;
                    Cv[idx] = kv < nkv ? (q ? 2.f : 1.f) * Tv[e].x : 0.f;
                } else {
                    const int t = idx - R1 * nkv4;
                    const int pp = t / d4u, ku = t - pp * hu4;
                    const int e = ku * pp - ((ku * pp) / du) * pu;
                    Cu[t] = ku <= hu ? (pp ? 2.f : 1.f) * Tu[e].x : 0.f;
                }
            }
        }
        __syncthreads();
        // A[p][4g .. 4g+3] per item: K row p (broadcast) against float4 of Cv
        {
            const int G4 = nkv4 / 4;
            const FastDiv dg = fast_div(G4);
            for (int idx = tid; idx < R1 * G4; idx += kFftThreads) {
                const int pp = idx / dg, g = idx - pp * G4;
                float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                const float *kr = Kq + pp * R1;
                const float4 *cv = reinterpret_cast<const float4 *>(Cv) + g;
                for (int q = 0; q < R1; ++q) {
                    const float k = kr[q];
                    const float4 c = cv[q * G4];
                    acc.x = fmaf(k, c.x, acc.x);
                    acc.y = fmaf(k, c.y, acc.y);
                    acc.z = fmaf(k, c.z, acc.z);
                    acc.w = fmaf(k, c.w, acc.w);
                }
                reinterpret_cast<float4 *>(A)[pp * G4 + g] = acc;
            }
        }
        __syncthreads();
        // Kf for kv' in {2i, 2i+1} and ku in [4g, 4g+4) per item
        {
            const float kscale = st.tdd * st.c2 / ((float)pu * (float)pv);
            const int U4 = hu4 / 4, V2 = (nkv + 1) / 2;
            const FastDiv du4 = fast_div(U4);
            for (int idx = tid; idx < V2 * U4; idx += kFftThreads) {
                const int i = idx / du4, g = idx - i * U4;
                float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
                const float4 *cu = reinterpret_cast<const float4 *>(Cu) + g;
                for (int pp = 0; pp < R1; ++pp) {
                    const float2 av = *reinterpret_cast<const float2 *>(A + pp * nkv4 + 2 * i);
                    const float4 c = cu[pp * U4];
                    a0.x = fmaf(av.x, c.x, a0.x); a0.y = fmaf(av.x, c.y, a0.y);
                    a0.z = fmaf(av.x, c.z, a0.z); a0.w = fmaf(av.x, c.w, a0.w);
                    a1.x = fmaf(av.y, c.x, a1.x); a1.y = fmaf(av.y, c.y, a1.y);
                    a1.z = fmaf(av.y, c.z, a1.z); a1.w = fmaf(av.y, c.w, a1.w);
                }
                const float r0[4] = {a0.x, a0.y, a0.z, a0.w}, r1[4] = {a1.x, a1.y, a1.z, a1.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int ku = 4 * g + e;
                    if (ku > hu) continue;
                    Kf[(2 * i) * G.pitch + ku] = r0[e] * kscale;
                    if (2 * i + 1 < nkv) Kf[(2 * i + 1) * G.pitch + ku] = r1[e] * kscale;
                }
            }
        }
        // fill tables (forward): per input column n the two fluence rows a
        // of its bilinear stencil (clamped into the support box) with their
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

        // fill: row j = v offset from the input box, packed (x[2m], x[2m+1])
        // along u; rows past the input are zero
        {
            const int n_fill = pv * (hu + 1);
            const FastDiv dp = fast_div(hu + 1);
            const float *fmap = P.fbuf + (long long)b * L.nu * L.nv;
            const int Fc = P.cptab[b].fc1 - P.cptab[b].fc0;
            const float *hsrc = P.region + (long long)bl * P.cap_o + st.off_o;
            const int h_w = st.oi1 - st.oi0;
            for (int idx = tid; idx < n_fill; idx += kFftThreads) {
                const int j = idx / dp, m = idx - j * (hu + 1);
                float x[2] = {0.f, 0.f};
                if (j < G.n_rows_in && m < hu) {
                    int2 ci;
                    float2 cw;
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
                }
                S[idx] = make_float2(x[0], x[1]);
            }
        }
        __syncthreads();
        // rows: complex FFT of length hu over the input rows
        fft_run<false, false>(S, G, G.n_rows_in, 0, hu, Tu, 2, Kf, kv_of, ku_of);
        // real-FFT split: X[k] = E_k + W^k O_k and X[hu - k] = conj(E_k - W^k O_k),
        // E_k = (Z_k + conj Z_{hu-k}) / 2, O_k = (Z_k - conj Z_{hu-k}) / (2i),
        // W = exp(-2 pi i / pu); X[hu] goes to column hu
        {
            const int half = hu / 2 + 1;
            for (int idx = tid; idx < G.n_rows_in * half; idx += kFftThreads) {
                const int j = idx / half, kk = idx - j * half;
                float2 *row = S + j * G.pitch;
                if (kk == 0) {
                    const float2 z = row[pos_u[0]];
                    row[pos_u[0]] = make_float2(z.x + z.y, 0.f);
                    row[hu] = make_float2(z.x - z.y, 0.f);
                    continue;
                }
                const int pk = pos_u[kk], pc = pos_u[hu - kk];
                const float2 zk = row[pk], zc = cconj(row[pc]);
                const float2 E = cscale(cadd(zk, zc), 0.5f);
                const float2 d = cscale(csub(zk, zc), 0.5f);
                const float2 O = make_float2(d.y, -d.x);   // d / i
                const float2 WO = cmul(Tu[kk], O);
                row[pk] = cadd(E, WO);
                if (pc != pk) row[pc] = cconj(csub(E, WO));
            }
        }
        __syncthreads();
        // columns: forward FFT of length pv, then product and inverse
        fft_run<true, false>(S, G, hu + 1, 0, pv, Tv, 1, Kf, kv_of, ku_of);
        fft_run<true, true>(S, G, hu + 1, 0, pv, Tv, 1, Kf, kv_of, ku_of);
        // inverse real FFT of the output rows: Z[k] = (X_k + conj X_{hu-k})
        // + i exp(2 pi i k / pu) (X_k - conj X_{hu-k}), stored at pos_u(k)
        {
            const int half = hu / 2 + 1;
            for (int idx = tid; idx < G.n_rows_out * half; idx += kFftThreads) {
                const int rr = idx / half, kk = idx - rr * half;
                int row_i = G.out_row0 + rr;
                if (row_i >= pv) row_i -= pv;
                float2 *row = S + row_i * G.pitch;
                const int pk = pos_u[kk];
                const float2 xk = row[pk];
                const float2 xc = cconj(kk == 0 ? row[hu] : row[pos_u[hu - kk]]);
                const float2 sum = cadd(xk, xc), dif = csub(xk, xc);
                const float2 wd = cmul(cconj(Tu[kk]), dif);
                row[pk] = make_float2(sum.x - wd.y, sum.y + wd.x);   // sum + i wd
                if (kk > 0 && 2 * kk != hu) {
                    // Z[hu - k] = (X_{hu-k} + conj X_k) - i exp(-2 pi i k / pu) (X_{hu-k} - conj X_k)
                    const float2 yk = cconj(xc), yc = cconj(xk);   // X_{hu-k}, conj X_k
                    const float2 s2 = cadd(yk, yc), d2 = csub(yk, yc);
                    const float2 w2 = cmul(Tu[kk], d2);
                    row[pos_u[hu - kk]] = make_float2(s2.x + w2.y, s2.y - w2.x);   // s2 - i w2
                }
            }
        }
        __syncthreads();
        fft_run<false, true>(S, G, G.n_rows_out, G.out_row0, hu, Tu, 2, Kf, kv_of, ku_of);
        // output box: (u, v) reads real sample n = (u - in_i0) mod pu of row (v - in_j0) mod pv
        {
            float *dst = ADJ ? P.adjbuf + (long long)bl * P.cap_a + st.off_a
                             : P.region + (long long)bl * P.cap_o + st.off_o;
            const int out_w = bx.out_i1 - bx.out_i0;
            const int n_out = out_w * G.n_rows_out;
            for (int idx = tid; idx < n_out; idx += kFftThreads) {
                const int rr = idx / out_w, uo = idx - rr * out_w;
                int row_i = G.out_row0 + rr;
                if (row_i >= pv) row_i -= pv;
                int n = bx.out_i0 + uo - bx.in_i0;
                if (n < 0) n += pu;
                const float2 z = S[row_i * G.pitch + (n >> 1)];
                dst[(long long)rr * out_w + uo] = (n & 1) ? z.y : z.x;
            }
        }
    }
}

cudaError_t launch_conv_fft(const PlanDev &P, int b0, int nb, bool adjoint, int pmax, unsigned int *counter,
                            int *over_list, unsigned int *over_count, int grid_blocks, cudaStream_t s)
{
    const int smem = conv_fft_smem_bytes(pmax);
    if (adjoint)
        k_conv_fft<true><<<grid_blocks, kFftThreads, smem, s>>>(P, b0, nb, pmax, counter, over_list, over_count);
    else
        k_conv_fft<false><<<grid_blocks, kFftThreads, smem, s>>>(P, b0, nb, pmax, counter, over_list, over_count);
    return cudaGetLastError();
}

// CTAs of one direction per SM at a size limit (shared memory, registers)
cudaError_t conv_fft_ctas(int pmax, bool adjoint, int *ctas)
{
    *ctas = 0;
    if (!fft_size_for(pmax) || fft_size_for(pmax) != pmax) return cudaSuccess;
    cudaError_t e = adjoint ? allow_full_smem(k_conv_fft<true>) : allow_full_smem(k_conv_fft<false>);
    if (e != cudaSuccess) return e;
    int dev = 0, smem_sm = 0, resv = 0, regs_sm = 0, optin = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, adjoint ? (const void *)k_conv_fft<true>
                                                                  : (const void *)k_conv_fft<false>);
    if (e != cudaSuccess) return e;
    const int smem = conv_fft_smem_bytes(pmax);
    if (smem + (int)fa.sharedSizeBytes > optin) return cudaSuccess;
    const int by_smem = smem_sm / (smem + (int)fa.sharedSizeBytes + resv);
    const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
    const int by_regs = regs_sm / (regs_warp * (kFftThreads / 32));
    *ctas = by_smem < by_regs ? by_smem : by_regs;
    return cudaSuccess;
}

}  // namespace pdrt
