// Internal declarations of the sm_103a dose engine (not part of the C ABI).
//
// Data layout in device memory (per plan):
//   cpgeo  [n_cp]            static per-CP geometry (affine maps voxel -> beam lattice)
//   ukr    [n_cp][nw]        static needed u-range of every beam slice (int2)
//   cptab  [n_cp]            per-call CP state (projected MU, fluence support box, ...)
//   slices [n_cp][nw]        per-call slice table (depth, kernel, boxes, offsets)
//   gbox   [n_cp][nw]        the gather's copy of each slice's output box and
//                            region offset, one 16-byte record
//   fbuf   [n_cp][nu*nv]     fluence maps over their support boxes, [a][c] (c fastest)
//   gfbuf  [n_cp][nu*nv]     adjoint of the fluence maps, same layout
//   tbuf   [n_cp][nu*nv]     raw aperture map / its adjoint when the fluence
//                            corrections are on (each map over its own box)
//   region [chunk][cap_o]    beam-frame dose D' (forward) or gathered gradient h
//                            (adjoint) of one chunk of CPs; each slice's box is
//                            stored [j][i] (i fastest) at slices[].off_o
//   adjbuf [chunk][cap_a]    adjoint convolution output on the support boxes
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "pdrt.h"

namespace pdrt {

constexpr int kMaxCpPerChunk = 256;
constexpr int kConvThreads = 128;        // 4 warps: 32 output rows x (4 x 16) output columns
constexpr int kConvTJ = 16;              // output columns per lane
constexpr int kConvCols = 64;            // output columns per CTA
constexpr int kConvRows = 32;            // output rows per CTA (one per lane)
// tensor-core tile limits (output columns N, input columns K per chunk) per
// direction: the forward has wide outputs and narrow inputs, the adjoint the
// reverse; wider boxes are split into column tiles and input chunks
constexpr int kTcFwdMaxN = 128, kTcFwdMaxK = 48;
constexpr int kTcAdjMaxN = 64, kTcAdjMaxK = 48;

enum KernelId {
    K_HU = 0, K_RASTER = 1, K_TABLES = 2, K_CONV_FWD = 3, K_GATHER = 4,
    K_GATHER_T = 5, K_CONV_ADJ = 6, K_MAG_T_GRAD = 7, K_CONV_TC_FWD = 8, K_CONV_TC_ADJ = 9,
    K_CONV_FFT_FWD = 10, K_CONV_FFT_ADJ = 11
};

struct Lattice {
    int nu, nv, nw;
    float cu, cv, cw;     // isocentre lattice index (cu = cw integer)
    float du, dv;         // pitch along u/w and along v
};

// Machine constants in the precision the kernels use.
struct MachineDev {
    float sid;
    int n_pairs;
    float tau, wmin_leaf, wmin_jaw, f_leaf, f_jaw, eps_mu;
    int R;                // kernel half window
    int nq4;              // taps per kernel row rounded up to 4, / 4
    int kstride;          // smem row stride of the kernel table (4 * odd >= 4*nq4)
    float alpha[3][3], beta[3][3];
    int n_depth;
    float depth_step;
    float cal;
    int ste;
    // fluence corrections (Sec. 2.2.2); corr = 0 skips all of them
    int corr;
    int rbu, rbv;                                  // penumbra half-windows (0 = no blur)
    float gu[2 * PDRT_MAX_PEN_RADIUS_PX + 1];      // normalised Gaussian taps, index t + rb
    float gv[2 * PDRT_MAX_PEN_RADIUS_PX + 1];
    float oap[3];                                  // off-axis profile c0 + c1 r + c2 r^2
    int rot;                                       // collimator rotation on
    float rot_c, rot_s;                            // cos, sin of the collimator angle
};

struct CpGeo {
    float au, bu, cu0;    // fu = au*ix + bu*iy + cu0   (beam lattice index along u)
    float aw, bw, cw0;    // fw = aw*ix + bw*iy + cw0   (beam lattice index along w)
    float sx_w, sy_w;     // beam direction e_w projected to voxel index units (x, y)
    float px0, py0, pz0;  // isocentre in voxel index units
};

struct CpTab {
    float mu_hat;         // projected MU
    float cal_mu;         // cal * mu_hat
    int fa0, fa1, fc0, fc1;  // fluence support box [fa0,fa1) x [fc0,fc1) (pixels)
    int ra0, ra1, rc0, rc1;  // raw aperture box (jaw support) before the corrections
    int ca0, ca1, cc0, cc1;  // blurred box (raw box + penumbra half-windows)
    int ui0, ui1, vj0, vj1;  // union over slices of the output boxes (gather culling)
    int k0, k1;           // slices with work [k0,k1)
    long long tot_o, tot_a;  // floats used in the region / adjoint buffers
    long long n_support, n_region, n_active;  // work counters
};

struct alignas(16) SliceTab {
    float z, tdd, m, c2;      // WEPL, depth dose T(z), magnification, inverse square
    float a[3];               // kernel decays
    float pad0;
    float wn[3];              // kernel weights divided by their window sums
    float pad1;
    int pi0, pi1, pj0, pj1;   // conv input box (non-zero fluence volume)
    int oi0, oi1, oj0, oj1;   // forward output box (where D' is produced)
    int ai0, ai1, aj0, aj1;   // adjoint output box
    long long off_o, off_a;   // offsets (floats) inside the CP's region / adjoint slot
};
static_assert(sizeof(SliceTab) % 16 == 0, "SliceTab rows are read as int4");
static_assert(offsetof(SliceTab, oi0) % 16 == 0 && offsetof(SliceTab, ai0) % 16 == 0,
              "box fields must be 16-byte aligned");

struct PlanDev {
    Lattice lat;
    MachineDev mach;
    int n_cp;
    int nx, ny, nz;
    const float *red;        // grid density
    const float *leaf_bounds;  // [n_pairs+1] (device)
    const float *depth_dose;   // [n_depth] (device)
    const CpGeo *cpgeo;
    const int2 *ukr;
    CpTab *cptab;
    SliceTab *slices;
    int4 *gbox;              // [n_cp][nw] per slice: {off_o, oi0, oi1 - oi0, oj0 | oj1 << 16} for the gather
    float *fbuf, *gfbuf;
    float *tbuf;             // [n_cp][nu*nv] raw-map scratch of the corrections (NULL if off)
    float *region, *adjbuf;
    long long cap_o, cap_a;  // floats per CP slot
    unsigned int *flags;
    unsigned int *counters;  // work-queue counters (per chunk launch)
    int tc_enabled;          // 1: every slice with work goes to k_conv_tc
    int tc_phase[2];         // kernel rows per operand phase of k_conv_tc (forward, adjoint)
    int fft_pmax;            // > 0: k_conv_fft takes every slice whose padded sizes are at most
                             // this; k_conv_tc takes the rest from the overflow list
    int *fft_over;           // [chunk * nw] overflow list of one chunk launch (items)
    unsigned int *fft_ctr;   // [4 * n_cp]: per chunk {fwd counter, fwd overflow count,
                             // adj counter, adj overflow count}
    const float *fft_cos;    // c_p cos(2 pi k p / P) per supported size P (conv_fft_cos_table)
    // kernel-spectrum memo of the FFT convolution: entry b * nw + k holds the
    // spectrum Kf of slice k of control point b ([kv'][ku], nkv rows of pu/2
    // + 1) as the FFT kernel computed it, tagged kf_tag = (pu << 16) | pv (0:
    // empty); slices with sizes above kf_pmax are not memoised; NULL: off
    float *kf_memo;
    int *kf_tag;
    int kf_pmax;
    long long kf_stride;     // floats per entry (16-byte multiple)
};

// Same float expression in every kernel that samples or transposes the
// magnified fluence (forward tile fill and its adjoint).
__device__ __forceinline__ float mag_coord(float m, int idx, float c)
{
    return fmaf(m, (float)idx - c, c);
}

// Beam lattice coordinates of voxel (ix, iy) for one control point; shared
// by the gather and its transpose so both use bit-identical weights.
__device__ __forceinline__ void voxel_to_beam(const CpGeo &g, int ix, int iy, float &fu, float &fw)
{
    fu = fmaf(g.au, (float)ix, fmaf(g.bu, (float)iy, g.cu0));
    fw = fmaf(g.aw, (float)ix, fmaf(g.bw, (float)iy, g.cw0));
}

// Pull-form transpose of the gather (k_gather) at lattice column (i, k) of
// one control point: the voxels (ix, iy) of a plane whose bilinear stencil
// holds lattice point (i, k), with their weights.  Such a voxel's centre is
// within sqrt(2) voxels of the point's rotated position on each axis, so the
// 3 x 3 window around the rounded position holds all of them; the weights
// are the forward's (voxel_to_beam, 1 - |f - n|).  The taps depend on (i, k)
// only, not on the plane: they are written once (non-zero ones, row-major
// order, taps[q * stride] = {weight, in-plane offset iy * nx + ix}; the count
// is returned) and every plane j sums w_0 g_j[off_0] + w_1 g_j[off_1] + ...
// in that order.
struct GtTap {
    float w;
    int off;
};

__device__ __forceinline__ int gather_t_taps(const CpGeo &g, const Lattice &L, int nx, int ny, int i, int k,
                                             GtTap *taps, int stride)
{
    const float di = (float)i - L.cu, dk = (float)k - L.cw;
    const float fx = fmaf(di, g.au, fmaf(dk, g.aw, g.px0));
    const float fy = fmaf(di, g.bu, fmaf(dk, g.bw, g.py0));
    const int cx = __float2int_rn(fx), cy = __float2int_rn(fy);
    int n = 0;
#pragma unroll
    for (int r = -1; r <= 1; ++r) {
        const int iy = cy + r;
        const bool row_ok = iy >= 0 && iy < ny;
#pragma unroll
        for (int c = -1; c <= 1; ++c) {
            const int ix = cx + c;
            const bool ok = row_ok && ix >= 0 && ix < nx;
            float fu, fw;
            voxel_to_beam(g, ix, iy, fu, fw);
            const float wu = fmaxf(0.f, 1.f - fabsf(fu - (float)i));
            const float ww = fmaxf(0.f, 1.f - fabsf(fw - (float)k));
            const float wgt = ok ? ww * wu : 0.f;
            if (wgt != 0.f) {
                taps[n * stride] = GtTap{wgt, iy * nx + ix};
                ++n;
            }
        }
    }
    return n;
}

// Bilinear sample of fluence map b (stored over its support box) at the
// magnified position (fa, fc) of a lattice point (same expression in every
// convolution kernel that fills its input from the fluence).
__device__ __forceinline__ float fluence_sample(const float *__restrict__ F, int fa0, int fa1,
                                                int fc0, int fc1, float fa, float fc)
{
    const float ba = floorf(fa), bc = floorf(fc);
    const int a0 = (int)ba, c0 = (int)bc;
    const float ta = fa - ba, tc = fc - bc;
    const int Fc = fc1 - fc0;
    float s = 0.f;
#pragma unroll
    for (int da = 0; da < 2; ++da) {
        const int a = a0 + da;
        if (a < fa0 || a >= fa1) continue;
        const float wa = da ? ta : 1.f - ta;
#pragma unroll
        for (int dc = 0; dc < 2; ++dc) {
            const int c = c0 + dc;
            if (c < fc0 || c >= fc1) continue;
            const float wc = dc ? tc : 1.f - tc;
            s += wa * wc * __ldg(&F[(long long)(a - fa0) * Fc + (c - fc0)]);
        }
    }
    return s;
}

// Padded sizes of the FFT convolution: the sizes whose complex transform
// lengths (P along v, P / 2 along u) have radix plans in k_conv_fft.
__host__ __device__ inline int fft_size_for(int n)
{
    const int sizes[16] = {32, 40, 48, 60, 64, 72, 80, 90, 96, 100, 108, 120, 128, 144, 160, 192};
    for (int t = 0; t < 16; ++t)
        if (sizes[t] >= n) return sizes[t];
    return 0;
}

// Padded sizes (pu, pv) of one slice's convolution in one direction: the
// circular period along each axis that keeps every tap within R of an
// output and no tap beyond R (max distance between an output and an input
// point + R + 1), and at least the input and output extents; 0 for a slice
// without work, 1 << 20 if no supported size is large enough.
__host__ __device__ inline void fft_slice_sizes(const SliceTab &st, bool adj, int R, int &pu, int &pv)
{
    const int ii0 = adj ? st.oi0 : st.pi0, ii1 = adj ? st.oi1 : st.pi1;
    const int ij0 = adj ? st.oj0 : st.pj0, ij1 = adj ? st.oj1 : st.pj1;
    const int oi0 = adj ? st.ai0 : st.oi0, oi1 = adj ? st.ai1 : st.oi1;
    const int oj0 = adj ? st.aj0 : st.oj0, oj1 = adj ? st.aj1 : st.oj1;
    pu = pv = 0;
    if (!(oi1 > oi0 && oj1 > oj0 && ii1 > ii0 && ij1 > ij0)) return;
    int nu = (oi1 - 1 - ii0 > ii1 - 1 - oi0 ? oi1 - 1 - ii0 : ii1 - 1 - oi0) + R + 1;
    int nv = (oj1 - 1 - ij0 > ij1 - 1 - oj0 ? oj1 - 1 - ij0 : ij1 - 1 - oj0) + R + 1;
    nu = nu > ii1 - ii0 ? nu : ii1 - ii0;
    nu = nu > oi1 - oi0 ? nu : oi1 - oi0;
    nv = nv > ij1 - ij0 ? nv : ij1 - ij0;
    nv = nv > oj1 - oj0 ? nv : oj1 - oj0;
    pu = fft_size_for(nu);
    pv = fft_size_for(nv);
    if (!pu || !pv) pu = pv = 1 << 20;
}

// Off-axis profile factor of lattice pixel (a, c) (Sec. 2.2.2).
__device__ __forceinline__ float off_axis_factor(const MachineDev &M, const Lattice &L, int a, int c)
{
    const float u = ((float)a - L.cu) * L.du, v = ((float)c - L.cv) * L.dv;
    const float r = sqrtf(u * u + v * v);
    return fmaf(fmaf(M.oap[2], r, M.oap[1]), r, M.oap[0]);
}

// Fractional lattice indices that the collimator rotation brings to pixel
// (a, c): pixel x reads the corrected map at R(-angle) x.  One expression for
// the forward resampling and its transpose.
__device__ __forceinline__ void rotation_source(const MachineDev &M, const Lattice &L, int a, int c,
                                                float &fa, float &fc)
{
    const float u = ((float)a - L.cu) * L.du, v = ((float)c - L.cv) * L.dv;
    fa = L.cu + fmaf(M.rot_c, u, M.rot_s * v) / L.du;
    fc = L.cv + fmaf(-M.rot_s, u, M.rot_c * v) / L.dv;
}

__device__ __forceinline__ float overlap_f(float x, float lo, float hi, float d)
{
    float e = x + 0.5f * d, s = x - 0.5f * d;
    float top = (hi <= e) ? hi : e;
    float bot = (lo >= s) ? lo : s;
    float X = top - bot;
    return X > 0.f ? X / d : 0.f;
}


// Boxes of one slice for one convolution direction, and the column ranges the
// tensor-core path uses (input columns [s0, s0 + kt), kt and nt multiples of 16).
struct TcBoxes {
    int in_i0, in_i1, in_j0, in_j1, out_i0, out_i1, out_j0, out_j1;
};

__device__ __forceinline__ TcBoxes tc_boxes(const SliceTab &st, bool adj, int R)
{
    (void)R;
    TcBoxes b;
    if (adj) {
        b.in_i0 = st.oi0; b.in_i1 = st.oi1; b.in_j0 = st.oj0; b.in_j1 = st.oj1;
        b.out_i0 = st.ai0; b.out_i1 = st.ai1; b.out_j0 = st.aj0; b.out_j1 = st.aj1;
    } else {
        b.in_i0 = st.pi0; b.in_i1 = st.pi1; b.in_j0 = st.pj0; b.in_j1 = st.pj1;
        b.out_i0 = st.oi0; b.out_i1 = st.oi1; b.out_j0 = st.oj0; b.out_j1 = st.oj1;
    }
    return b;
}

// Every slice is convolved by exactly one of k_conv_tc (true) and k_conv
// (false): the tensor-core kernel tiles any box (column tiles and input
// chunks), so with tensor cores on it takes every slice with work.
__device__ __forceinline__ bool tc_takes_slice(const SliceTab &st, bool adj, int R, int tc_enabled)
{
    if (!tc_enabled) return false;
    const TcBoxes b = tc_boxes(st, adj, R);
    return b.out_i1 > b.out_i0 && b.out_j1 > b.out_j0 && b.in_i1 > b.in_i0 && b.in_j1 > b.in_j0;
}

// launchers (one per kernel); each returns cudaGetLastError() of its launch
cudaError_t launch_hu_to_red(const float *hu, float *red, long long n, const float *pts, int npts,
                             cudaStream_t s);
cudaError_t launch_raster(const PlanDev &P, const float *leaves, const float *jaws,
                          const float *mu, cudaStream_t s);
cudaError_t launch_tables(const PlanDev &P, cudaStream_t s);
cudaError_t launch_conv(const PlanDev &P, int b0, int nb, bool adjoint, unsigned int *counter,
                        int grid_blocks, cudaStream_t s);
cudaError_t launch_gather(const PlanDev &P, int b0, int nb, float *dose, bool first,
                          cudaStream_t s);
cudaError_t launch_gather_T(const PlanDev &P, int b0, int nb, const float *g, cudaStream_t s);
// What the gather and its transpose read of a plan: the batched launches
// carry one of these per entry in their kernel parameters.
struct GatherPlan {
    Lattice lat;
    int nx, ny, nz;
    const CpTab *cptab;
    const CpGeo *cpgeo;
    const SliceTab *slices;
    const int4 *gbox;
    float *region;
    long long cap_o;
};
inline GatherPlan gather_plan_of(const PlanDev &P)
{
    GatherPlan g;
    g.lat = P.lat;
    g.nx = P.nx;
    g.ny = P.ny;
    g.nz = P.nz;
    g.cptab = P.cptab;
    g.cpgeo = P.cpgeo;
    g.slices = P.slices;
    g.gbox = P.gbox;
    g.region = P.region;
    g.cap_o = P.cap_o;
    return g;
}
// one plan's pass in a batched gather (dose, first) or gather transpose (gd)
struct GatherEntry {
    GatherPlan p;
    float *dose;
    const float *gd;
    int b0, nb, first;
    int blk0, gx, gy;        // set by the launcher
};
constexpr int kGatherBatchMax = 128;
// one launch per group of up to kGatherBatchMax entries: the gathers
// (transpose = false: accumulate pass b0 .. b0 + nb - 1 into dose, first =
// overwrite) or the gather transposes (transpose = true: h of the pass from
// gd) of several plans, each CTA as in the per-plan launch
cudaError_t launch_gather_multi(const GatherEntry *ents, int n, bool transpose, cudaStream_t s);
cudaError_t launch_mag_T(const PlanDev &P, int b0, int nb, cudaStream_t s);
cudaError_t launch_param_grad(const PlanDev &P, const float *leaves, const float *jaws,
                              const float *mu, float *dleaves, float *djaws, float *dmu,
                              cudaStream_t s);
int conv_smem_bytes(const MachineDev &m);
int conv_nq4_for_radius(int R);
cudaError_t conv_prepare(const MachineDev &m, int *fwd_blocks_per_sm, int *adj_blocks_per_sm);
// list / list_n: when list != NULL the kernel takes only the items of the
// list (its first *list_n entries) instead of every item of the chunk
cudaError_t launch_conv_tc(const PlanDev &P, int b0, int nb, bool adjoint, unsigned int *counter,
                           int grid_blocks, cudaStream_t s, const int *list = nullptr,
                           const unsigned int *list_n = nullptr);
cudaError_t launch_conv_fft(const PlanDev &P, int b0, int nb, bool adjoint, int pmax, unsigned int *counter,
                            int *over_list, unsigned int *over_count, int grid_blocks, cudaStream_t s);
int conv_fft_smem_bytes(int pmax, int R);
// the kernel spectra of pass b0 .. b0 + nb - 1 into the plan's memo, for the
// padded sizes of one direction (a no-op without a memo); the FFT
// convolution of the pass then takes them from it
cudaError_t launch_spectrum(const PlanDev &P, int b0, int nb, bool adjoint, int pmax, cudaStream_t s);
// What the FFT convolution reads of a plan: the batched launch carries one
// of these per entry in its kernel parameters.
struct FftPlan {
    Lattice lat;
    const SliceTab *slices;
    const CpTab *cptab;
    const float *fbuf;
    float *region, *adjbuf;
    const float *fft_cos;
    int *fft_over;
    unsigned int *fft_ctr;
    long long cap_o, cap_a;
    int R, fft_pmax;
    float *kf_memo;
    int *kf_tag;
    int kf_pmax;
    long long kf_stride;
};
inline FftPlan fft_plan_of(const PlanDev &P)
{
    FftPlan f;
    f.lat = P.lat;
    f.slices = P.slices;
    f.cptab = P.cptab;
    f.fbuf = P.fbuf;
    f.region = P.region;
    f.adjbuf = P.adjbuf;
    f.fft_cos = P.fft_cos;
    f.fft_over = P.fft_over;
    f.fft_ctr = P.fft_ctr;
    f.cap_o = P.cap_o;
    f.cap_a = P.cap_a;
    f.R = P.mach.R;
    f.fft_pmax = P.fft_pmax;
    f.kf_memo = P.kf_memo;
    f.kf_tag = P.kf_tag;
    f.kf_pmax = P.kf_pmax;
    f.kf_stride = P.kf_stride;
    return f;
}
// entries of one batched FFT launch (its kernel parameters stay under the
// 32 KB limit)
constexpr int kFftBatchMax = 160;
// one persistent FFT launch per group of up to kFftBatchMax entries (plan
// passes): plans[e] with round[e] = {b0, nb, -, pass index} for e < n_ent;
// counters[g] is the work counter of group g (zeroed beforehand); smem for
// the largest size limit and kernel radius among them, grid = CTAs per SM x
// SMs.  Groups: (n_ent + kFftBatchMax - 1) / kFftBatchMax.
cudaError_t launch_conv_fft_multi(const FftPlan *plans, const int4 *round, int n_ent, int pmax, int smem,
                                  int grid_blocks, bool adjoint, unsigned int *counters, cudaStream_t s);
// CTAs per SM of k_conv_fft for a size limit (0 if it does not fit or is
// below 2 R + 2); uploads the constant size tables to the current device
cudaError_t conv_fft_ctas(int pmax, int R, bool adjoint, int *ctas);
// the plan's cosine table of the kernel spectrum: its length (floats) and
// contents (host) for a kernel half-width R
int conv_fft_cos_floats(int R);
void conv_fft_cos_table(int R, float *out);
cudaError_t conv_tc_prepare(int R, int *fwd_blocks_per_sm, int *adj_blocks_per_sm, int *fwd_phase,
                            int *adj_phase);
// CTAs per SM of k_conv_tc for a phase depth (0 if the phase does not fit).
cudaError_t conv_tc_ctas(int R, bool adjoint, int phase, int *ctas);
// Device form of a machine's fluence corrections (taps, profile, rotation);
// returns an error text or NULL.  Pitches du, dv in mm.
const char *machine_corrections(const pdrt_machine *m, double du, double dv, MachineDev &M);

// Raises a kernel's dynamic shared-memory limit to everything the device
// offers one block and asks for the largest shared-memory carve-out. The
// limit is a property of the kernel, not of a launch: plans of different
// kernel radii share one instantiation, so it is never lowered to one plan's
// need (a smaller later plan would invalidate a larger earlier one).
template <typename Kern>
inline cudaError_t allow_full_smem(Kern kern)
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    return e;
}
int conv_tc_smem_bytes(int R, bool adjoint, int phase);
// u-range [lo, hi) of beam slice k needed by some voxel of the grid whose
// corners map to lattice indices (fu[c], fw[c]) (host; one definition for the
// plan upload and the allocation-free entry point, so both size their regions
// identically)
void needed_u_range(const double fu[4], const double fw[4], int k, int nu, int &lo, int &hi);
void internal_set_error(const char *msg);   // sets pdrt_last_error() for this thread
void internal_count_launch();                // counts one launch in pdrt_launch_count()

}  // namespace pdrt
