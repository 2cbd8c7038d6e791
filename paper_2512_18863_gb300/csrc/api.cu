// C ABI of the dose engine (declared in include/pdrt.h): argument checks, the
// beam-frame lattice and per-slice needed ranges (host, double precision),
// scratch allocation at plan upload, and the launch sequence of the forward
// and adjoint passes.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <string>
#include <vector>

#include "pdrt_impl.cuh"

using namespace pdrt;

namespace {

thread_local std::string g_last_error;
std::atomic<long long> g_launches{0};

pdrt_status fail(pdrt_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

pdrt_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(e == cudaErrorMemoryAllocation ? PDRT_ENOMEM : PDRT_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define CU_TRY(expr, what)                         \
    do {                                           \
        cudaError_t e_ = (expr);                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

}  // namespace

struct pdrt_grid_s {
    int device;
    int sm_count;
    int nx, ny, nz;
    double sx, sy, sz;
    double origin[3];
    float *red;
};

struct ProfileRec {
    int kid;
    int ev;
};

struct pdrt_plan_s {
    pdrt_grid_t grid;
    int n_cp;
    int chunk;
    int chunk_max;            // control points per pass the scratch was sized for
    int conv_blocks_fwd, conv_blocks_adj;
    int tc_blocks;            // persistent grid of k_conv_tc<false> (0: path unavailable)
    int tc_blocks_adj;        // persistent grid of k_conv_tc<true>
    int fft_blocks[2];        // persistent grids of k_conv_fft (forward, adjoint) at dev.fft_pmax
    PlanDev dev;
    size_t scratch_bytes;
    std::vector<void *> allocs;
    size_t memo_bytes = 0;    // kernel-spectrum memo (dev.kf_memo, dev.kf_tag), held apart from allocs
    // profiling
    bool profiling = false;
    std::vector<cudaEvent_t> events;
    std::vector<ProfileRec> recs;
    int next_ev = 0;
    bool overflow = false;
};

static const char *kKernelNames[PDRT_NUM_KERNELS] = {
    "hu_to_red", "project_raster", "wepl_tables", "conv_forward",
    "gather_accumulate", "gather_transpose", "conv_adjoint", "mag_transpose_param_grad",
    "conv_forward_tc", "conv_adjoint_tc", "conv_forward_fft", "conv_adjoint_fft"};

namespace {

template <typename T>
cudaError_t dalloc(pdrt_plan_t p, T **ptr, size_t count)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    p->allocs.push_back(q);
    p->scratch_bytes += std::max<size_t>(count, 1) * sizeof(T);
    *ptr = static_cast<T *>(q);
    return cudaSuccess;
}

// Launch with optional event timing on the launch stream.
template <typename F>
cudaError_t timed(pdrt_plan_t p, int kid, cudaStream_t s, F &&launch)
{
    int ev = -1;
    if (p && p->profiling) {
        if (p->next_ev + 2 <= (int)p->events.size()) {
            ev = p->next_ev;
            p->next_ev += 2;
            cudaEventRecord(p->events[ev], s);
        } else {
            p->overflow = true;
        }
    }
    cudaError_t e = launch();
    g_launches.fetch_add(1);
    if (ev >= 0) {
        cudaEventRecord(p->events[ev + 1], s);
        p->recs.push_back({kid, ev});
    }
    return e;
}

bool is_fin(double x) { return std::isfinite(x); }

}  // namespace

// u-range [lo, hi) of the beam lattice points of slice k that some voxel's
// bilinear stencil can touch: the rotated grid rectangle in (fu, fw) index
// space clipped to the band fw in [k-1, k+1], widened by one point.
void pdrt::needed_u_range(const double fu[4], const double fw[4], int k, int nu, int &lo, int &hi)
{
    double umin = 1e300, umax = -1e300;
    const double b0 = k - 1.0, b1 = k + 1.0;
    for (int e = 0; e < 4; ++e) {
        const int f = (e + 1) & 3;
        const double w0 = fw[e], w1 = fw[f], u0 = fu[e], u1 = fu[f];
        double tlo, thi;
        if (fabs(w1 - w0) < 1e-12) {
            if (w0 < b0 || w0 > b1) continue;
            tlo = 0.0;
            thi = 1.0;
        } else {
            double t0 = (b0 - w0) / (w1 - w0), t1 = (b1 - w0) / (w1 - w0);
            tlo = std::max(0.0, std::min(t0, t1));
            thi = std::min(1.0, std::max(t0, t1));
            if (tlo > thi) continue;
        }
        for (double t : {tlo, thi}) {
            const double u = u0 + t * (u1 - u0);
            umin = std::min(umin, u);
            umax = std::max(umax, u);
        }
    }
    if (umin > umax) {
        lo = hi = 0;
        return;
    }
    lo = std::max((int)floor(umin) - 1, 0);
    hi = std::min((int)floor(umax) + 3, nu);
    if (hi < lo) hi = lo;
}

// Hooks for entry points defined in other translation units.
void pdrt::internal_set_error(const char *msg) { g_last_error = msg ? msg : ""; }
void pdrt::internal_count_launch() { g_launches.fetch_add(1); }

// Penumbra taps, off-axis profile and collimator rotation of a machine
// (Sec. 2.2.2) in device form; returns an error text or NULL.  The Gaussian
// taps are evaluated and normalised in double precision on the host.
const char *pdrt::machine_corrections(const pdrt_machine *m, double du, double dv, MachineDev &M)
{
    const double fw[2] = {m->pen_fwhm_u_mm, m->pen_fwhm_v_mm}, pitch[2] = {du, dv};
    int rb[2] = {0, 0};
    for (int ax = 0; ax < 2; ++ax) {
        float *taps = ax ? M.gv : M.gu;
        for (int t = 0; t < 2 * PDRT_MAX_PEN_RADIUS_PX + 1; ++t) taps[t] = 0.f;
        if (!(fw[ax] > 0)) continue;
        const double sigma = fw[ax] / (2.0 * sqrt(2.0 * log(2.0)));
        const double r = ceil(3.0 * sigma / pitch[ax]);
        if (r > PDRT_MAX_PEN_RADIUS_PX) return "penumbra blur wider than PDRT_MAX_PEN_RADIUS_PX pixels";
        rb[ax] = (int)r;
        double w[2 * PDRT_MAX_PEN_RADIUS_PX + 1], sum = 0.0;
        for (int t = -rb[ax]; t <= rb[ax]; ++t) {
            const double x = t * pitch[ax];
            w[t + rb[ax]] = exp(-x * x / (2.0 * sigma * sigma));
            sum += w[t + rb[ax]];
        }
        for (int t = 0; t <= 2 * rb[ax]; ++t) taps[t] = (float)(w[t] / sum);
    }
    M.rbu = rb[0];
    M.rbv = rb[1];
    for (int q = 0; q < 3; ++q) M.oap[q] = (float)m->off_axis[q];
    const bool oap_on = !(m->off_axis[0] == 1.0 && m->off_axis[1] == 0.0 && m->off_axis[2] == 0.0);
    M.rot = m->collimator_deg != 0.0 ? 1 : 0;
    const double th = m->collimator_deg * M_PI / 180.0;
    M.rot_c = (float)cos(th);
    M.rot_s = (float)sin(th);
    M.corr = (M.rbu > 0 || M.rbv > 0 || oap_on || M.rot) ? 1 : 0;
    return nullptr;
}

extern "C" {

const char *pdrt_last_error(void) { return g_last_error.c_str(); }

int64_t pdrt_launch_count(void) { return g_launches.load(); }

pdrt_status pdrt_grid_create(pdrt_grid_t *out, const float *hu_dev, int32_t nx, int32_t ny,
                             int32_t nz, double sx, double sy, double sz, const double origin_mm[3],
                             const double *hu_red_host, int32_t n_pts, pdrt_stream_t stream)
{
    g_last_error.clear();
    if (!out || !hu_dev || !origin_mm || !hu_red_host) return fail(PDRT_EINVAL, "NULL argument");
    *out = nullptr;
    if (nx <= 0 || ny <= 0 || nz <= 0) return fail(PDRT_ESHAPE, "grid dimensions must be positive");
    if (!(sx > 0) || !(sy > 0) || !(sz > 0) || !is_fin(sx) || !is_fin(sy) || !is_fin(sz))
        return fail(PDRT_EINVAL, "voxel spacing must be positive and finite");
    if (fabs(sx - sy) > 1e-6 * sx) return fail(PDRT_EINVAL, "sx must equal sy (got %g, %g)", sx, sy);
    for (int d = 0; d < 3; ++d)
        if (!is_fin(origin_mm[d])) return fail(PDRT_EINVAL, "origin must be finite");
    if (n_pts < 2 || n_pts > PDRT_MAX_HU_POINTS)
        return fail(PDRT_EINVAL, "HU calibration needs 2..%d points", PDRT_MAX_HU_POINTS);
    for (int i = 0; i < n_pts; ++i) {
        if (!is_fin(hu_red_host[2 * i]) || !is_fin(hu_red_host[2 * i + 1]))
            return fail(PDRT_EINVAL, "HU calibration point %d is not finite", i);
        if (i > 0 && !(hu_red_host[2 * i] > hu_red_host[2 * i - 2]))
            return fail(PDRT_EINVAL, "HU calibration points must be strictly ascending in HU");
    }
    int dev = 0;
    CU_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    cudaDeviceProp prop;
    CU_TRY(cudaGetDeviceProperties(&prop, dev), "cudaGetDeviceProperties");
    if (prop.major * 10 + prop.minor != 103)
        return fail(PDRT_EDEVICE, "device %d is sm_%d%d; this library is built for sm_103a", dev,
                    prop.major, prop.minor);
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, hu_dev) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail(PDRT_EINVAL, "hu_dev is not a device pointer");
    }
    const long long n = (long long)nx * ny * nz;
    pdrt_grid_t g = new pdrt_grid_s();
    g->device = dev;
    g->sm_count = prop.multiProcessorCount;
    g->nx = nx; g->ny = ny; g->nz = nz;
    g->sx = sx; g->sy = sy; g->sz = sz;
    for (int d = 0; d < 3; ++d) g->origin[d] = origin_mm[d];
    cudaError_t e = cudaMalloc(&g->red, n * sizeof(float));
    if (e != cudaSuccess) {
        delete g;
        return cuda_fail(e, "cudaMalloc(density)");
    }
    float pts[2 * PDRT_MAX_HU_POINTS];
    for (int i = 0; i < 2 * n_pts; ++i) pts[i] = (float)hu_red_host[i];
    e = launch_hu_to_red(hu_dev, g->red, n, pts, n_pts, (cudaStream_t)stream);
    g_launches.fetch_add(1);
    if (e != cudaSuccess) {
        cudaFree(g->red);
        delete g;
        return cuda_fail(e, "hu_to_red launch");
    }
    *out = g;
    return PDRT_OK;
}

void pdrt_grid_destroy(pdrt_grid_t g)
{
    if (!g) return;
    cudaFree(g->red);
    delete g;
}

namespace {

void memo_free(pdrt_plan_t p)
{
    cudaFree(p->dev.kf_memo);
    cudaFree(p->dev.kf_tag);
    p->dev.kf_memo = nullptr;
    p->dev.kf_tag = nullptr;
    p->dev.kf_pmax = 0;
    p->dev.kf_stride = 0;
    p->memo_bytes = 0;
}

// kernel-spectrum memo for slices of padded sizes up to pmax: one entry of
// (pmax/2 + 1)^2 floats (rounded up to 4) per (control point, slice), tags
// cleared before it returns
cudaError_t memo_alloc(pdrt_plan_t p, int pmax)
{
    memo_free(p);
    const long long entries = (long long)p->n_cp * p->dev.lat.nw;
    const long long stride = (((long long)(pmax / 2 + 1) * (pmax / 2 + 1)) + 3) & ~3LL;
    float *memo = nullptr;
    int *tag = nullptr;
    cudaError_t e = cudaMalloc(&memo, sizeof(float) * (size_t)(entries * stride));
    if (e == cudaSuccess) e = cudaMalloc(&tag, sizeof(int) * (size_t)entries);
    if (e == cudaSuccess) e = cudaMemset(tag, 0, sizeof(int) * (size_t)entries);
    // the tags must be clear before any stream (non-blocking ones included)
    // runs a convolution of the plan: a stale tag would read as a stored
    // spectrum
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) {
        cudaFree(memo);
        cudaFree(tag);
        return e;
    }
    p->dev.kf_memo = memo;
    p->dev.kf_tag = tag;
    p->dev.kf_pmax = pmax;
    p->dev.kf_stride = stride;
    p->memo_bytes = sizeof(float) * (size_t)(entries * stride) + sizeof(int) * (size_t)entries;
    return cudaSuccess;
}

}  // namespace

void pdrt_plan_destroy(pdrt_plan_t p)
{
    if (!p) return;
    memo_free(p);
    for (void *q : p->allocs) cudaFree(q);
    for (cudaEvent_t e : p->events) cudaEventDestroy(e);
    delete p;
}

pdrt_status pdrt_plan_upload(pdrt_plan_t *out, pdrt_grid_t g, int32_t n_cp,
                             const double *gantry_deg_host, const double iso_mm[3],
                             const pdrt_machine *m, size_t scratch_budget_bytes,
                             pdrt_stream_t stream)
{
    g_last_error.clear();
    if (!out || !g || !gantry_deg_host || !iso_mm || !m) return fail(PDRT_EINVAL, "NULL argument");
    *out = nullptr;
    if (n_cp <= 0) return fail(PDRT_ESHAPE, "n_cp must be positive");
    for (int b = 0; b < n_cp; ++b)
        if (!is_fin(gantry_deg_host[b])) return fail(PDRT_EINVAL, "gantry angle %d is not finite", b);
    for (int d = 0; d < 3; ++d)
        if (!is_fin(iso_mm[d])) return fail(PDRT_EINVAL, "isocentre must be finite");
    if (m->n_pairs < 1 || m->n_pairs > PDRT_MAX_PAIRS)
        return fail(PDRT_EINVAL, "n_pairs must be in 1..%d", PDRT_MAX_PAIRS);
    for (int i = 0; i <= m->n_pairs; ++i) {
        if (!is_fin(m->leaf_bounds_mm[i])) return fail(PDRT_EINVAL, "leaf bound %d not finite", i);
        if (i > 0 && !(m->leaf_bounds_mm[i] > m->leaf_bounds_mm[i - 1]))
            return fail(PDRT_EINVAL, "leaf bounds must be strictly ascending");
    }
    if (m->kernel_radius_px < 0 || m->kernel_radius_px > PDRT_MAX_RADIUS_PX)
        return fail(PDRT_EINVAL, "kernel radius must be in 0..%d px", PDRT_MAX_RADIUS_PX);
    if (m->n_depth < 2 || m->n_depth > PDRT_MAX_DEPTH_TABLE || !(m->depth_step_mm > 0))
        return fail(PDRT_EINVAL, "depth-dose table needs 2..%d entries and a positive step",
                    PDRT_MAX_DEPTH_TABLE);
    if (!(m->tau >= 0 && m->tau <= 1)) return fail(PDRT_EINVAL, "tau must be in [0,1]");
    if (!(m->wmin_leaf_mm >= 0) || !(m->wmin_jaw_mm >= 0) || !(m->f_leaf_mm >= 0) ||
        !(m->f_jaw_mm >= 0) || !(m->eps_mu >= 0) || !is_fin(m->cal) || !is_fin(m->sid_mm))
        return fail(PDRT_EINVAL, "machine limits must be non-negative and finite");
    for (int c = 0; c < 3; ++c)
        for (int q = 0; q < 3; ++q)
            if (!is_fin(m->kernel_alpha[c][q]) || !is_fin(m->kernel_beta[c][q]))
                return fail(PDRT_EINVAL, "kernel polynomial coefficients must be finite");
    for (int i = 0; i < m->n_depth; ++i)
        if (!is_fin(m->depth_dose[i])) return fail(PDRT_EINVAL, "depth-dose entry %d not finite", i);
    if (!(m->pen_fwhm_u_mm >= 0) || !(m->pen_fwhm_v_mm >= 0) || !is_fin(m->pen_fwhm_u_mm) ||
        !is_fin(m->pen_fwhm_v_mm))
        return fail(PDRT_EINVAL, "penumbra FWHM must be non-negative and finite");
    for (int q = 0; q < 3; ++q)
        if (!is_fin(m->off_axis[q])) return fail(PDRT_EINVAL, "off-axis coefficients must be finite");
    if (!is_fin(m->collimator_deg)) return fail(PDRT_EINVAL, "collimator angle must be finite");
    int dev = 0;
    CU_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != g->device) return fail(PDRT_EINVAL, "current device differs from the grid's device");

    // ---- lattice (same definition as the model: +-H pixels, H covers every voxel)
    double rmax = 0.0;
    for (int cx = 0; cx < 2; ++cx)
        for (int cy = 0; cy < 2; ++cy) {
            double x = g->origin[0] + (cx ? g->nx - 1 : 0) * g->sx - iso_mm[0];
            double y = g->origin[1] + (cy ? g->ny - 1 : 0) * g->sy - iso_mm[1];
            rmax = std::max(rmax, sqrt(x * x + y * y));
        }
    const int H = (int)ceil(rmax / g->sx - 1e-9) + 1;
    Lattice L;
    L.nu = L.nw = 2 * H + 1;
    L.nv = g->nz;
    L.cu = L.cw = (float)H;
    const double cv = (iso_mm[2] - g->origin[2]) / g->sz;
    L.cv = (float)cv;
    L.du = (float)g->sx;
    L.dv = (float)g->sz;
    if (!(m->sid_mm > (H + 2) * g->sx))
        return fail(PDRT_EINVAL, "SID %.1f mm must exceed the grid's reach from the isocentre (%.1f mm)",
                    m->sid_mm, (H + 2) * g->sx);

    MachineDev M;
    memset(&M, 0, sizeof(M));
    M.sid = (float)m->sid_mm;
    M.n_pairs = m->n_pairs;
    M.tau = (float)m->tau;
    M.wmin_leaf = (float)m->wmin_leaf_mm;
    M.wmin_jaw = (float)m->wmin_jaw_mm;
    M.f_leaf = (float)m->f_leaf_mm;
    M.f_jaw = (float)m->f_jaw_mm;
    M.eps_mu = (float)m->eps_mu;
    M.R = m->kernel_radius_px;
    M.nq4 = conv_nq4_for_radius(M.R);
    if (M.nq4 < 0) return fail(PDRT_EINVAL, "no convolution variant for radius %d", M.R);
    M.kstride = 4 * ((M.nq4 & 1) ? M.nq4 : M.nq4 + 1);
    for (int c = 0; c < 3; ++c)
        for (int q = 0; q < 3; ++q) {
            M.alpha[c][q] = (float)m->kernel_alpha[c][q];
            M.beta[c][q] = (float)m->kernel_beta[c][q];
        }
    M.n_depth = m->n_depth;
    M.depth_step = (float)m->depth_step_mm;
    M.cal = (float)m->cal;
    M.ste = m->ste ? 1 : 0;
    {
        const char *why = machine_corrections(m, g->sx, g->sz, M);
        if (why) return fail(PDRT_EINVAL, "%s", why);
    }

    // ---- per-CP geometry and needed slice ranges
    std::vector<CpGeo> geo(n_cp);
    std::vector<int2> ukr((size_t)n_cp * L.nw);
    const double px0 = (iso_mm[0] - g->origin[0]) / g->sx;
    const double py0 = (iso_mm[1] - g->origin[1]) / g->sy;
    const double pz0 = cv;
    long long cap_o = 1, cap_a = 1;
    const int R = M.R;
    for (int b = 0; b < n_cp; ++b) {
        const double phi = gantry_deg_host[b] * M_PI / 180.0;
        const double cs = cos(phi), sn = sin(phi);
        const double au = cs, bu = -sn, aw = sn, bw = cs;
        CpGeo &G = geo[b];
        G.au = (float)au; G.bu = (float)bu; G.aw = (float)aw; G.bw = (float)bw;
        G.cu0 = (float)(H - au * px0 - bu * py0);
        G.cw0 = (float)(H - aw * px0 - bw * py0);
        G.sx_w = (float)sn;
        G.sy_w = (float)cs;
        G.px0 = (float)px0; G.py0 = (float)py0; G.pz0 = (float)pz0;
        double fu[4], fw[4];
        const int cxs[4] = {0, g->nx - 1, g->nx - 1, 0}, cys[4] = {0, 0, g->ny - 1, g->ny - 1};
        for (int c = 0; c < 4; ++c) {
            fu[c] = au * (cxs[c] - px0) + bu * (cys[c] - py0) + H;
            fw[c] = aw * (cxs[c] - px0) + bw * (cys[c] - py0) + H;
        }
        long long so = 0, sa = 0;
        for (int k = 0; k < L.nw; ++k) {
            int lo, hi;
            needed_u_range(fu, fw, k, L.nu, lo, hi);
            ukr[(size_t)b * L.nw + k] = make_int2(lo, hi);
            if (hi > lo) {
                so += (long long)(hi - lo) * L.nv;
                sa += (long long)std::min(hi - lo + 2 * R, L.nu) * L.nv;
            }
        }
        cap_o = std::max(cap_o, so);
        cap_a = std::max(cap_a, sa);
    }

    if (cap_o >= (1LL << 31) || L.nv > 32767)
        return fail(PDRT_EINVAL, "grid too large for one control point's beam-frame region");
    pdrt_plan_t p = new pdrt_plan_s();
    p->grid = g;
    p->n_cp = n_cp;
    p->scratch_bytes = 0;
    PlanDev &P = p->dev;
    memset(&P, 0, sizeof(P));
    P.lat = L;
    P.mach = M;
    P.n_cp = n_cp;
    P.nx = g->nx; P.ny = g->ny; P.nz = g->nz;
    P.red = g->red;
    P.cap_o = cap_o;
    P.cap_a = cap_a;

    const size_t fixed = sizeof(float) * (M.corr ? 3 : 2) * (size_t)n_cp * L.nu * L.nv +
                         sizeof(SliceTab) * (size_t)n_cp * L.nw;
    size_t budget = scratch_budget_bytes;
    if (!budget) {   // default: a quarter of the free device memory, 1..4 GiB
        size_t free_b = 0, total_b = 0;
        CU_TRY(cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo");
        budget = std::min<size_t>(std::max<size_t>(free_b / 4, (size_t)1 << 30), (size_t)4 << 30);
    }
    const size_t per_cp = sizeof(float) * (size_t)(cap_o + cap_a);
    long long chunk = budget > fixed ? (long long)((budget - fixed) / per_cp) : 1;
    chunk = std::max(1LL, std::min<long long>(chunk, std::min(n_cp, kMaxCpPerChunk)));
    {   // equal passes: the same number of passes with the CPs spread evenly
        const long long passes = (n_cp + chunk - 1) / chunk;
        chunk = (n_cp + passes - 1) / passes;
    }
    p->chunk = (int)chunk;
    p->chunk_max = (int)chunk;

    cudaError_t e = cudaSuccess;
    float *lb = nullptr, *dd = nullptr;
    CpGeo *dgeo = nullptr;
    int2 *dukr = nullptr;
#define PLAN_TRY(expr, what)                      \
    do {                                          \
        e = (expr);                               \
        if (e != cudaSuccess) {                   \
            pdrt_status st_ = cuda_fail(e, what); \
            pdrt_plan_destroy(p);                 \
            return st_;                           \
        }                                         \
    } while (0)
    PLAN_TRY(dalloc(p, &lb, m->n_pairs + 1), "cudaMalloc(leaf bounds)");
    PLAN_TRY(dalloc(p, &dd, m->n_depth), "cudaMalloc(depth dose)");
    PLAN_TRY(dalloc(p, &dgeo, n_cp), "cudaMalloc(cp geometry)");
    PLAN_TRY(dalloc(p, &dukr, (size_t)n_cp * L.nw), "cudaMalloc(slice ranges)");
    PLAN_TRY(dalloc(p, &P.cptab, n_cp), "cudaMalloc(cp table)");
    PLAN_TRY(dalloc(p, &P.slices, (size_t)n_cp * L.nw), "cudaMalloc(slice table)");
    PLAN_TRY(dalloc(p, &P.gbox, (size_t)n_cp * L.nw), "cudaMalloc(gather boxes)");
    PLAN_TRY(dalloc(p, &P.fbuf, (size_t)n_cp * L.nu * L.nv), "cudaMalloc(fluence)");
    PLAN_TRY(dalloc(p, &P.gfbuf, (size_t)n_cp * L.nu * L.nv), "cudaMalloc(fluence adjoint)");
    if (M.corr) PLAN_TRY(dalloc(p, &P.tbuf, (size_t)n_cp * L.nu * L.nv), "cudaMalloc(raw fluence)");
    PLAN_TRY(dalloc(p, &P.region, (size_t)chunk * cap_o), "cudaMalloc(beam-frame region)");
    PLAN_TRY(dalloc(p, &P.adjbuf, (size_t)chunk * cap_a), "cudaMalloc(adjoint region)");
    PLAN_TRY(dalloc(p, &P.flags, 1), "cudaMalloc(flags)");
    PLAN_TRY(dalloc(p, &P.counters, 4 * (size_t)n_cp + 2), "cudaMalloc(counters)");
    PLAN_TRY(dalloc(p, &P.fft_ctr, 4 * (size_t)n_cp + 4), "cudaMalloc(fft counters)");
    PLAN_TRY(dalloc(p, &P.fft_over, (size_t)chunk * L.nw), "cudaMalloc(fft overflow list)");
    float *fcos = nullptr;
    PLAN_TRY(dalloc(p, &fcos, (size_t)conv_fft_cos_floats(M.R)), "cudaMalloc(fft cosine table)");
    P.fft_cos = fcos;
    std::vector<float> hcos(conv_fft_cos_floats(M.R));
    conv_fft_cos_table(M.R, hcos.data());
    P.leaf_bounds = lb;
    P.depth_dose = dd;
    P.cpgeo = dgeo;
    P.ukr = dukr;

    std::vector<float> hlb(m->n_pairs + 1), hdd(m->n_depth);
    for (int i = 0; i <= m->n_pairs; ++i) hlb[i] = (float)m->leaf_bounds_mm[i];
    for (int i = 0; i < m->n_depth; ++i) hdd[i] = (float)m->depth_dose[i];
    cudaStream_t s = (cudaStream_t)stream;
    PLAN_TRY(cudaMemcpyAsync(lb, hlb.data(), hlb.size() * sizeof(float), cudaMemcpyHostToDevice, s),
             "upload leaf bounds");
    PLAN_TRY(cudaMemcpyAsync(dd, hdd.data(), hdd.size() * sizeof(float), cudaMemcpyHostToDevice, s),
             "upload depth dose");
    PLAN_TRY(cudaMemcpyAsync(dgeo, geo.data(), geo.size() * sizeof(CpGeo), cudaMemcpyHostToDevice, s),
             "upload geometry");
    PLAN_TRY(cudaMemcpyAsync(dukr, ukr.data(), ukr.size() * sizeof(int2), cudaMemcpyHostToDevice, s),
             "upload slice ranges");
    PLAN_TRY(cudaMemcpyAsync(fcos, hcos.data(), hcos.size() * sizeof(float), cudaMemcpyHostToDevice, s),
             "upload fft cosine table");
    PLAN_TRY(cudaMemsetAsync(P.flags, 0, sizeof(unsigned), s), "clear flags");
    // host vectors go out of scope: wait for the copies
    PLAN_TRY(cudaStreamSynchronize(s), "plan upload sync");

    int bf = 1, ba = 1;
    PLAN_TRY(conv_prepare(M, &bf, &ba), "convolution kernel set-up");
    p->conv_blocks_fwd = std::max(1, bf) * g->sm_count;
    p->conv_blocks_adj = std::max(1, ba) * g->sm_count;
    // tensor-core convolution: phase depth and CTAs per SM per direction
    p->tc_blocks = 0;
    p->tc_blocks_adj = 0;
    P.tc_enabled = 0;
    {
        int bt_f = 0, bt_a = 0, ph_f = 1, ph_a = 1;
        PLAN_TRY(conv_tc_prepare(M.R, &bt_f, &bt_a, &ph_f, &ph_a), "tensor-core convolution set-up");
        if (bt_f > 0 && bt_a > 0) {
            p->tc_blocks = bt_f * g->sm_count;
            p->tc_blocks_adj = bt_a * g->sm_count;
            P.tc_phase[0] = ph_f;
            P.tc_phase[1] = ph_a;
            P.tc_enabled = 1;
        }
    }
    // FFT convolution: default size limit from the kernel radius (inputs up
    // to ~48 pixels wide fit; wider slices take the tensor-core path), raised
    // to the largest size with as many CTAs per SM (a larger limit only
    // changes the shared-memory layout, not a slice's work); needs the
    // tensor-core kernel for the overflow
    P.fft_pmax = 0;
    p->fft_blocks[0] = p->fft_blocks[1] = 0;
    if (P.tc_enabled) {
        const int want = fft_size_for(2 * M.R + 48) ? fft_size_for(2 * M.R + 48) : 192;
        const int sizes[16] = {192, 160, 144, 128, 120, 108, 100, 96, 90, 80, 72, 64, 60, 48, 40, 32};
        int base_f = 0, base_a = 0;
        for (int t = 0; t < 16 && !P.fft_pmax; ++t) {   // the base limit
            const int pm = sizes[t];
            if (pm > want || pm < 2 * M.R + 2) continue;
            PLAN_TRY(conv_fft_ctas(pm, M.R, false, &base_f), "fft convolution set-up");
            PLAN_TRY(conv_fft_ctas(pm, M.R, true, &base_a), "fft convolution set-up");
            if (base_f > 0 && base_a > 0) P.fft_pmax = pm;
        }
        for (int t = 0; t < 16 && P.fft_pmax && sizes[t] > P.fft_pmax; ++t) {   // as many CTAs
            int cf = 0, ca = 0;
            PLAN_TRY(conv_fft_ctas(sizes[t], M.R, false, &cf), "fft convolution set-up");
            PLAN_TRY(conv_fft_ctas(sizes[t], M.R, true, &ca), "fft convolution set-up");
            if (cf == base_f && ca == base_a) P.fft_pmax = sizes[t];
        }
        if (P.fft_pmax) {
            p->fft_blocks[0] = base_f * g->sm_count;
            p->fft_blocks[1] = base_a * g->sm_count;
        }
    }
    // the kernel-spectrum memo for the default size limit (off if it does
    // not fit in device memory: the FFT then computes every spectrum)
    if (P.fft_pmax && memo_alloc(p, P.fft_pmax) != cudaSuccess) cudaGetLastError();
#undef PLAN_TRY
    *out = p;
    return PDRT_OK;
}


static pdrt_status check_call(pdrt_grid_t g, pdrt_plan_t p)
{
    g_last_error.clear();
    if (!g || !p) return fail(PDRT_EINVAL, "NULL handle");
    if (p->grid != g) return fail(PDRT_EINVAL, "plan was uploaded for a different grid");
    int dev = 0;
    CU_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != g->device) return fail(PDRT_EINVAL, "current device differs from the grid's device");
    return PDRT_OK;
}

pdrt_status pdrt_dose_forward(pdrt_grid_t g, pdrt_plan_t p, const float *leaves_dev,
                              const float *jaws_dev, const float *mu_dev, float *dose_dev,
                              pdrt_stream_t stream)
{
    pdrt_status st = check_call(g, p);
    if (st != PDRT_OK) return st;
    if (!leaves_dev || !jaws_dev || !mu_dev || !dose_dev) return fail(PDRT_EINVAL, "NULL buffer");
    cudaStream_t s = (cudaStream_t)stream;
    const PlanDev &P = p->dev;
    CU_TRY(timed(p, K_RASTER, s, [&] { return launch_raster(P, leaves_dev, jaws_dev, mu_dev, s); }),
           "project_raster launch");
    CU_TRY(timed(p, K_TABLES, s, [&] { return launch_tables(P, s); }), "wepl_tables launch");
    const int n_chunks = (p->n_cp + p->chunk - 1) / p->chunk;
    CU_TRY(cudaMemsetAsync(P.counters, 0, sizeof(unsigned) * 4 * n_chunks, s), "clear counters");
    if (P.fft_pmax) CU_TRY(cudaMemsetAsync(P.fft_ctr, 0, sizeof(unsigned) * 4 * n_chunks, s), "clear counters");
    for (int c = 0; c < n_chunks; ++c) {
        const int b0 = c * p->chunk, nb = std::min(p->chunk, p->n_cp - b0);
        if (P.fft_pmax) {
            // FFT for the slices within the size limit (their kernel spectra
            // first, into the memo), tensor cores for the overflow list it
            // leaves
            unsigned int *fc = P.fft_ctr + 4 * c;
            CU_TRY(timed(p, K_CONV_FFT_FWD, s,
                         [&] {
                             const cudaError_t x = launch_spectrum(P, b0, nb, false, P.fft_pmax, s);
                             if (x != cudaSuccess) return x;
                             return launch_conv_fft(P, b0, nb, false, P.fft_pmax, fc, P.fft_over, fc + 1,
                                                    p->fft_blocks[0], s);
                         }),
                   "conv_forward_fft launch");
            CU_TRY(timed(p, K_CONV_TC_FWD, s,
                         [&] {
                             return launch_conv_tc(P, b0, nb, false, P.counters + 2 * n_chunks + c,
                                                   p->tc_blocks, s, P.fft_over, fc + 1);
                         }),
                   "conv_forward_tc launch");
        } else if (P.tc_enabled)
            CU_TRY(timed(p, K_CONV_TC_FWD, s,
                         [&] {
                             return launch_conv_tc(P, b0, nb, false, P.counters + 2 * n_chunks + c,
                                                   p->tc_blocks, s);
                         }),
                   "conv_forward_tc launch");
        // with tensor cores on, k_conv_tc takes every slice (tc_takes_slice)
        if (!P.tc_enabled)
            CU_TRY(timed(p, K_CONV_FWD, s,
                         [&] { return launch_conv(P, b0, nb, false, P.counters + c, p->conv_blocks_fwd, s); }),
                   "conv_forward launch");
        CU_TRY(timed(p, K_GATHER, s, [&] { return launch_gather(P, b0, nb, dose_dev, c == 0, s); }),
               "gather launch");
    }
    return PDRT_OK;
}

pdrt_status pdrt_dose_backward(pdrt_grid_t g, pdrt_plan_t p, const float *leaves_dev,
                               const float *jaws_dev, const float *mu_dev,
                               const float *dose_grad_dev, float *dleaves_dev, float *djaws_dev,
                               float *dmu_dev, pdrt_stream_t stream)
{
    pdrt_status st = check_call(g, p);
    if (st != PDRT_OK) return st;
    if (!leaves_dev || !jaws_dev || !mu_dev || !dose_grad_dev || !dleaves_dev || !djaws_dev ||
        !dmu_dev)
        return fail(PDRT_EINVAL, "NULL buffer");
    cudaStream_t s = (cudaStream_t)stream;
    const PlanDev &P = p->dev;
    CU_TRY(timed(p, K_RASTER, s, [&] { return launch_raster(P, leaves_dev, jaws_dev, mu_dev, s); }),
           "project_raster launch");
    CU_TRY(timed(p, K_TABLES, s, [&] { return launch_tables(P, s); }), "wepl_tables launch");
    const int n_chunks = (p->n_cp + p->chunk - 1) / p->chunk;
    unsigned int *ctr = P.counters + n_chunks;
    CU_TRY(cudaMemsetAsync(P.counters, 0, sizeof(unsigned) * 4 * n_chunks, s), "clear counters");
    if (P.fft_pmax) CU_TRY(cudaMemsetAsync(P.fft_ctr, 0, sizeof(unsigned) * 4 * n_chunks, s), "clear counters");
    for (int c = 0; c < n_chunks; ++c) {
        const int b0 = c * p->chunk, nb = std::min(p->chunk, p->n_cp - b0);
        // the gathered gradient h is formed by its own kernel (fusing the
        // gather into the tensor-core adjoint's operand build measured slower:
        // its few warps do not hide the gather's load latency)
        CU_TRY(timed(p, K_GATHER_T, s, [&] { return launch_gather_T(P, b0, nb, dose_grad_dev, s); }),
               "gather_transpose launch");
        if (P.fft_pmax) {
            unsigned int *fc = P.fft_ctr + 4 * c + 2;
            CU_TRY(timed(p, K_CONV_FFT_ADJ, s,
                         [&] {
                             const cudaError_t x = launch_spectrum(P, b0, nb, true, P.fft_pmax, s);
                             if (x != cudaSuccess) return x;
                             return launch_conv_fft(P, b0, nb, true, P.fft_pmax, fc, P.fft_over, fc + 1,
                                                    p->fft_blocks[1], s);
                         }),
                   "conv_adjoint_fft launch");
            CU_TRY(timed(p, K_CONV_TC_ADJ, s,
                         [&] {
                             return launch_conv_tc(P, b0, nb, true, P.counters + 3 * n_chunks + c,
                                                   p->tc_blocks_adj, s, P.fft_over, fc + 1);
                         }),
                   "conv_adjoint_tc launch");
        } else if (P.tc_enabled)
            CU_TRY(timed(p, K_CONV_TC_ADJ, s,
                         [&] {
                             return launch_conv_tc(P, b0, nb, true, P.counters + 3 * n_chunks + c,
                                                   p->tc_blocks_adj, s);
                         }),
                   "conv_adjoint_tc launch");
        else
            CU_TRY(timed(p, K_CONV_ADJ, s,
                         [&] { return launch_conv(P, b0, nb, true, ctr + c, p->conv_blocks_adj, s); }),
                   "conv_adjoint launch");
        CU_TRY(timed(p, K_MAG_T_GRAD, s, [&] { return launch_mag_T(P, b0, nb, s); }),
               "mag_transpose launch");
    }
    CU_TRY(timed(p, K_MAG_T_GRAD, s,
                 [&] {
                     return launch_param_grad(P, leaves_dev, jaws_dev, mu_dev, dleaves_dev, djaws_dev,
                                              dmu_dev, s);
                 }),
           "param_grad launch");
    return PDRT_OK;
}

pdrt_status pdrt_plan_set_tensor_cores(pdrt_plan_t p, int32_t enable)
{
    g_last_error.clear();
    if (!p) return fail(PDRT_EINVAL, "NULL plan");
    if (enable && p->tc_blocks <= 0)
        return fail(PDRT_EINVAL, "the tensor-core convolution does not fit this kernel radius");
    p->dev.tc_enabled = enable ? 1 : 0;
    if (!enable) p->dev.fft_pmax = 0;   // the FFT path hands its overflow to the tensor cores
    return PDRT_OK;
}

pdrt_status pdrt_plan_set_fft(pdrt_plan_t p, int32_t pmax)
{
    g_last_error.clear();
    if (!p) return fail(PDRT_EINVAL, "NULL plan");
    if (pmax == 0) {
        p->dev.fft_pmax = 0;
        return PDRT_OK;
    }
    if (!p->dev.tc_enabled)
        return fail(PDRT_EINVAL, "the FFT convolution needs the tensor-core path for its overflow");
    if (pmax < 0 || fft_size_for(pmax) != pmax)
        return fail(PDRT_EINVAL, "unsupported FFT size %d (32, 40, 48, 60, 64, 72, 80, 90, 96, 100, 108, 120, 128, 144, 160, 192)", pmax);
    if (pmax < 2 * p->dev.mach.R + 2)
        return fail(PDRT_EINVAL, "FFT size %d is below 2 R + 2 = %d for this kernel radius", pmax,
                    2 * p->dev.mach.R + 2);
    int cf = 0, ca = 0;
    CU_TRY(conv_fft_ctas(pmax, p->dev.mach.R, false, &cf), "fft convolution set-up");
    CU_TRY(conv_fft_ctas(pmax, p->dev.mach.R, true, &ca), "fft convolution set-up");
    if (cf <= 0 || ca <= 0) return fail(PDRT_EINVAL, "FFT size %d does not fit in shared memory", pmax);
    p->dev.fft_pmax = pmax;
    p->fft_blocks[0] = cf * p->grid->sm_count;
    p->fft_blocks[1] = ca * p->grid->sm_count;
    return PDRT_OK;
}

pdrt_status pdrt_plan_get_info(pdrt_plan_t p, pdrt_plan_info *out)
{
    g_last_error.clear();
    if (!p || !out) return fail(PDRT_EINVAL, "NULL argument");
    const Lattice &L = p->dev.lat;
    out->nu = L.nu; out->nv = L.nv; out->nw = L.nw;
    out->cu = L.cu; out->cv = L.cv; out->cw = L.cw;
    out->n_cp = p->n_cp;
    out->chunk_cp = p->chunk;
    out->scratch_bytes = p->scratch_bytes;
    out->tensor_cores = p->dev.tc_enabled;
    out->tc_ctas_per_sm[0] = p->grid->sm_count > 0 ? p->tc_blocks / p->grid->sm_count : 0;
    out->tc_ctas_per_sm[1] = p->grid->sm_count > 0 ? p->tc_blocks_adj / p->grid->sm_count : 0;
    out->simt_ctas_per_sm[0] = p->grid->sm_count > 0 ? p->conv_blocks_fwd / p->grid->sm_count : 0;
    out->simt_ctas_per_sm[1] = p->grid->sm_count > 0 ? p->conv_blocks_adj / p->grid->sm_count : 0;
    out->tc_phase[0] = p->dev.tc_phase[0];
    out->tc_phase[1] = p->dev.tc_phase[1];
    out->fft_pmax = p->dev.fft_pmax;
    out->fft_ctas_per_sm[0] = p->dev.fft_pmax && p->grid->sm_count > 0 ? p->fft_blocks[0] / p->grid->sm_count : 0;
    out->fft_ctas_per_sm[1] = p->dev.fft_pmax && p->grid->sm_count > 0 ? p->fft_blocks[1] / p->grid->sm_count : 0;
    out->spectrum_memo_pmax = p->dev.kf_pmax;
    out->spectrum_memo_bytes = p->memo_bytes;
    return PDRT_OK;
}

pdrt_status pdrt_plan_set_spectrum_memo(pdrt_plan_t p, int32_t enable)
{
    g_last_error.clear();
    if (!p) return fail(PDRT_EINVAL, "NULL plan");
    if (!enable) {
        memo_free(p);
        return PDRT_OK;
    }
    if (p->dev.kf_memo) return PDRT_OK;
    const int pmax = p->dev.fft_pmax ? p->dev.fft_pmax : 0;
    if (!pmax) return fail(PDRT_EINVAL, "the FFT convolution is off: no spectra to memoise");
    CU_TRY(memo_alloc(p, pmax), "cudaMalloc(spectrum memo)");
    return PDRT_OK;
}

pdrt_status pdrt_plan_reset_spectrum_memo(pdrt_plan_t p, pdrt_stream_t stream)
{
    g_last_error.clear();
    if (!p) return fail(PDRT_EINVAL, "NULL plan");
    if (!p->dev.kf_tag) return PDRT_OK;
    CU_TRY(cudaMemsetAsync(p->dev.kf_tag, 0, sizeof(int) * (size_t)p->n_cp * p->dev.lat.nw,
                           (cudaStream_t)stream),
           "clear spectrum memo");
    return PDRT_OK;
}

pdrt_status pdrt_plan_status(pdrt_plan_t p, pdrt_stream_t stream, uint32_t *flags_out)
{
    g_last_error.clear();
    if (!p || !flags_out) return fail(PDRT_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned int f = 0;
    CU_TRY(cudaStreamSynchronize(s), "stream sync");
    CU_TRY(cudaMemcpy(&f, p->dev.flags, sizeof(f), cudaMemcpyDeviceToHost), "read flags");
    CU_TRY(cudaMemset(p->dev.flags, 0, sizeof(f)), "clear flags");
    *flags_out = f;
    return PDRT_OK;
}

pdrt_status pdrt_plan_work(pdrt_plan_t p, pdrt_stream_t stream, pdrt_work *out)
{
    g_last_error.clear();
    if (!p || !out) return fail(PDRT_EINVAL, "NULL argument");
    CU_TRY(cudaStreamSynchronize((cudaStream_t)stream), "stream sync");
    std::vector<CpTab> t(p->n_cp);
    CU_TRY(cudaMemcpy(t.data(), p->dev.cptab, sizeof(CpTab) * p->n_cp, cudaMemcpyDeviceToHost),
           "read work counters");
    memset(out, 0, sizeof(*out));
    for (const CpTab &c : t) {
        out->active_slices += c.n_active;
        out->support_points += c.n_support;
        out->region_points += c.n_region;
    }
    const long long n = 2LL * p->dev.mach.R + 1;
    out->taps = n * n;
    out->conv_flops = 2.0 * (double)out->taps * (double)out->support_points;
    out->mma_flops = 0.0;
    out->fft_flops = 0.0;
    if (p->dev.tc_enabled) {
        // replay the tensor-core tiling of k_conv_tc (row tiles of 128 rows
        // with a last tile of at most 64 rows as M = 64, column tiles, input
        // chunks)
        const Lattice &L = p->dev.lat;
        const int R = p->dev.mach.R;
        std::vector<SliceTab> sl((size_t)p->n_cp * L.nw);
        CU_TRY(cudaMemcpy(sl.data(), p->dev.slices, sizeof(SliceTab) * sl.size(), cudaMemcpyDeviceToHost),
               "read slice tables");
        for (const SliceTab &st : sl) {
            int fpu = 0, fpv = 0;   // the forward's padded sizes (its spectrum)
            fft_slice_sizes(st, false, R, fpu, fpv);
            for (int adj = 0; adj < 2; ++adj) {
                if (p->dev.fft_pmax) {
                    int pu = 0, pv = 0;
                    fft_slice_sizes(st, adj != 0, R, pu, pv);
                    if (pu == 0) continue;
                    if (pu <= p->dev.fft_pmax && pv <= p->dev.fft_pmax) {
                        const double n = (double)pu * pv, hu1 = pu / 2 + 1, kv1 = pv / 2 + 1;
                        // the spectrum once per call and size: the adjoint
                        // takes the forward's from the memo when it pads alike
                        const bool memo_hit = adj && p->dev.kf_memo && pu == fpu && pv == fpv &&
                                              pu <= p->dev.kf_pmax && pv <= p->dev.kf_pmax;
                        out->fft_flops += 2.0 * 2.5 * n * log2(n) + 2.0 * pv * hu1;
                        if (!memo_hit)
                            out->fft_flops += 2.0 * (R + 1) * (R + 1) * kv1 + 2.0 * (R + 1) * kv1 * hu1;
                        out->fft_slices += 1;
                        continue;
                    }
                    out->tc_slices += 1;
                }
                const int ii0 = adj ? st.oi0 : st.pi0, ii1 = adj ? st.oi1 : st.pi1;
                const int ij0 = adj ? st.oj0 : st.pj0, ij1 = adj ? st.oj1 : st.pj1;
                const int oi0 = adj ? st.ai0 : st.oi0, oi1 = adj ? st.ai1 : st.oi1;
                const int oj0 = adj ? st.aj0 : st.oj0, oj1 = adj ? st.aj1 : st.oj1;
                if (oi1 <= oi0 || oj1 <= oj0) continue;
                if (ii1 <= ii0 || ij1 <= ij0) continue;
                const int maxn = adj ? kTcAdjMaxN : kTcFwdMaxN, maxk = adj ? kTcAdjMaxK : kTcFwdMaxK;
                // rows of all M tiles of the box: 128 per full tile, and 64 or
                // 128 for the last one
                const int h = oi1 - oi0, full = (h - 1) / 128, last = h - 128 * full;
                const double m_rows = 128.0 * full + (last <= 64 ? 64.0 : 128.0);
                const int ow = oj1 - oj0, n_ct = (ow + maxn - 1) / maxn;
                const int w_ct = (((ow + n_ct - 1) / n_ct) + 15) & ~15;
                for (int ct = 0; ct < n_ct; ++ct) {
                    const int j0 = oj0 + ct * w_ct, j1 = std::min(oj1, j0 + w_ct);
                    const int nt = ((j1 - j0) + 15) & ~15;
                    const int sa = std::max(ij0, j0 - R), sb = std::min(ij1, j0 + nt + R);
                    const int n_kc = sb > sa ? (sb - sa + maxk - 1) / maxk : 0;
                    const int w_kc = n_kc ? (((sb - sa + n_kc - 1) / n_kc) + 15) & ~15 : 16;
                    for (int kc = 0; kc < n_kc; ++kc) {
                        const int ka = sa + kc * w_kc, kb = std::min(sb, ka + w_kc);
                        const int kt = ((kb - ka) + 15) & ~15;
                        out->mma_flops += m_rows * (2 * R + 1) * (kt / 16) * 3 * 2.0 * nt * 16;
                    }
                }
            }
        }
    }
    return PDRT_OK;
}

pdrt_status pdrt_profile_enable(pdrt_plan_t p, int32_t enable)
{
    g_last_error.clear();
    if (!p) return fail(PDRT_EINVAL, "NULL plan");
    if (enable && p->events.empty()) {
        p->events.resize(16384);
        for (auto &e : p->events) CU_TRY(cudaEventCreate(&e), "cudaEventCreate");
    }
    p->profiling = enable != 0;
    if (enable) {
        p->recs.clear();
        p->next_ev = 0;
        p->overflow = false;
    }
    return PDRT_OK;
}

pdrt_status pdrt_profile_read(pdrt_plan_t p, pdrt_stream_t stream, pdrt_profile *out)
{
    g_last_error.clear();
    if (!p || !out) return fail(PDRT_EINVAL, "NULL argument");
    CU_TRY(cudaStreamSynchronize((cudaStream_t)stream), "stream sync");
    memset(out, 0, sizeof(*out));
    for (int k = 0; k < PDRT_NUM_KERNELS; ++k) out->name[k] = kKernelNames[k];
    for (const ProfileRec &r : p->recs) {
        float ms = 0.f;
        CU_TRY(cudaEventElapsedTime(&ms, p->events[r.ev], p->events[r.ev + 1]), "cudaEventElapsedTime");
        out->launches[r.kid] += 1;
        out->total_ms[r.kid] += ms;
    }
    out->overflow = p->overflow ? 1 : 0;
    return PDRT_OK;
}


pdrt_status pdrt_plan_set_chunk(pdrt_plan_t p, int32_t chunk_cp)
{
    g_last_error.clear();
    if (!p) return fail(PDRT_EINVAL, "NULL plan");
    if (chunk_cp < 1 || chunk_cp > p->chunk_max)
        return fail(PDRT_EINVAL, "chunk must be in 1..%d (the scratch bound)", p->chunk_max);
    p->chunk = chunk_cp;
    return PDRT_OK;
}

pdrt_status pdrt_plan_set_tc_phase(pdrt_plan_t p, int32_t phase_forward, int32_t phase_adjoint)
{
    g_last_error.clear();
    if (!p) return fail(PDRT_EINVAL, "NULL plan");
    if (p->tc_blocks <= 0) return fail(PDRT_EINVAL, "tensor-core path unavailable for this plan");
    int nf = 0, na = 0;
    CU_TRY(conv_tc_ctas(p->dev.mach.R, false, phase_forward, &nf), "tensor-core occupancy");
    CU_TRY(conv_tc_ctas(p->dev.mach.R, true, phase_adjoint, &na), "tensor-core occupancy");
    if (phase_forward > 4 || phase_adjoint > 4 || nf < 1 || na < 1)
        return fail(PDRT_EINVAL, "phase depths must be in 1..4 and fit in shared memory");
    p->dev.tc_phase[0] = phase_forward;
    p->dev.tc_phase[1] = phase_adjoint;
    p->tc_blocks = nf * p->grid->sm_count;
    p->tc_blocks_adj = na * p->grid->sm_count;
    return PDRT_OK;
}

pdrt_status pdrt_plan_autotune(pdrt_grid_t g, pdrt_plan_t p, const float *leaves_dev,
                               const float *jaws_dev, const float *mu_dev, float *dose_dev,
                               const float *dose_grad_dev, float *dleaves_dev, float *djaws_dev,
                               float *dmu_dev, pdrt_stream_t stream, pdrt_tune_result *out)
{
    pdrt_status st = check_call(g, p);
    if (st != PDRT_OK) return st;
    if (!out || !dose_dev) return fail(PDRT_EINVAL, "NULL argument");
    if (dose_grad_dev && (!dleaves_dev || !djaws_dev || !dmu_dev))
        return fail(PDRT_EINVAL, "adjoint outputs are NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const bool prof = p->profiling;
    p->profiling = false;
    const int sm = g->sm_count, R = p->dev.mach.R;
    struct Sched {
        int tc, chunk, ph_f, ph_a, fft;
    };
    const bool tc_ok = p->tc_blocks > 0;
    const Sched start = {p->dev.tc_enabled, p->chunk, p->dev.tc_phase[0], p->dev.tc_phase[1], p->dev.fft_pmax};
    int ctas_f = tc_ok ? p->tc_blocks / sm : 0, ctas_a = tc_ok ? p->tc_blocks_adj / sm : 0;
    // FFT size limits that fit (each with its CTAs per SM)
    std::vector<int> fft_ok;
    if (tc_ok)
        for (int pm : {32, 40, 48, 60, 64, 72, 80, 90, 96, 100, 108, 120, 128, 144, 160, 192}) {
            if (pm < 2 * R + 2) continue;
            int cf = 0, ca = 0;
            CU_TRY(conv_fft_ctas(pm, R, false, &cf), "fft occupancy");
            CU_TRY(conv_fft_ctas(pm, R, true, &ca), "fft occupancy");
            if (cf > 0 && ca > 0) fft_ok.push_back(pm);
        }
    auto apply = [&](const Sched &c) -> pdrt_status {
        p->dev.tc_enabled = c.tc;
        p->chunk = c.chunk;
        p->dev.fft_pmax = 0;
        if (c.fft && c.tc) {
            int cf = 0, ca = 0;
            CU_TRY(conv_fft_ctas(c.fft, R, false, &cf), "fft occupancy");
            CU_TRY(conv_fft_ctas(c.fft, R, true, &ca), "fft occupancy");
            p->dev.fft_pmax = c.fft;
            p->fft_blocks[0] = cf * sm;
            p->fft_blocks[1] = ca * sm;
        }
        if (tc_ok) {
            int nf = 0, na = 0;
            CU_TRY(conv_tc_ctas(R, false, c.ph_f, &nf), "tensor-core occupancy");
            CU_TRY(conv_tc_ctas(R, true, c.ph_a, &na), "tensor-core occupancy");
            p->dev.tc_phase[0] = c.ph_f;
            p->dev.tc_phase[1] = c.ph_a;
            p->tc_blocks = nf * sm;
            p->tc_blocks_adj = na * sm;
            ctas_f = nf;
            ctas_a = na;
        }
        return PDRT_OK;
    };
    cudaEvent_t e0, e1;
    CU_TRY(cudaEventCreate(&e0), "cudaEventCreate");
    CU_TRY(cudaEventCreate(&e1), "cudaEventCreate");
    int n_timed = 0;
    auto time_of = [&](const Sched &c, float *ms) -> pdrt_status {
        pdrt_status r = apply(c);
        if (r != PDRT_OK) return r;
        auto pass = [&]() -> pdrt_status {
            pdrt_status q = pdrt_dose_forward(g, p, leaves_dev, jaws_dev, mu_dev, dose_dev, stream);
            if (q == PDRT_OK && dose_grad_dev)
                q = pdrt_dose_backward(g, p, leaves_dev, jaws_dev, mu_dev, dose_grad_dev, dleaves_dev,
                                       djaws_dev, dmu_dev, stream);
            return q;
        };
        if ((r = pass()) != PDRT_OK) return r;   // warm-up
        cudaEventRecord(e0, s);
        for (int k = 0; k < 2 && r == PDRT_OK; ++k) r = pass();
        cudaEventRecord(e1, s);
        if (r != PDRT_OK) return r;
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
        if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
        *ms *= 0.5f;
        ++n_timed;
        return PDRT_OK;
    };
    Sched best = start;
    float best_ms = 1e30f;
    pdrt_status rst = time_of(best, &best_ms);
    auto consider = [&](const Sched &c) {
        if (rst != PDRT_OK) return;
        float ms = 0.f;
        rst = time_of(c, &ms);
        if (rst == PDRT_OK && ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    };
    // 1) convolution path: FFT (+ tensor-core overflow), tensor cores alone,
    //    FP32 SIMT; then the FFT size limit
    if (tc_ok) {
        const Sched cand[3] = {{1, best.chunk, best.ph_f, best.ph_a, fft_ok.empty() ? 0 : best.fft},
                               {1, best.chunk, best.ph_f, best.ph_a, 0},
                               {0, best.chunk, best.ph_f, best.ph_a, 0}};
        if (!best.fft && !fft_ok.empty()) {
            Sched c = best;
            c.tc = 1;
            c.fft = fft_ok[0];
            for (int pm : fft_ok)
                if (pm <= fft_size_for(2 * R + 48)) c.fft = pm;
            consider(c);
        }
        for (const Sched &c : cand)
            if (c.tc != best.tc || c.fft != best.fft) consider(c);
        if (best.fft) {
            const int cur = best.fft;
            for (int pm : fft_ok)
                if (pm != cur) {
                    Sched c = best;
                    c.fft = pm;
                    consider(c);
                }
        }
    }
    // 2) tensor-core tile shape per direction (phase depths that fit)
    if (tc_ok && best.tc) {
        for (int dir = 0; dir < 2; ++dir)
            for (int ph = 1; ph <= 4; ++ph) {
                if (ph == (dir ? best.ph_a : best.ph_f)) continue;
                int n = 0;
                if (conv_tc_ctas(R, dir == 1, ph, &n) != cudaSuccess || n < 1) continue;
                Sched c = best;
                (dir ? c.ph_a : c.ph_f) = ph;
                consider(c);
            }
    }
    // 3) control points per pass
    for (int ch : {p->chunk_max, (p->chunk_max + 1) / 2, (p->chunk_max + 3) / 4}) {
        if (ch < 1 || ch == best.chunk) continue;
        Sched c = best;
        c.chunk = ch;
        consider(c);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    pdrt_status ra = apply(rst == PDRT_OK ? best : start);
    p->profiling = prof;
    if (rst != PDRT_OK) return rst;
    if (ra != PDRT_OK) return ra;
    out->tensor_cores = best.tc;
    out->chunk_cp = best.chunk;
    out->best_ms = best_ms;
    out->n_candidates = n_timed;
    out->phase[0] = best.ph_f;
    out->phase[1] = best.ph_a;
    out->tc_ctas_per_sm[0] = ctas_f;
    out->tc_ctas_per_sm[1] = ctas_a;
    out->fft_pmax = best.tc ? best.fft : 0;
    return PDRT_OK;
}

}  // extern "C"

struct pdrt_batch_s {
    int n = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaStream_t> branches;   // [0] origin (recording), [1 .. nbr] branches
    std::vector<cudaEvent_t> events;      // [0] fork, [1 .. nbr] joins (graph edges only)
    std::vector<cudaEvent_t> marks;       // [0] start, [1 .. n] plan done (event-record nodes)
    long long kernels = 0;
    std::vector<int> pass_cp;             // control points per pass of each plan
    unsigned int *d_ctr = nullptr;        // work counters of the batched FFT launches
};

static void batch_free(pdrt_batch_t b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaEvent_t e : b->events) cudaEventDestroy(e);
    for (cudaEvent_t e : b->marks) cudaEventDestroy(e);
    for (cudaStream_t s : b->branches) cudaStreamDestroy(s);
    cudaFree(b->d_ctr);
    delete b;
}

extern "C" {

pdrt_status pdrt_batch_create(pdrt_batch_t *out, int32_t n, const pdrt_grid_t *grids,
                              const pdrt_plan_t *plans, const float *const *leaves_dev,
                              const float *const *jaws_dev, const float *const *mu_dev,
                              float *const *dose_dev, const float *const *dose_grad_dev,
                              float *const *dleaves_dev, float *const *djaws_dev,
                              float *const *dmu_dev, int32_t n_branches, pdrt_stream_t stream)
{
    g_last_error.clear();
    if (!out || !grids || !plans || !leaves_dev || !jaws_dev || !mu_dev || !dose_dev)
        return fail(PDRT_EINVAL, "NULL argument");
    *out = nullptr;
    if (n < 1) return fail(PDRT_EINVAL, "empty batch");
    for (int i = 0; i < n; ++i) {
        if (!plans[i] || !grids[i] || plans[i]->grid != grids[i])
            return fail(PDRT_EINVAL, "plan %d missing or uploaded for another grid", i);
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return fail(PDRT_EINVAL, "plan %d appears twice", i);
        if (!leaves_dev[i] || !jaws_dev[i] || !mu_dev[i] || !dose_dev[i])
            return fail(PDRT_EINVAL, "a buffer of plan %d is NULL", i);
        if (grids[i]->device != grids[0]->device) return fail(PDRT_EINVAL, "plans on different devices");
        if (dose_grad_dev && dose_grad_dev[i] &&
            (!dleaves_dev || !djaws_dev || !dmu_dev || !dleaves_dev[i] || !djaws_dev[i] || !dmu_dev[i]))
            return fail(PDRT_EINVAL, "adjoint outputs of plan %d are NULL", i);
    }
    int dev = 0;
    CU_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != grids[0]->device) return fail(PDRT_EINVAL, "current device differs from the plans' device");
    const int nbr = std::max(1, std::min<int>(n_branches, n));
    const int sm = grids[0]->sm_count;
    (void)stream;   // recording uses an internal origin stream (the caller's may be the legacy one)

    // the shared FFT launch is sized for the largest size limit and kernel
    // radius of the batch; if that does not fit in shared memory every FFT
    // plan keeps its own launches
    int pmax_l = 0, r_l = 0;
    for (int i = 0; i < n; ++i)
        if (plans[i]->dev.fft_pmax > 0) {
            pmax_l = std::max(pmax_l, plans[i]->dev.fft_pmax);
            r_l = std::max(r_l, plans[i]->dev.mach.R);
        }
    int fft_grid[2] = {0, 0};
    if (pmax_l) {
        CU_TRY(conv_fft_ctas(pmax_l, r_l, false, &fft_grid[0]), "fft convolution set-up");
        CU_TRY(conv_fft_ctas(pmax_l, r_l, true, &fft_grid[1]), "fft convolution set-up");
        if (fft_grid[0] <= 0 || fft_grid[1] <= 0) fft_grid[0] = fft_grid[1] = 0;
    }
    const int fft_smem = pmax_l ? conv_fft_smem_bytes(pmax_l, r_l) : 0;
    std::vector<int> nch(n);
    std::vector<bool> adj(n), shared(n);
    int rounds = 0;
    for (int i = 0; i < n; ++i) {
        nch[i] = (plans[i]->n_cp + plans[i]->chunk - 1) / plans[i]->chunk;
        adj[i] = dose_grad_dev && dose_grad_dev[i];
        shared[i] = plans[i]->dev.fft_pmax > 0 && fft_grid[0] > 0;
        rounds = std::max(rounds, nch[i]);
    }
    // entries of the shared FFT launch of round c, direction d: pass c of
    // every FFT plan that has one; counters: one per launch group
    std::vector<std::vector<FftPlan>> ent_p(2 * rounds);
    std::vector<std::vector<int4>> ent_r(2 * rounds);
    std::vector<int> ctr0(2 * rounds);
    int n_ctr = 0;
    for (int d = 0; d < 2; ++d)
        for (int c = 0; c < rounds; ++c) {
            const int r = d * rounds + c;
            for (int i = 0; i < n; ++i) {
                if (!shared[i] || c >= nch[i] || (d == 1 && !adj[i])) continue;
                const int b0 = c * plans[i]->chunk, nb = std::min(plans[i]->chunk, plans[i]->n_cp - b0);
                ent_p[r].push_back(fft_plan_of(plans[i]->dev));
                ent_r[r].push_back(make_int4(b0, nb, 0, c));
            }
            ctr0[r] = n_ctr;
            n_ctr += ((int)ent_p[r].size() + kFftBatchMax - 1) / kFftBatchMax;
        }
    pdrt_batch_t b = new pdrt_batch_s();
    b->n = n;
    for (int i = 0; i < n; ++i) b->pass_cp.push_back(plans[i]->chunk);
    cudaError_t e = cudaMalloc(&b->d_ctr, sizeof(unsigned) * std::max(n_ctr, 1));
    cudaStream_t s = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->branches.push_back(s);
    for (int k = 0; k < nbr && e == cudaSuccess; ++k) {
        cudaStream_t bs;
        e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
        if (e == cudaSuccess) b->branches.push_back(bs);
    }
    for (int k = 0; k < 1 + nbr && e == cudaSuccess; ++k) {
        cudaEvent_t x;
        e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
        if (e == cudaSuccess) b->events.push_back(x);
    }
    for (int k = 0; k < 1 + n && e == cudaSuccess; ++k) {
        cudaEvent_t x;
        e = cudaEventCreate(&x);
        if (e == cudaSuccess) b->marks.push_back(x);
    }
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, "batch set-up");
    }
    // plans to branches, balanced by a work estimate (control points x voxels)
    std::vector<int> owner(n);
    {
        std::vector<int> order(n);
        std::vector<double> load(nbr, 0.0);
        for (int i = 0; i < n; ++i) order[i] = i;
        auto cost = [&](int i) { return (double)plans[i]->n_cp * grids[i]->nx * grids[i]->ny * grids[i]->nz; };
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
        for (int i : order) {
            const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            owner[i] = k;
            load[k] += cost(i);
        }
    }
    std::vector<bool> prof(n);
    for (int i = 0; i < n; ++i) {
        prof[i] = plans[i]->profiling;
        plans[i]->profiling = false;
    }
    auto chk = [&](cudaError_t x) {
        if (x != cudaSuccess && e == cudaSuccess) e = x;
    };
    auto bstream = [&](int i) { return b->branches[1 + owner[i]]; };
    auto fork = [&]() {
        cudaEventRecord(b->events[0], s);
        for (int k = 0; k < nbr; ++k) cudaStreamWaitEvent(b->branches[1 + k], b->events[0], 0);
    };
    auto join = [&]() {
        for (int k = 0; k < nbr; ++k) {
            cudaEventRecord(b->events[1 + k], b->branches[1 + k]);
            cudaStreamWaitEvent(s, b->events[1 + k], 0);
        }
    };
    // the convolution of pass c of plan i beside the shared FFT launch: the
    // tensor-core pass over its overflow list, or (a plan off the shared
    // launch) its own FFT + overflow, tensor-core or SIMT convolution
    auto conv_rest = [&](int i, int c, bool ad) -> cudaError_t {
        pdrt_plan_t p = plans[i];
        const PlanDev &P = p->dev;
        const int b0 = c * p->chunk, nb = std::min(p->chunk, p->n_cp - b0), nc = nch[i];
        cudaStream_t bs = bstream(i);
        unsigned int *fc = P.fft_ctr + 4 * c + (ad ? 2 : 0);
        if (P.fft_pmax && !shared[i]) {
            const cudaError_t x = launch_conv_fft(P, b0, nb, ad, P.fft_pmax, fc, P.fft_over, fc + 1,
                                                  p->fft_blocks[ad ? 1 : 0], bs);
            if (x != cudaSuccess) return x;
        }
        if (P.fft_pmax)
            return launch_conv_tc(P, b0, nb, ad, P.counters + (ad ? 3 : 2) * nc + c,
                                  ad ? p->tc_blocks_adj : p->tc_blocks, bs, P.fft_over, fc + 1);
        if (P.tc_enabled)
            return launch_conv_tc(P, b0, nb, ad, P.counters + (ad ? 3 : 2) * nc + c,
                                  ad ? p->tc_blocks_adj : p->tc_blocks, bs);
        return launch_conv(P, b0, nb, ad, P.counters + (ad ? nc : 0) + c,
                           ad ? p->conv_blocks_adj : p->conv_blocks_fwd, bs);
    };
    auto fft_round = [&](int d, int c) {
        const int r = d * rounds + c;
        if (!ent_p[r].empty())
            chk(launch_conv_fft_multi(ent_p[r].data(), ent_r[r].data(), (int)ent_p[r].size(), pmax_l, fft_smem,
                                      fft_grid[d] * sm, d == 1, b->d_ctr + ctr0[r], s));
    };
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaEventRecordWithFlags(b->marks[0], s, cudaEventRecordExternal);
        cudaMemsetAsync(b->d_ctr, 0, sizeof(unsigned) * std::max(n_ctr, 1), s);
        // counters, projection, fluence and slice tables of every plan (the
        // adjoint of the same parameters reuses them)
        fork();
        for (int i = 0; i < n; ++i) {
            const PlanDev &P = plans[i]->dev;
            cudaMemsetAsync(P.counters, 0, sizeof(unsigned) * 4 * nch[i], bstream(i));
            cudaMemsetAsync(P.fft_ctr, 0, sizeof(unsigned) * 4 * nch[i], bstream(i));
            chk(launch_raster(P, leaves_dev[i], jaws_dev[i], mu_dev[i], bstream(i)));
            chk(launch_tables(P, bstream(i)));
            // the forward's kernel spectra of every control point into the
            // plan's memo (no-op without one): the FFT rounds take them
            if (P.fft_pmax) chk(launch_spectrum(P, 0, plans[i]->n_cp, false, P.fft_pmax, bstream(i)));
        }
        join();
        // forward: per round the shared FFT launch over pass c of every FFT
        // plan, then per plan on its branch the rest of its convolution, then
        // one shared gather launch over pass c of every plan
        std::vector<GatherEntry> gents;
        auto gather_round = [&](int c, bool transpose) {
            gents.clear();
            for (int i = 0; i < n; ++i) {
                if (c >= nch[i] || (transpose && !adj[i])) continue;
                pdrt_plan_t p = plans[i];
                GatherEntry E;
                memset(&E, 0, sizeof(E));
                E.p = gather_plan_of(p->dev);
                E.b0 = c * p->chunk;
                E.nb = std::min(p->chunk, p->n_cp - E.b0);
                E.first = c == 0;
                E.dose = dose_dev[i];
                E.gd = transpose ? dose_grad_dev[i] : nullptr;
                gents.push_back(E);
            }
            if (!gents.empty()) chk(launch_gather_multi(gents.data(), (int)gents.size(), transpose, s));
        };
        for (int c = 0; c < rounds; ++c) {
            fft_round(0, c);
            fork();
            for (int i = 0; i < n; ++i) {
                if (c >= nch[i]) continue;
                chk(conv_rest(i, c, false));
            }
            join();
            gather_round(c, false);
            for (int i = 0; i < n; ++i)
                if (c == nch[i] - 1 && !adj[i]) cudaEventRecordWithFlags(b->marks[1 + i], s, cudaEventRecordExternal);
        }
        // adjoint in the same rounds: shared gradient-gather launch, shared
        // FFT launch, overflow and transposed magnification per plan
        for (int c = 0; c < rounds; ++c) {
            gather_round(c, true);
            fft_round(1, c);
            fork();
            for (int i = 0; i < n; ++i) {
                if (!adj[i] || c >= nch[i]) continue;
                pdrt_plan_t p = plans[i];
                const int b0 = c * p->chunk, nb = std::min(p->chunk, p->n_cp - b0);
                chk(conv_rest(i, c, true));
                chk(launch_mag_T(p->dev, b0, nb, bstream(i)));
            }
            join();
        }
        fork();
        for (int i = 0; i < n; ++i) {
            if (!adj[i]) continue;
            chk(launch_param_grad(plans[i]->dev, leaves_dev[i], jaws_dev[i], mu_dev[i], dleaves_dev[i],
                                  djaws_dev[i], dmu_dev[i], bstream(i)));
            cudaEventRecordWithFlags(b->marks[1 + i], bstream(i), cudaEventRecordExternal);
        }
        join();
        cudaError_t e2 = cudaStreamEndCapture(s, &b->graph);
        if (e == cudaSuccess) e = e2;
    }
    for (int i = 0; i < n; ++i) plans[i]->profiling = prof[i];
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e == cudaSuccess) {
        size_t nn = 0;
        e = cudaGraphGetNodes(b->graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (e == cudaSuccess && nn) e = cudaGraphGetNodes(b->graph, nodes.data(), &nn);
        for (size_t q = 0; q < nn && e == cudaSuccess; ++q) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nodes[q], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
                ++b->kernels;
        }
    }
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, "batch graph recording");
    }
    *out = b;
    return PDRT_OK;
}

pdrt_status pdrt_batch_launch(pdrt_batch_t b, pdrt_stream_t stream)
{
    g_last_error.clear();
    if (!b || !b->exec) return fail(PDRT_EINVAL, "NULL batch");
    CU_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream), "cudaGraphLaunch");
    g_launches.fetch_add(b->kernels);
    return PDRT_OK;
}

pdrt_status pdrt_batch_plan_times(pdrt_batch_t b, pdrt_stream_t stream, float *ms_out)
{
    g_last_error.clear();
    if (!b || !ms_out) return fail(PDRT_EINVAL, "NULL argument");
    CU_TRY(cudaStreamSynchronize((cudaStream_t)stream), "stream sync");
    for (int i = 0; i < b->n; ++i)
        CU_TRY(cudaEventElapsedTime(&ms_out[i], b->marks[0], b->marks[1 + i]), "cudaEventElapsedTime");
    return PDRT_OK;
}

int64_t pdrt_batch_kernels(pdrt_batch_t b) { return b ? b->kernels : 0; }

int32_t pdrt_batch_pass_cp(pdrt_batch_t b, int32_t i)
{
    return b && i >= 0 && i < b->n ? b->pass_cp[i] : 0;
}

void pdrt_batch_destroy(pdrt_batch_t b) { batch_free(b); }

}  // extern "C"
