// pdrt_cp_dose_static: forward dose of ONE control point that allocates no
// device memory.  Everything the pass needs beyond the caller's input and
// output buffers (fluence map, slice tables, beam-frame dose region, counters)
// lives in one file-scope device array, g_static_scratch, of fixed size.
//
// Who needs this: callers that cannot call cudaMalloc -- e.g. a plug-in hosted
// by a framework that owns all device memory and hands it only input and
// output buffers, or a latency-critical loop that must never enter the CUDA
// allocator (cudaMalloc/cudaFree can synchronise the device and can fail when
// memory is fragmented).  pdrt_grid_create/pdrt_plan_upload allocate, so they
// are not available to such callers; this entry point takes the density grid
// and the beam model directly.
//
// The array is held by every GPU that loads the library until the process
// exits.  Its device address is obtained once per device with
// cudaGetSymbolAddress on the first call made with that device current.
// Every call shares the array and it keeps the previous call's contents: the
// counters and flags are cleared at the start of each call, and calls that
// can overlap on the GPU (two streams, two host threads) race on it.  The
// call is synchronous: it copies pageable host tables to the array,
// synchronises the stream and reads the device flags back before returning,
// so none of its calls can be recorded into a stream capture.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "pdrt_impl.cuh"

using namespace pdrt;

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[PDRT_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_conv_ready[kMaxDevices] = {};   // bit q: conv variant nq4 == q prepared
int g_conv_blocks[kMaxDevices][64] = {};

pdrt_status err(pdrt_status st, const std::string &m)
{
    internal_set_error(m.c_str());
    return st;
}

pdrt_status cuda_err(cudaError_t e, const char *what)
{
    return err(PDRT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" pdrt_status pdrt_cp_dose_static(const float *red_dev, int32_t nx, int32_t ny, int32_t nz,
                                           double sx, double sy, double sz,
                                           const double origin_mm[3], const double iso_mm[3],
                                           double gantry_deg, const pdrt_machine *m,
                                           const float *leaves_dev, const float *jaws_dev,
                                           const float *mu_dev, float *dose_dev,
                                           pdrt_stream_t stream)
{
    internal_set_error("");
    if (!red_dev || !origin_mm || !iso_mm || !m || !leaves_dev || !jaws_dev || !mu_dev || !dose_dev)
        return err(PDRT_EINVAL, "NULL argument");
    if (nx <= 0 || ny <= 0 || nz <= 0) return err(PDRT_ESHAPE, "grid dimensions must be positive");
    if (!(sx > 0) || !(sy > 0) || !(sz > 0) || !std::isfinite(sx) || !std::isfinite(sz))
        return err(PDRT_EINVAL, "voxel spacing must be positive and finite");
    if (fabs(sx - sy) > 1e-6 * sx) return err(PDRT_EINVAL, "sx must equal sy");
    if (!std::isfinite(gantry_deg)) return err(PDRT_EINVAL, "gantry angle is not finite");
    for (int d = 0; d < 3; ++d)
        if (!std::isfinite(origin_mm[d]) || !std::isfinite(iso_mm[d]))
            return err(PDRT_EINVAL, "origin and isocentre must be finite");
    if (m->n_pairs < 1 || m->n_pairs > PDRT_MAX_PAIRS) return err(PDRT_EINVAL, "bad n_pairs");
    for (int i = 1; i <= m->n_pairs; ++i)
        if (!(m->leaf_bounds_mm[i] > m->leaf_bounds_mm[i - 1]))
            return err(PDRT_EINVAL, "leaf bounds must be strictly ascending");
    if (m->kernel_radius_px < 0 || m->kernel_radius_px > PDRT_MAX_RADIUS_PX)
        return err(PDRT_EINVAL, "kernel radius out of range");
    if (m->n_depth < 2 || m->n_depth > PDRT_MAX_DEPTH_TABLE || !(m->depth_step_mm > 0))
        return err(PDRT_EINVAL, "bad depth-dose table");
    if (!(m->tau >= 0 && m->tau <= 1)) return err(PDRT_EINVAL, "tau must be in [0,1]");

    // lattice: +-H pixels around the isocentre covering every voxel
    double rmax = 0.0;
    for (int cx = 0; cx < 2; ++cx)
        for (int cy = 0; cy < 2; ++cy) {
            const double x = origin_mm[0] + (cx ? nx - 1 : 0) * sx - iso_mm[0];
            const double y = origin_mm[1] + (cy ? ny - 1 : 0) * sy - iso_mm[1];
            rmax = std::max(rmax, sqrt(x * x + y * y));
        }
    const int H = (int)ceil(rmax / sx - 1e-9) + 1;
    Lattice L;
    L.nu = L.nw = 2 * H + 1;
    L.nv = nz;
    L.cu = L.cw = (float)H;
    const double cv = (iso_mm[2] - origin_mm[2]) / sz;
    L.cv = (float)cv;
    L.du = (float)sx;
    L.dv = (float)sz;
    if (!(m->sid_mm > (H + 2) * sx)) return err(PDRT_EINVAL, "SID must exceed the grid's reach");
    // the gather's slice records pack the v bounds of a box in 16 bits each
    if (L.nv > 32767) return err(PDRT_EINVAL, "grid too large: nz must be at most 32767");

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
    if (M.nq4 < 0) return err(PDRT_EINVAL, "no convolution variant for this radius");
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
    if (const char *why = machine_corrections(m, sx, sz, M)) return err(PDRT_EINVAL, why);

    // geometry of the control point and the needed slice ranges (host, double)
    const double px0 = (iso_mm[0] - origin_mm[0]) / sx, py0 = (iso_mm[1] - origin_mm[1]) / sy;
    const double phi = gantry_deg * M_PI / 180.0, cs = cos(phi), sn = sin(phi);
    CpGeo G;
    G.au = (float)cs; G.bu = (float)-sn; G.aw = (float)sn; G.bw = (float)cs;
    G.cu0 = (float)(H - cs * px0 + sn * py0);
    G.cw0 = (float)(H - sn * px0 - cs * py0);
    G.sx_w = (float)sn; G.sy_w = (float)cs;
    G.px0 = (float)px0; G.py0 = (float)py0; G.pz0 = (float)cv;
    double fu[4], fw[4];
    const int cxs[4] = {0, nx - 1, nx - 1, 0}, cys[4] = {0, 0, ny - 1, ny - 1};
    for (int c = 0; c < 4; ++c) {
        fu[c] = cs * (cxs[c] - px0) - sn * (cys[c] - py0) + H;
        fw[c] = sn * (cxs[c] - px0) + cs * (cys[c] - py0) + H;
    }
    std::vector<int2> ukr(L.nw);
    long long cap_o = 1;
    for (int k = 0; k < L.nw; ++k) {
        int lo, hi;
        needed_u_range(fu, fw, k, L.nu, lo, hi);
        ukr[k] = make_int2(lo, hi);
        cap_o += (long long)(hi - lo) * L.nv;
    }

    // layout inside the static array
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    const size_t o_flags = take(sizeof(unsigned) * 4);
    const size_t o_cptab = take(sizeof(CpTab));
    const size_t o_geo = take(sizeof(CpGeo));
    const size_t o_lb = take(sizeof(float) * (m->n_pairs + 1));
    const size_t o_dd = take(sizeof(float) * m->n_depth);
    const size_t o_ukr = take(sizeof(int2) * L.nw);
    const size_t o_slices = take(sizeof(SliceTab) * L.nw);
    const size_t o_gbox = take(sizeof(int4) * L.nw);
    const size_t o_f = take(sizeof(float) * (size_t)L.nu * L.nv);
    const size_t o_region = take(sizeof(float) * (size_t)cap_o);
    // corrections: raw map and blurred map scratch
    const size_t o_t = M.corr ? take(sizeof(float) * (size_t)L.nu * L.nv) : 0;
    const size_t o_g = M.corr ? take(sizeof(float) * (size_t)L.nu * L.nv) : 0;
    if (off > (size_t)PDRT_STATIC_SCRATCH_BYTES) {
        char msg[256];
        snprintf(msg, sizeof(msg),
                 "grid needs %.1f MiB of scratch; the allocation-free entry point holds %.1f MiB "
                 "(PDRT_STATIC_SCRATCH_BYTES): use pdrt_plan_upload/pdrt_dose_forward",
                 off / 1048576.0, PDRT_STATIC_SCRATCH_BYTES / 1048576.0);
        return err(PDRT_EINVAL, msg);
    }

    // once per device: device address of the static array, convolution set-up
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return err(PDRT_EDEVICE, "device index out of range");
    unsigned char *base = nullptr;
    int conv_blocks = 0;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            int major = 0, minor = 0;
            cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
            if (major * 10 + minor != 103)
                return err(PDRT_EDEVICE, "this library is built for sm_103a");
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess) return cuda_err(e, "cudaGetSymbolAddress(g_static_scratch)");
            g_scratch_ptr[dev] = p;
        }
        base = static_cast<unsigned char *>(g_scratch_ptr[dev]);
        if (!(g_conv_ready[dev] >> M.nq4 & 1ull)) {
            int bf = 1, ba = 1, sms = 1;
            e = conv_prepare(M, &bf, &ba);
            if (e != cudaSuccess) return cuda_err(e, "convolution kernel set-up");
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            g_conv_blocks[dev][M.nq4] = std::max(1, bf) * std::max(1, sms);
            g_conv_ready[dev] |= 1ull << M.nq4;
        }
        conv_blocks = g_conv_blocks[dev][M.nq4];
    }

    PlanDev P;
    memset(&P, 0, sizeof(P));
    P.lat = L;
    P.mach = M;
    P.n_cp = 1;
    P.nx = nx; P.ny = ny; P.nz = nz;
    P.red = red_dev;
    P.leaf_bounds = reinterpret_cast<const float *>(base + o_lb);
    P.depth_dose = reinterpret_cast<const float *>(base + o_dd);
    P.cpgeo = reinterpret_cast<const CpGeo *>(base + o_geo);
    P.ukr = reinterpret_cast<const int2 *>(base + o_ukr);
    P.cptab = reinterpret_cast<CpTab *>(base + o_cptab);
    P.slices = reinterpret_cast<SliceTab *>(base + o_slices);
    P.gbox = reinterpret_cast<int4 *>(base + o_gbox);
    P.fbuf = reinterpret_cast<float *>(base + o_f);
    if (M.corr) {
        P.tbuf = reinterpret_cast<float *>(base + o_t);
        P.gfbuf = reinterpret_cast<float *>(base + o_g);
    }
    P.region = reinterpret_cast<float *>(base + o_region);
    P.cap_o = cap_o;
    P.cap_a = 1LL << 62;   // forward only: the adjoint buffer is never touched
    P.flags = reinterpret_cast<unsigned *>(base + o_flags);
    P.counters = P.flags + 1;

    std::vector<float> lb(m->n_pairs + 1), dd(m->n_depth);
    for (int i = 0; i <= m->n_pairs; ++i) lb[i] = (float)m->leaf_bounds_mm[i];
    for (int i = 0; i < m->n_depth; ++i) dd[i] = (float)m->depth_dose[i];
    cudaStream_t s = (cudaStream_t)stream;
    // pageable host sources: each copy returns once its data is staged
    if ((e = cudaMemsetAsync(base + o_flags, 0, sizeof(unsigned) * 4, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(base + o_lb, lb.data(), lb.size() * sizeof(float),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(base + o_dd, dd.data(), dd.size() * sizeof(float),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(base + o_geo, &G, sizeof(G), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(base + o_ukr, ukr.data(), ukr.size() * sizeof(int2),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_err(e, "static scratch upload");
    if ((e = launch_raster(P, leaves_dev, jaws_dev, mu_dev, s)) != cudaSuccess)
        return cuda_err(e, "project_raster launch");
    internal_count_launch();
    if ((e = launch_tables(P, s)) != cudaSuccess) return cuda_err(e, "wepl_tables launch");
    internal_count_launch();
    if ((e = launch_conv(P, 0, 1, false, P.counters, conv_blocks, s)) != cudaSuccess)
        return cuda_err(e, "conv_forward launch");
    internal_count_launch();
    if ((e = launch_gather(P, 0, 1, dose_dev, true, s)) != cudaSuccess)
        return cuda_err(e, "gather launch");
    internal_count_launch();
    // the pageable sources above must stay valid until their copies are staged
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_err(e, "stream sync");
    // device-detected input problems of this call (cleared at its start)
    unsigned flags = 0;
    if ((e = cudaMemcpy(&flags, base + o_flags, sizeof(flags), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_err(e, "flag read-back");
    if (flags & PDRT_FLAG_NAN_INPUT)
        return err(PDRT_EINVAL, "a leaf, jaw or MU value is NaN or infinite (PDRT_FLAG_NAN_INPUT)");
    if (flags & PDRT_FLAG_CAPACITY)
        return err(PDRT_EINVAL, "a beam slice exceeded the scratch bound and was dropped (PDRT_FLAG_CAPACITY)");
    if (flags) return err(PDRT_EINVAL, "device flag raised during the call");
    return PDRT_OK;
}
