// pdrt_calibrate: output calibration of Sec. 2.4 with the engine's own
// kernels.  The paper normalises the machine output so that a set number of
// reference MU gives 1 Gy at its reference conditions (10 cm x 10 cm field,
// 10 cm depth in water, SSD 90 cm), by computing the dose in a virtual water
// phantom and adjusting the scaling factor.  The discrete set-up (a reading,
// stated in include/pdrt.h): the reference point is the isocentre, 100 mm
// below the water surface on the central axis at gantry 0 (SSD = SID - 100
// mm); the field is 100 x 100 mm at the isocentre plane (jaws and every leaf
// pair at +-50 mm, collimator 0); the grid has the caller's pitch with the
// isocentre on a voxel centre, and a voxel row holds the water fraction of its
// extent as density, so that the midpoint depth sum reaches exactly 100 mm at
// the isocentre.  Host code only: it builds the phantom, runs one forward
// through the public entry points and reads one voxel back.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pdrt_impl.cuh"

using namespace pdrt;

namespace {

// frees what one calibration run allocated, on every exit path
struct CalScratch {
    float *hu = nullptr, *leaves = nullptr, *jaws = nullptr, *mu = nullptr, *dose = nullptr;
    pdrt_grid_t grid = nullptr;
    pdrt_plan_t plan = nullptr;
    ~CalScratch()
    {
        if (plan) pdrt_plan_destroy(plan);
        if (grid) pdrt_grid_destroy(grid);
        cudaFree(hu);
        cudaFree(leaves);
        cudaFree(jaws);
        cudaFree(mu);
        cudaFree(dose);
    }
};

pdrt_status cal_fail(pdrt_status st, const char *msg)
{
    internal_set_error(msg);
    return st;
}

pdrt_status cal_cuda(cudaError_t e, const char *what)
{
    char buf[256];
    snprintf(buf, sizeof(buf), "pdrt_calibrate: %s: %s", what, cudaGetErrorString(e));
    internal_set_error(buf);
    return e == cudaErrorMemoryAllocation ? PDRT_ENOMEM : PDRT_ECUDA;
}

}  // namespace

extern "C" pdrt_status pdrt_calibrate(const pdrt_machine *m, double sxy, double sz, double ref_mu,
                                      double ref_gy, double *cal_out, pdrt_stream_t stream)
{
    internal_set_error("");
    if (!m || !cal_out) return cal_fail(PDRT_EINVAL, "pdrt_calibrate: NULL argument");
    if (!(sxy > 0) || !(sz > 0) || !std::isfinite(sxy) || !std::isfinite(sz))
        return cal_fail(PDRT_EINVAL, "pdrt_calibrate: pitches must be positive and finite");
    if (!(ref_mu > 0) || !(ref_gy > 0) || !std::isfinite(ref_mu) || !std::isfinite(ref_gy))
        return cal_fail(PDRT_EINVAL, "pdrt_calibrate: reference MU and dose must be positive");
    if (m->n_pairs < 1 || m->n_pairs > PDRT_MAX_PAIRS)
        return cal_fail(PDRT_EINVAL, "pdrt_calibrate: bad n_pairs");
    if (m->kernel_radius_px < 0 || m->kernel_radius_px > PDRT_MAX_RADIUS_PX)
        return cal_fail(PDRT_EINVAL, "pdrt_calibrate: kernel radius out of range");

    // reference beam model: the caller's, at unit output and collimator 0
    pdrt_machine mr = *m;
    mr.cal = 1.0;
    mr.collimator_deg = 0.0;
    MachineDev M;
    memset(&M, 0, sizeof(M));
    if (const char *why = machine_corrections(&mr, sxy, sz, M)) return cal_fail(PDRT_EINVAL, why);

    // every lattice pixel the isocentre's dose reads: the kernel window (its
    // corner sqrt(2) R away, in mm), the penumbra half-window, two more pixels
    const int R = mr.kernel_radius_px;
    const double reach = R * sqrt(sxy * sxy + sz * sz);
    const int hx = (int)ceil(reach / sxy) + M.rbu + 2;
    const int hz = (int)ceil(reach / sz) + M.rbv + 2;
    const int above = (int)ceil(100.0 / sxy + 0.5) + 2;   // voxel rows above the isocentre
    const int nx = 2 * hx + 1, nz = 2 * hz + 1, ny = above + 3;
    const size_t nvox = (size_t)nx * ny * nz;

    // HU through the curve (-1000, 0) - (0, 1): density = water fraction
    std::vector<float> hu(nvox);
    for (int j = 0; j < ny; ++j) {
        const double y = (j - above) * sxy;                 // row centre, mm from the isocentre
        const double f = std::min(1.0, std::max(0.0, (y + 0.5 * sxy + 100.0) / sxy));
        const float h = (float)(1000.0 * (f - 1.0));
        for (int k = 0; k < nz; ++k)
            std::fill(hu.begin() + ((size_t)k * ny + j) * nx, hu.begin() + ((size_t)k * ny + j + 1) * nx, h);
    }
    const double curve[4] = {-1000.0, 0.0, 0.0, 1.0};
    const double origin[3] = {-hx * sxy, -above * sxy, -hz * sz};
    const double iso[3] = {0.0, 0.0, 0.0};
    const double gantry = 0.0;
    std::vector<float> leaves(2 * (size_t)mr.n_pairs);
    for (int i = 0; i < mr.n_pairs; ++i) {
        leaves[2 * i] = -50.0f;
        leaves[2 * i + 1] = 50.0f;
    }
    const float jaws[4] = {-50.0f, 50.0f, -50.0f, 50.0f};
    const float mu = (float)ref_mu;

    cudaStream_t s = (cudaStream_t)stream;
    CalScratch c;
    cudaError_t e;
    if ((e = cudaMalloc(&c.hu, nvox * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&c.dose, nvox * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&c.leaves, leaves.size() * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&c.jaws, sizeof(jaws))) != cudaSuccess ||
        (e = cudaMalloc(&c.mu, sizeof(float))) != cudaSuccess)
        return cal_cuda(e, "allocation");
    if ((e = cudaMemcpyAsync(c.hu, hu.data(), nvox * sizeof(float), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c.leaves, leaves.data(), leaves.size() * sizeof(float), cudaMemcpyHostToDevice,
                             s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c.jaws, jaws, sizeof(jaws), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c.mu, &mu, sizeof(float), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cal_cuda(e, "upload");
    pdrt_status st = pdrt_grid_create(&c.grid, c.hu, nx, ny, nz, sxy, sxy, sz, origin, curve, 2, stream);
    if (st != PDRT_OK) return st;
    st = pdrt_plan_upload(&c.plan, c.grid, 1, &gantry, iso, &mr, 0, stream);
    if (st != PDRT_OK) return st;
    st = pdrt_dose_forward(c.grid, c.plan, c.leaves, c.jaws, c.mu, c.dose, stream);
    if (st != PDRT_OK) return st;
    uint32_t flags = 0;
    st = pdrt_plan_status(c.plan, stream, &flags);   // synchronises the stream
    if (st != PDRT_OK) return st;
    if (flags) return cal_fail(PDRT_ECUDA, "pdrt_calibrate: device flag raised in the reference forward");
    float d_ref = 0.f;
    const size_t iref = ((size_t)hz * ny + above) * nx + hx;
    if ((e = cudaMemcpy(&d_ref, c.dose + iref, sizeof(float), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cal_cuda(e, "read-back");
    if (!(d_ref > 0.f) || !std::isfinite(d_ref))
        return cal_fail(PDRT_EINVAL, "pdrt_calibrate: the reference dose is not positive "
                                     "(depth-dose table or kernel give no dose at 10 cm)");
    *cal_out = ref_gy / (double)d_ref;
    return PDRT_OK;
}
