/*
 * pdrt.h -- C ABI of the GB300 (sm_103a) pencil-beam VMAT dose engine.
 *
 * The engine maps delivery parameters (MLC leaf positions, jaws, MUs at each
 * control point of a VMAT arc) to a 3-D dose on a CT grid, and back-propagates
 * a dose gradient to those parameters.  It implements the layer chain of
 * arXiv 2512.18863, Sec. 2.1-2.2.7:
 *   hardware projection (Sec. 2.2.1) -> fluence map (Sec. 2.2.2, fractional
 *   overlap, jaw masking, MLC transmission) -> divergent fluence volume
 *   (Sec. 2.2.3, magnification SID/d and inverse square) -> radiological depth
 *   on the central ray (Sec. 2.2.4) -> depth-dependent radial kernel
 *   (Sec. 2.2.5) -> per-slice 2-D convolution (Sec. 2.2.6) -> rotation to the
 *   patient grid and MU-weighted sum (Sec. 2.2.7, Eq. D_total).
 *
 * Conventions shared by every entry point
 *   - Lengths in mm, angles in degrees, MU in monitor units.  Leaf and jaw
 *     positions are given at the isocentre plane.
 *   - Volumes are [nz][ny][nx] float32, x fastest.  Voxel (0,0,0) is centred
 *     at origin_mm.  sx must equal sy (the beam frame uses one in-plane pitch).
 *   - Leaves are [n_cp][n_pairs][2] float32: (left, right) edge of each pair.
 *     Jaws are [n_cp][4] float32: (x-, x+, y-, y+).  MU is [n_cp] float32.
 *   - Geometry: the gantry rotates about the patient z axis; the beam
 *     direction is e_w = (sin g, cos g, 0), leaves travel along
 *     e_u = (cos g, -sin g, 0), leaf pairs are stacked along e_v = +z, and the
 *     source sits at iso - SID e_w.
 *   - Pointers named *_dev are device pointers (cudaMalloc / PyTorch CUDA
 *     tensors) on the device that was current at pdrt_grid_create; pointers
 *     named *_host or passed by value are host memory read during the call.
 *   - Streams: pdrt_stream_t is a cudaStream_t (NULL = legacy default stream).
 *     pdrt_dose_forward / pdrt_dose_backward only enqueue work on that stream
 *     and return; they allocate nothing (all scratch is owned by the plan and
 *     is allocated in pdrt_plan_upload).  One plan must not be used by two
 *     calls that can overlap on the GPU (they share the plan's scratch).
 *   - Ownership: the caller owns every buffer passed in; the library owns the
 *     grid and plan handles and frees them in pdrt_*_destroy.
 *   - Errors: every call returns a pdrt_status; on failure pdrt_last_error()
 *     gives a message (thread-local, valid until the next call on the same
 *     thread).  Argument errors are detected on the host before any work is
 *     enqueued.  Bad values inside device buffers (NaN leaves, jaws or MU) are
 *     detected on the device and reported by pdrt_plan_status.
 */
#ifndef PDRT_H
#define PDRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PDRT_MAX_PAIRS 160        /* leaf pairs per bank */
#define PDRT_MAX_RADIUS_PX 44     /* kernel half-window, pixels */
#define PDRT_MAX_PEN_RADIUS_PX 16 /* source-penumbra blur half-window ceil(3 sigma / pitch) */
#define PDRT_MAX_DEPTH_TABLE 4096 /* depth-dose table entries */
#define PDRT_MAX_HU_POINTS 32     /* HU -> density calibration points */

typedef struct pdrt_grid_s *pdrt_grid_t;
typedef struct pdrt_plan_s *pdrt_plan_t;
typedef void *pdrt_stream_t;

typedef enum {
    PDRT_OK = 0,
    PDRT_EINVAL = 1,   /* invalid argument value (NULL pointer, NaN, out of range) */
    PDRT_ESHAPE = 2,   /* inconsistent sizes */
    PDRT_ECUDA = 3,    /* a CUDA runtime call or kernel launch failed */
    PDRT_ENOMEM = 4,   /* device or host allocation failed */
    PDRT_EDEVICE = 5   /* the device is not sm_103a, the only architecture the library is compiled for */
} pdrt_status;

/* Device-detected input problems, reported by pdrt_plan_status. */
#define PDRT_FLAG_NAN_INPUT 1u     /* a leaf, jaw or MU value was NaN/inf */
#define PDRT_FLAG_CAPACITY 2u      /* internal: a slice's work exceeded the plan's scratch
                                      bound and was dropped (dose incomplete) */
#define PDRT_FLAG_TIMEOUT 4u       /* a bounded wait on the tensor cores expired; the
                                      kernel stopped early (result incomplete) */

/*
 * Beam model (machine) constants, Sec. 2.2 and Sec. 2.4.
 *   sid_mm          source-isocentre distance.
 *   leaf_bounds_mm  n_pairs+1 ascending positions along e_v of the leaf-pair
 *                   boundaries at the isocentre plane.
 *   tau             MLC transmission (Sec. 2.2.2): F = f_jaw (tau + (1-tau) f_leaf).
 *   wmin_*_mm, f_*_mm  minimum opening and half travel range of the aperture
 *                   centre in the projection of Sec. 2.2.1 (jaw values apply
 *                   to both jaw pairs).
 *   eps_mu          lower MU bound of Sec. 2.2.1.
 *   kernel_radius_px  half window R of the (2R+1)^2 lateral kernel (Sec. 2.2.5).
 *   kernel_alpha[c][k], kernel_beta[c][k]  three radial exponentials
 *                   K(r;z) = sum_c w_c(z) exp(-a_c(z) r) / S_c(z) with
 *                   a_c = max(alpha_c0 + alpha_c1 z + alpha_c2 z^2, 1e-4) /mm,
 *                   w_c = max(beta_c0 + beta_c1 z + beta_c2 z^2, 0), normalised
 *                   to sum 1, S_c the sum of exp(-a_c r) over the window.
 *   depth_dose[n_depth], depth_step_mm  depth-dose table T(z) at z = m step,
 *                   linearly interpolated and clamped at both ends.
 *   cal             output calibration factor (Sec. 2.4).
 *   ste             1: the projection of Sec. 2.2.1 is the identity in the
 *                   backward pass (straight-through estimator); 0: exact
 *                   Jacobian (zero gradient through active clamps).
 *   pen_fwhm_u_mm, pen_fwhm_v_mm  source penumbra (Sec. 2.2.2): the aperture
 *                   fluence is blurred along e_u, then along e_v, by a discrete
 *                   Gaussian exp(-(t pitch)^2 / (2 sigma^2)), sigma = FWHM /
 *                   (2 sqrt(2 ln 2)), |t| <= ceil(3 sigma / pitch), normalised
 *                   to unit sum, zero outside the lattice. 0 = no blur.
 *   off_axis[3]     off-axis profile (Sec. 2.2.2): the blurred map is
 *                   multiplied by c0 + c1 r + c2 r^2, r = distance (mm) of the
 *                   pixel centre from the central axis. (1, 0, 0) = off.
 *   collimator_deg  collimator angle of every control point (Sec. 2.2.2, last
 *                   paragraph): the corrected map is turned by this angle in the
 *                   (e_u, e_v) plane; pixel x reads it bilinearly at R(-angle) x,
 *                   zero outside the lattice. 0 = off.
 */
typedef struct {
    double sid_mm;
    int32_t n_pairs;
    double leaf_bounds_mm[PDRT_MAX_PAIRS + 1];
    double tau;
    double wmin_leaf_mm, wmin_jaw_mm;
    double f_leaf_mm, f_jaw_mm;
    double eps_mu;
    int32_t kernel_radius_px;
    double kernel_alpha[3][3];
    double kernel_beta[3][3];
    int32_t n_depth;
    double depth_step_mm;
    double depth_dose[PDRT_MAX_DEPTH_TABLE];
    double cal;
    int32_t ste;
    double pen_fwhm_u_mm, pen_fwhm_v_mm;
    double off_axis[3];
    double collimator_deg;
} pdrt_machine;

/* Beam-frame lattice and scratch layout of a plan (host-side query). */
typedef struct {
    int32_t nu, nv, nw;          /* lattice size along e_u, e_v, e_w */
    double cu, cv, cw;           /* lattice index of the isocentre */
    int32_t n_cp;
    int32_t chunk_cp;            /* control points processed per pass */
    size_t scratch_bytes;        /* device scratch owned by the plan */
    int32_t tensor_cores;        /* 1: the convolution runs on the tensor cores (every slice) */
    int32_t tc_ctas_per_sm[2];   /* tensor-core convolution CTAs per SM (forward, adjoint) */
    int32_t simt_ctas_per_sm[2]; /* resident FP32 convolution CTAs per SM (forward, adjoint) */
    int32_t tc_phase[2];         /* tensor-core kernel rows per operand phase (forward, adjoint) */
    int32_t fft_pmax;            /* > 0: FFT convolution for slices whose padded sizes are at most
                                    this, tensor cores for the rest; 0: FFT off */
    int32_t fft_ctas_per_sm[2];  /* FFT convolution CTAs per SM (forward, adjoint) */
    int32_t spectrum_memo_pmax;  /* kernel-spectrum memo: largest padded size memoised (0: off) */
    size_t spectrum_memo_bytes;  /* device memory of the memo (not part of scratch_bytes) */
} pdrt_plan_info;

/*
 * Kernel-spectrum memo of the FFT convolution (Sec. 2.2.6).  The spectrum
 * of slice k of control point b -- the DFT of the kernel K(z_k), scaled by
 * T(z_k) C(d_k) -- depends only on what the plan fixes (the slice's WEPL
 * depth, kernel parameters and magnification) and on the slice's padded
 * transform sizes (pu, pv), which follow from the fluence support of the
 * call.  With the memo on, the FFT convolution stores each spectrum it
 * computes, tagged with (pu, pv), and takes it from the memo while the sizes
 * stay the same: the adjoint of a call takes what its forward computed (the
 * two directions pad a slice to the same sizes), later calls take what
 * earlier ones computed.  The stored spectra are bit-identical to
 * recomputed ones, so every result is the same with the memo on or off.
 * The upload turns it on for its default size limit when the memory
 * (n_cp x nw x (pmax/2 + 1)^2 floats, pdrt_plan_info.spectrum_memo_bytes)
 * can be allocated; slices padded beyond that limit are not memoised.
 * pdrt_plan_set_spectrum_memo: enable = 0 frees it, 1 allocates it for the
 * current FFT size limit (host, synchronous).  pdrt_plan_reset_spectrum_memo
 * forgets every stored spectrum (asynchronous on stream; the next call
 * computes them again).  A batch (pdrt_batch_create) records the memo of
 * each of its plans: do not turn a plan's memo on or off while a batch
 * holds the plan.  Errors: EINVAL (NULL plan; enable with the FFT
 * convolution off), ECUDA (allocation).
 */
pdrt_status pdrt_plan_set_spectrum_memo(pdrt_plan_t p, int32_t enable);
pdrt_status pdrt_plan_reset_spectrum_memo(pdrt_plan_t p, pdrt_stream_t stream);

/* Work counters of the last forward/backward call (for roofline accounting). */
typedef struct {
    int64_t active_slices;       /* (control point, beam slice) pairs with work */
    int64_t support_points;      /* beam-frame points with non-zero fluence input */
    int64_t region_points;       /* beam-frame points where dose is produced */
    int64_t taps;                /* (2R+1)^2 */
    double conv_flops;           /* 2 * taps * support_points: one convolution pass */
    double mma_flops;            /* tensor-core FLOPs issued by one forward + one adjoint
                                    convolution pass (BF16 three-term split, padded tiles) on
                                    the slices the tensor cores take */
    double fft_flops;            /* FP32 FLOPs of the FFT convolution of one forward + one
                                    adjoint pass on the slices it takes: per slice and direction
                                    2 x 2.5 N log2 N for the forward and inverse real 2-D FFTs
                                    (N = Pu Pv) and the product 2 Pv (Pu/2+1); the kernel
                                    spectrum's cosine sums 2 (R+1)^2 (Pv/2+1) +
                                    2 (R+1)(Pv/2+1)(Pu/2+1) per slice in the forward, and in
                                    the adjoint where the spectrum memo does not hold its
                                    sizes */
    int64_t fft_slices;          /* (slice, direction) pairs the FFT convolution takes */
    int64_t tc_slices;           /* (slice, direction) pairs left to the tensor cores */
} pdrt_work;

/* Per-kernel device time accumulated while profiling is enabled. */
#define PDRT_NUM_KERNELS 12
typedef struct {
    const char *name[PDRT_NUM_KERNELS];
    int64_t launches[PDRT_NUM_KERNELS];
    double total_ms[PDRT_NUM_KERNELS];
    int32_t overflow;            /* 1 if the event pool ran out (times incomplete) */
} pdrt_profile;

/*
 * Create a CT grid on the current device.
 *   out         receives the handle.
 *   hu_dev      [nz][ny][nx] Hounsfield units (device, read once, not kept).
 *   sx,sy,sz    voxel spacing (mm); sx == sy required.
 *   origin_mm   centre of voxel (0,0,0) (host, 3 values).
 *   hu_red_host n_pts (HU, relative electron density) pairs, ascending HU
 *               (host); the commissioned piecewise-linear curve of Sec. 2.2,
 *               clamped at both ends.
 * Errors: EINVAL (NULL pointers, non-positive sizes or spacing, sx != sy,
 * unsorted or too many points), EDEVICE (device is not sm_103), ENOMEM, ECUDA.
 */
pdrt_status pdrt_grid_create(pdrt_grid_t *out, const float *hu_dev, int32_t nx, int32_t ny,
                             int32_t nz, double sx, double sy, double sz, const double origin_mm[3],
                             const double *hu_red_host, int32_t n_pts, pdrt_stream_t stream);
void pdrt_grid_destroy(pdrt_grid_t g);

/*
 * Upload a VMAT plan geometry (Sec. 2.2: beam sequence of control points).
 *   gantry_deg_host  [n_cp] gantry angle of each control point (host).
 *   iso_mm           isocentre, patient frame (host, 3 values).
 *   m                beam model (host, copied).
 *   scratch_budget_bytes  upper bound on the device scratch the plan may own
 *                    (0 = library default: a quarter of the free device
 *                    memory, between 1 and 4 GiB); it sets how many control
 *                    points one pass processes (passes are balanced).  Fewer,
 *                    longer passes are faster (a 256x256x160 two-arc plan
 *                    runs 2 passes at 24 GB and is ~15 % slower at 4 GB);
 *                    the kernel-spectrum memo is allocated beside it.
 * The plan owns all device scratch the forward and backward passes need.
 * Errors: ESHAPE (n_cp < 1: an arc needs a control point), EINVAL (bad
 * values; kernel radius above PDRT_MAX_RADIUS_PX; SID not larger than the
 * grid's reach from the isocentre), ENOMEM, ECUDA.
 */
pdrt_status pdrt_plan_upload(pdrt_plan_t *out, pdrt_grid_t g, int32_t n_cp,
                             const double *gantry_deg_host, const double iso_mm[3],
                             const pdrt_machine *m, size_t scratch_budget_bytes,
                             pdrt_stream_t stream);
void pdrt_plan_destroy(pdrt_plan_t p);

/*
 * Forward dose (Eq. D_total):
 *   dose(x) = cal sum_b MU^_b  Rot_b( T(z) (K(z) * Phi_b) )(x)
 * with Phi_b the divergent fluence volume of control point b.
 *   leaves_dev [n_cp][n_pairs][2], jaws_dev [n_cp][4], mu_dev [n_cp] (device, raw:
 *   the projection of Sec. 2.2.1 is applied inside).
 *   dose_dev   [nz][ny][nx] (device), overwritten.
 * Errors: EINVAL (NULL pointers, handles from different grids), ECUDA.
 */
pdrt_status pdrt_dose_forward(pdrt_grid_t g, pdrt_plan_t p, const float *leaves_dev,
                              const float *jaws_dev, const float *mu_dev, float *dose_dev,
                              pdrt_stream_t stream);

/*
 * Adjoint of pdrt_dose_forward: given dL/d dose, writes dL/d leaves, dL/d jaws
 * and dL/d MU (raw parameters; through the projection of Sec. 2.2.1 as set by
 * machine.ste).  Radiological depths and kernels are recomputed, not stored.
 *   dose_grad_dev [nz][ny][nx] (device, read).
 *   dleaves_dev, djaws_dev, dmu_dev: same shapes as the inputs, overwritten.
 * Leaf edges are differentiated as the piecewise-linear overlap of
 * Sec. 2.2.2 (one-sided at pixel boundaries).
 * Errors: as pdrt_dose_forward.
 */
pdrt_status pdrt_dose_backward(pdrt_grid_t g, pdrt_plan_t p, const float *leaves_dev,
                               const float *jaws_dev, const float *mu_dev,
                               const float *dose_grad_dev, float *dleaves_dev, float *djaws_dev,
                               float *dmu_dev, pdrt_stream_t stream);

/*
 * Output calibration (Sec. 2.4): the paper normalises the output so that a
 * set number of reference MU gives 1 Gy at reference conditions (10 cm x 10 cm
 * field, 10 cm depth in water, SSD 90 cm), computing the dose in a virtual
 * water phantom.  This call runs that forward with the engine's kernels and
 * returns cal = ref_gy / D_ref, D_ref being the dose of ref_mu MU of the
 * reference field at the reference point with cal = 1; pass the result as
 * pdrt_machine.cal of the plans.
 * Reading of the discrete set-up: the reference point is the isocentre,
 * 100 mm below the water surface on the central axis at gantry 0 (SSD = SID -
 * 100 mm, i.e. 90 cm at SID 1 m); the field is 100 x 100 mm at the isocentre
 * plane (jaws and every leaf pair at +-50 mm, collimator 0; the model's
 * transmission, penumbra and off-axis profile apply); voxels sxy x sxy x sz,
 * the patient grid's pitch, so that kernel_radius_px means the same; the
 * isocentre on a voxel centre; a voxel row holds the water fraction of its
 * extent as density, so that the midpoint depth at the isocentre is exactly
 * 100 mm; the grid reaches every lattice pixel the isocentre's dose reads.
 *   m        beam model (host; its cal and collimator_deg are ignored).
 *   sxy, sz  voxel pitch in-plane and along z (mm).
 *   ref_mu, ref_gy  the reference MU and the dose they must give (e.g. 100, 1).
 *   cal_out  receives the factor (host).
 * Allocates and frees temporary device memory and synchronises `stream`.
 * Errors: EINVAL (NULL, non-positive values, bad beam model, or a model that
 * gives no dose at the reference point), ENOMEM, ECUDA, EDEVICE.
 */
pdrt_status pdrt_calibrate(const pdrt_machine *m, double sxy, double sz, double ref_mu,
                           double ref_gy, double *cal_out, pdrt_stream_t stream);

/*
 * Route the per-slice convolution (Sec. 2.2.6) to the tensor cores (enable = 1,
 * the default: BF16 three-term split, FP32 accumulation, every slice tiled;
 * with the FFT convolution on, only the slices it leaves) or to the FP32 SIMT
 * kernel (enable = 0, which also turns the FFT convolution off).  Host only.
 * Errors: EINVAL if enable = 1 and the tensor-core kernel does not fit in
 * shared memory (it fits for every radius up to PDRT_MAX_RADIUS_PX).
 */
pdrt_status pdrt_plan_set_tensor_cores(pdrt_plan_t p, int32_t enable);

/*
 * FFT convolution (Sec. 2.2.6 computed by FP32 FFTs in shared memory, the
 * default): slices whose padded transform sizes are at most pmax are
 * convolved by FFT, the others by the tensor-core kernel.  pmax = 0 turns it
 * off; otherwise one of 32, 40, 48, 60, 64, 72, 80, 90, 96, 100, 108, 120,
 * 128, 144, 160, 192 (sets the shared memory per CTA and so the CTAs per SM).  The upload picks the
 * smallest size that holds a 48-pixel input plus the kernel's 2R margin,
 * raised to the largest size that keeps as many CTAs per SM.
 * Host only.  Errors: EINVAL (NULL plan, unsupported size, size below
 * 2 kernel_radius_px + 2, size that does not fit in shared memory, or the
 * tensor-core path is off: it takes the overflow).
 */
pdrt_status pdrt_plan_set_fft(pdrt_plan_t p, int32_t pmax);

/* Lattice and scratch sizes of a plan (host only, no device work).
 * Errors: EINVAL (NULL argument). */
pdrt_status pdrt_plan_get_info(pdrt_plan_t p, pdrt_plan_info *out);

/*
 * Synchronises `stream`, returns the device-detected input flags
 * (PDRT_FLAG_*) raised since the previous call, and clears them.
 * Errors: EINVAL (NULL argument), ECUDA (the synchronisation or the flag
 * copy failed, e.g. an earlier kernel of the stream faulted).
 */
pdrt_status pdrt_plan_status(pdrt_plan_t p, pdrt_stream_t stream, uint32_t *flags_out);

/* Synchronises `stream` and returns the work counters of the last call.
 * Errors: EINVAL (NULL argument), ECUDA. */
pdrt_status pdrt_plan_work(pdrt_plan_t p, pdrt_stream_t stream, pdrt_work *out);

/*
 * Per-kernel timing with CUDA events recorded on the launch stream around
 * every kernel the plan launches.  enable != 0 starts (and clears) a
 * measurement; pdrt_profile_read synchronises `stream` and returns the sums.
 * Errors: EINVAL (NULL argument), ECUDA (event creation, synchronisation).
 */
pdrt_status pdrt_profile_enable(pdrt_plan_t p, int32_t enable);
pdrt_status pdrt_profile_read(pdrt_plan_t p, pdrt_stream_t stream, pdrt_profile *out);

/*
 * Allocation-free forward dose of ONE control point.  The paper has no
 * counterpart: this is an integration variant of pdrt_dose_forward for
 * callers that cannot call cudaMalloc -- for example a plug-in hosted by a
 * framework that owns all device memory and hands it only input and output
 * buffers, or a latency-critical loop that must never enter the CUDA
 * allocator (cudaMalloc/cudaFree can synchronise the device and can fail on
 * fragmented memory).  pdrt_grid_create and pdrt_plan_upload allocate, so this
 * entry point takes the density grid and the beam model directly and uses
 * no handle.
 *   red_dev     [nz][ny][nx] relative electron density (device; the HU curve
 *               of pdrt_grid_create already applied by the caller).
 *   nx..origin_mm  grid as in pdrt_grid_create; iso_mm, gantry_deg, m as in
 *               pdrt_plan_upload for a one-point plan.
 *   leaves_dev [n_pairs][2], jaws_dev [4], mu_dev [1] (device, raw).
 *   dose_dev   [nz][ny][nx] (device), overwritten with this point's dose.
 * Scratch: all intermediate data lives in one static device array of
 * PDRT_STATIC_SCRATCH_BYTES inside the library, held by every GPU that loads
 * the library until the process exits.  The first call made with a device
 * current looks up that array's device address (cudaGetSymbolAddress) and
 * prepares the kernels for that device.  Every call shares the array, which
 * keeps the last call's contents (counters and flags are cleared at the start
 * of each call); calls that can overlap on the GPU (other streams, other host
 * threads) race on it.
 * Synchronous: the call copies host tables, synchronises `stream` and reads
 * the device flags back before it returns, so it cannot be recorded into a
 * stream capture.
 * Errors: EINVAL (bad arguments; nz > 32767; a grid whose scratch would
 * exceed PDRT_STATIC_SCRATCH_BYTES, with the needed size in the message; a
 * NaN or infinite leaf, jaw or MU value found on the device, in which case
 * the dose is not valid), EDEVICE, ECUDA.  Calls no cudaMalloc/cudaFree.
 */
#define PDRT_STATIC_SCRATCH_BYTES (64u << 20)
pdrt_status pdrt_cp_dose_static(const float *red_dev, int32_t nx, int32_t ny, int32_t nz,
                                double sx, double sy, double sz, const double origin_mm[3],
                                const double iso_mm[3], double gantry_deg, const pdrt_machine *m,
                                const float *leaves_dev, const float *jaws_dev,
                                const float *mu_dev, float *dose_dev, pdrt_stream_t stream);

/*
 * Control points per pass (1 .. the count chosen at upload; the scratch was
 * sized for that count).  Fewer points per pass keep each pass's beam-frame
 * dose closer to L2; more points mean fewer launches.  Host only.
 * Errors: EINVAL (NULL plan, chunk_cp outside 1 .. the upload's count).
 */
pdrt_status pdrt_plan_set_chunk(pdrt_plan_t p, int32_t chunk_cp);

/*
 * Tensor-core tile shape: kernel rows per operand phase of the forward and
 * adjoint convolution (1..4; sets the shared memory per CTA and so the CTAs
 * per SM).  The upload picks, per direction, the deepest phase that keeps the
 * most CTAs per SM.  Errors: EINVAL (tensor-core path unavailable, or a phase
 * outside 1..4 or that does not fit).  Host only.
 */
pdrt_status pdrt_plan_set_tc_phase(pdrt_plan_t p, int32_t phase_forward, int32_t phase_adjoint);

/*
 * Autotuner: times forward (+ adjoint if dose_grad_dev != NULL) passes of the
 * plan with CUDA events on `stream` and keeps the fastest schedule, searched
 * one coordinate at a time from the upload's choice: the convolution path
 * (FFT with tensor-core overflow, tensor cores alone or FP32 SIMT) and the
 * FFT size limit, then the tensor-core tile shape of each
 * direction (kernel rows per operand phase, 1..4, which sets the shared
 * memory and so the CTAs per SM), then the control points per pass (the
 * uploaded count, 1/2 and 1/4 of it).  Output buffers are overwritten.
 * Synchronous.
 */
typedef struct {
    int32_t tensor_cores;        /* chosen convolution path */
    int32_t chunk_cp;            /* chosen control points per pass */
    float best_ms;               /* time of the chosen schedule */
    int32_t n_candidates;        /* schedules timed */
    int32_t phase[2];            /* tensor-core kernel rows per operand phase (forward, adjoint) */
    int32_t tc_ctas_per_sm[2];   /* resulting tensor-core CTAs per SM (forward, adjoint) */
    int32_t fft_pmax;            /* chosen FFT size limit (0: FFT convolution off) */
} pdrt_tune_result;
pdrt_status pdrt_plan_autotune(pdrt_grid_t g, pdrt_plan_t p, const float *leaves_dev,
                               const float *jaws_dev, const float *mu_dev, float *dose_dev,
                               const float *dose_grad_dev, float *dleaves_dev, float *djaws_dev,
                               float *dmu_dev, pdrt_stream_t stream, pdrt_tune_result *out);

/*
 * Batched launch (Sec. 2.2: the beam sequence is organised for batched
 * operation).  Records the forward dose -- and the adjoint for every i with
 * dose_grad_dev[i] != NULL -- of n independent plans into ONE CUDA graph;
 * pdrt_batch_launch replays it with a single graph launch.  The graph runs in
 * rounds, round c covering the c-th pass of control points of every plan:
 * the FFT convolution of all FFT plans' (plan, control point, slice) items of
 * the round is ONE persistent launch pulling items from one work counter, the
 * gather (forward) and its transpose (adjoint) of every plan's pass are one
 * launch each, and the remaining per-plan kernels (projection, tables,
 * tensor-core overflow or convolution, magnification transpose, gradients)
 * run on n_branches parallel branches.
 * Each plan keeps the pass size (pdrt_plan_set_chunk) it had at creation.
 * Every array argument has n entries (device pointers as in pdrt_dose_forward
 * / pdrt_dose_backward); a plan may appear once per batch; plans, grids and
 * buffers must stay valid and unchanged while the batch exists.  Creation
 * allocates the batch's small device tables (plan descriptors, round
 * entries, counters), freed by pdrt_batch_destroy; a launch allocates
 * nothing.  Errors: EINVAL (NULL, n < 1, repeated plan, mismatched grid),
 * ECUDA.
 */
typedef struct pdrt_batch_s *pdrt_batch_t;
pdrt_status pdrt_batch_create(pdrt_batch_t *out, int32_t n, const pdrt_grid_t *grids,
                              const pdrt_plan_t *plans, const float *const *leaves_dev,
                              const float *const *jaws_dev, const float *const *mu_dev,
                              float *const *dose_dev, const float *const *dose_grad_dev,
                              float *const *dleaves_dev, float *const *djaws_dev,
                              float *const *dmu_dev, int32_t n_branches, pdrt_stream_t stream);
pdrt_status pdrt_batch_launch(pdrt_batch_t b, pdrt_stream_t stream);
/* Synchronises `stream`; ms_out[i] = completion time of plan i in the last
 * launch, measured from the start of that launch (CUDA events in the graph).
 * Errors: EINVAL (NULL argument), ECUDA (no launch yet, or a fault). */
pdrt_status pdrt_batch_plan_times(pdrt_batch_t b, pdrt_stream_t stream, float *ms_out);
/* Number of kernel nodes in the batch's graph (kernels run per launch). */
int64_t pdrt_batch_kernels(pdrt_batch_t b);
/* Control points per pass of plan i in the batch (0 if b is NULL or i is out
 * of range).  A plan's dose and gradients equal, bit for bit, those of
 * pdrt_dose_forward / pdrt_dose_backward at this pass size. */
int32_t pdrt_batch_pass_cp(pdrt_batch_t b, int32_t i);
void pdrt_batch_destroy(pdrt_batch_t b);

/* Number of kernels this library has launched since it was loaded. */
int64_t pdrt_launch_count(void);

/* Message of the last failed call on this thread ("" if none). */
const char *pdrt_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PDRT_H */
