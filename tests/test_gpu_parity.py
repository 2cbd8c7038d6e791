"""GPU (sm_103a, FP32) vs FP64 oracle parity, through the C ABI.

Bars (FP32 path vs FP64 oracle): dose max |dD| <= 1e-4 * max D;
gradients ||dg||_inf <= 1e-3 * ||g||_inf per parameter class (leaves, jaws, MU).
Inputs are seeded synthetic workloads (paper_2512_18863_gb300.synth); no
expected value comes from the CUDA path.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2512_18863_gb300 import synth as S
from paper_2512_18863_gb300.engine import DoseEngine

pytestmark = pytest.mark.gpu

DOSE_TOL = 1e-4
GRAD_TOL = 1e-3


def _engine(w, **kw):
    return DoseEngine(w.phantom, w.machine, w.plan.gantry_deg, w.plan.iso, **kw)


def _gpu_dose(w, leaves=None, jaws=None, mu=None, **kw):
    eng = _engine(w, **kw)
    d = eng.forward(w.plan.leaves if leaves is None else leaves,
                    w.plan.jaws if jaws is None else jaws,
                    w.plan.mu if mu is None else mu)
    out = d.cpu().numpy().astype(np.float64)
    eng.close()
    return out


def _assert_dose(gpu, ref, tol=DOSE_TOL):
    err = np.abs(gpu - ref).max()
    assert err <= tol * ref.max(), f"max |dD| = {err:.3e} vs {tol} * {ref.max():.4e}"


def _assert_grad(gpu, ref, name):
    scale = np.abs(ref).max()
    err = np.abs(gpu - ref).max()
    assert err <= GRAD_TOL * scale, f"{name}: |dg|_inf = {err:.3e} vs {GRAD_TOL} * {scale:.4e}"


# ---------------------------------------------------------------------------
# forward
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("conv", ["fft", "tc", "simt"])
def test_water_static_10x10_matches_oracle_and_closed_form(conv):
    w = S.water_static_64()
    gpu = _gpu_dose(w, conv=conv)
    ref = O.Model(w.phantom, w.machine, w.plan).dose()
    _assert_dose(gpu, ref)
    iy = np.arange(64)
    T = np.interp((iy + 0.5) * 2.5, np.arange(len(w.machine.t_table)) * w.machine.dz_t,
                  w.machine.t_table)
    cal = O.calibrate(w.machine, 2.5, 2.5)        # the workload's output factor (Sec. 2.4)
    closed = cal * 100.0 * T * (1000.0 / (1000.0 + (iy - 32) * 2.5)) ** 2
    np.testing.assert_allclose(gpu[32, :, 32], closed, rtol=2e-5)


@pytest.mark.parametrize("conv", ["fft", "tc", "simt"])
@pytest.mark.parametrize("n,spacing,n_cp,r_px,seed", [
    ((24, 40, 40), 3.0, 6, 4, 7),      # several CTA tiles per slice
    ((23, 37, 41), 3.0, 5, 3, 8),      # ragged, odd grid, nx != ny
    ((20, 33, 33), 4.0, 4, 10, 9),     # R = 10 px
    ((18, 30, 30), 4.0, 3, 21, 10),    # R = 21 px
    ((16, 28, 28), 5.0, 2, 44, 11),    # maximum radius: column tiles and input chunks
    ((40, 48, 48), 2.0, 3, 13, 12),    # 2 mm grid, R = 13
])
def test_pelvis_forward_matches_oracle(n, spacing, n_cp, r_px, seed, conv):
    w = S.small_pelvis(seed=seed, n=n, spacing=spacing, n_cp=n_cp, r_px=r_px)
    gpu = _gpu_dose(w, conv=conv)
    ref = O.Model(w.phantom, w.machine, w.plan).dose()
    assert ref.max() > 0
    _assert_dose(gpu, ref)


def test_pelvis_128_arc_subset_matches_oracle():
    """128x128x96 at 3 mm (kernel radius 4 cm): 8 control points spread
    around the 178-CP arc."""
    w = S.pelvis_arc_128()
    sel = np.arange(0, 178, 22)[:8]
    sub = S.Workload(w.name, w.phantom, w.machine,
                     S.Plan(w.plan.gantry_deg[sel], w.plan.iso, w.plan.leaves[sel],
                            w.plan.jaws[sel], w.plan.mu[sel]))
    gpu = _gpu_dose(sub)
    ref = O.Model(sub.phantom, sub.machine, sub.plan).dose()
    _assert_dose(gpu, ref)


def test_chunking_does_not_change_the_dose():
    """One CP per pass (tiny scratch budget) vs all CPs in one pass."""
    w = S.small_pelvis(n=(20, 36, 36), n_cp=7, r_px=5)
    a = _gpu_dose(w, scratch_budget_bytes=1)
    b = _gpu_dose(w)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-6 * b.max())


# ---------------------------------------------------------------------------
# gradients
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("conv", ["fft", "tc", "simt"])
@pytest.mark.parametrize("ste", [1, 0])
def test_gradients_match_oracle(ste, conv):
    w = S.small_pelvis(seed=21, n=(20, 36, 36), n_cp=5, r_px=6)
    w.machine.ste = ste
    w.plan.leaves[1, 30] = (2.1, 2.4)          # a pair under w_min: clamp active
    w.plan.mu[2] = 0.004                       # below eps_mu
    rng = np.random.default_rng(5)
    g = rng.standard_normal(w.phantom.shape)
    eng = _engine(w, conv=conv)
    dl, dj, dm = (t.cpu().numpy().astype(np.float64)
                  for t in eng.backward(w.plan.leaves, w.plan.jaws, w.plan.mu, g))
    rl, rj, rm = O.Model(w.phantom, w.machine, w.plan).dose_grad(g)
    _assert_grad(dl, rl, "leaves")
    _assert_grad(dj, rj, "jaws")
    _assert_grad(dm, rm, "mu")
    eng.close()


def _assert_case(w, conv, seed):
    eng = _engine(w, conv=conv)
    model = O.Model(w.phantom, w.machine, w.plan)
    gpu = eng.forward(w.plan.leaves, w.plan.jaws, w.plan.mu).cpu().numpy().astype(np.float64)
    ref = model.dose()
    assert ref.max() > 0
    _assert_dose(gpu, ref)
    g = np.random.default_rng(seed).standard_normal(w.phantom.shape)
    dl, dj, dm = (t.cpu().numpy().astype(np.float64)
                  for t in eng.backward(w.plan.leaves, w.plan.jaws, w.plan.mu, g))
    rl, rj, rm = model.dose_grad(g)
    _assert_grad(dl, rl, "leaves")
    _assert_grad(dj, rj, "jaws")
    _assert_grad(dm, rm, "mu")
    eng.close()


@pytest.mark.parametrize("conv", ["fft", "tc", "simt"])
def test_zero_radius_kernel_matches_oracle(conv):
    """R = 0: a one-tap lateral kernel (on the tensor cores a single operand
    phase and one issuer per direction)."""
    _assert_case(S.small_pelvis(seed=23, n=(18, 32, 32), n_cp=4, r_px=0), conv, 6)


@pytest.mark.parametrize("conv", ["fft", "tc", "simt"])
def test_field_wider_than_64_pixels_across_leaf_pairs_matches_oracle(conv):
    """A field 18 cm long along the leaf-pair axis on 2.5 mm pixels: the
    adjoint's output columns exceed 64, so its tensor-core tiles run with one
    issuing warp and seven building warps."""
    m = S.machine_model(1011, r_px=3)
    ph = S.water_phantom((80, 32, 32), (2.5, 2.5, 2.5))
    plan = S.static_field(m, gantry_deg=30.0, half_x=20.0, half_y=90.0)
    _assert_case(S.Workload("wide_v", ph, m, plan), conv, 7)


def test_autograd_function_matches_oracle():
    """DoseFn inside a torch graph: quadratic objective on the PTV and an OAR."""
    w = S.small_pelvis(seed=22, n=(20, 36, 36), n_cp=4, r_px=5)
    eng = _engine(w)
    dev = eng.device
    leaves = torch.tensor(w.plan.leaves, dtype=torch.float32, device=dev, requires_grad=True)
    jaws = torch.tensor(w.plan.jaws, dtype=torch.float32, device=dev, requires_grad=True)
    mu = torch.tensor(w.plan.mu, dtype=torch.float32, device=dev, requires_grad=True)
    ptv = torch.tensor(w.phantom.masks["ptv"], device=dev, dtype=torch.float32)
    D = eng(leaves, jaws, mu)
    loss = ((D - 2.0) ** 2 * ptv).sum() + 0.1 * (D ** 2 * (1 - ptv)).sum()
    loss.backward()
    mod = O.Model(w.phantom, w.machine, w.plan)
    Dr = mod.dose()
    pm = w.phantom.masks["ptv"].astype(np.float64)
    g = 2 * (Dr - 2.0) * pm + 0.2 * Dr * (1 - pm)      # dL/dD from the oracle's own dose
    rl, rj, rm = mod.dose_grad(g)
    _assert_grad(leaves.grad.cpu().numpy(), rl, "leaves")
    _assert_grad(jaws.grad.cpu().numpy(), rj, "jaws")
    _assert_grad(mu.grad.cpu().numpy(), rm, "mu")
    eng.close()


def test_row_tiles_of_64_and_128_rows_match_oracle():
    """Support boxes whose heights straddle 64 and 128 rows: the tensor-core
    convolution's M = 64 and M = 128 row tiles, a 128-row tile followed by a
    last tile of at most 64 rows, and column tiles with one and with two
    MMA issuers.  Water, 100 x 100 x 16 voxels of 1 x 1 x 2 mm (lattice rows
    along x at 1 mm), R = 4 px; four control points with x half-widths 30,
    33, 63 and 66 mm, so that over the magnification range of the lattice
    (0.93..1.08) the support boxes are 56..65, 62..71, 118..136 and 123..142
    rows high (the forward's output boxes 2R = 8 rows more).  Dose and
    gradients on the oracle's bars."""
    m = S.machine_model(1010, r_px=4)
    ph = S.water_phantom((16, 100, 100), (1.0, 1.0, 2.0))
    fields = [S.static_field(m, gantry_deg=37.0 * q, half_x=h, half_y=14.0, mu=80.0 + 10 * q)
              for q, h in enumerate([30.0, 33.0, 63.0, 66.0])]
    plan = S.Plan(np.concatenate([f.gantry_deg for f in fields]), fields[0].iso,
                  np.concatenate([f.leaves for f in fields]), np.concatenate([f.jaws for f in fields]),
                  np.concatenate([f.mu for f in fields]))
    w = S.Workload("water100x100x16_row_tiles", ph, m, plan)
    mod = O.Model(w.phantom, w.machine, w.plan)
    ref = mod.dose()
    eng = _engine(w)
    d = eng.forward(plan.leaves, plan.jaws, plan.mu).cpu().numpy().astype(np.float64)
    _assert_dose(d, ref)
    g = np.random.default_rng(31).standard_normal(ph.shape)
    dl, dj, dm = (t.cpu().numpy().astype(np.float64) for t in eng.backward(plan.leaves, plan.jaws, plan.mu, g))
    assert eng.status_flags() == 0
    eng.close()
    rl, rj, rm = mod.dose_grad(g)
    _assert_grad(dl, rl, "leaves")
    _assert_grad(dj, rj, "jaws")
    _assert_grad(dm, rm, "mu")


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
def test_closed_jaws_give_zero_dose_and_gradient():
    w = S.small_pelvis(n=(16, 24, 24), n_cp=3, r_px=3)
    w.machine.wmin_jaw = 0.0
    jaws = w.plan.jaws.copy()
    jaws[:] = (5.0, 5.0, -3.0, -3.0)
    eng = _engine(w)
    d = eng.forward(w.plan.leaves, jaws, w.plan.mu)
    assert float(d.abs().max()) == 0.0
    g = np.ones(w.phantom.shape)
    dl, dj, dm = eng.backward(w.plan.leaves, jaws, w.plan.mu, g)
    assert float(dl.abs().max()) == 0.0 and float(dm.abs().max()) == 0.0
    eng.close()


def test_field_larger_than_lattice_and_single_cp():
    w = S.small_pelvis(n=(16, 24, 24), n_cp=1, r_px=4)
    w.plan.jaws[0] = (-300.0, 300.0, -300.0, 300.0)
    w.plan.leaves[0, :, 0] = -250.0
    w.plan.leaves[0, :, 1] = 250.0
    gpu = _gpu_dose(w)
    ref = O.Model(w.phantom, w.machine, w.plan).dose()
    _assert_dose(gpu, ref)


def test_tensor_and_simt_paths_match_oracle_on_arc_subset():
    """128x128x96 @ 3 mm, R = 13: the convolution paths against the oracle,
    and no device flag (timeout, capacity) raised."""
    w = S.pelvis_arc_128()
    sel = np.arange(3, 178, 12)
    sub = S.Workload(w.name, w.phantom, w.machine,
                     S.Plan(w.plan.gantry_deg[sel], w.plan.iso, w.plan.leaves[sel],
                            w.plan.jaws[sel], w.plan.mu[sel]))
    ref = O.Model(sub.phantom, sub.machine, sub.plan).dose()
    for conv in ("fft", "tc", "simt"):
        eng = _engine(sub, conv=conv)
        d = eng.forward(sub.plan.leaves, sub.plan.jaws, sub.plan.mu).cpu().numpy()
        assert eng.status_flags() == 0
        eng.close()
        _assert_dose(d.astype(np.float64), ref)


@pytest.mark.parametrize("pmax", [32, 48, 60, 64, 72, 80, 90, 96, 100, 108, 120, 128, 144, 160, 192])
def test_fft_size_limits_and_overflow_match_oracle(pmax):
    """The FFT convolution at every supported size limit: slices whose padded
    sizes exceed it go to the tensor cores through the overflow list (at the
    small limits most of them), the rest by FFT; dose and gradients against
    the oracle, and the work counters account for every (slice, direction)."""
    w = S.small_pelvis(seed=27, n=(26, 44, 44), spacing=3.0, n_cp=4, r_px=9)
    eng = _engine(w, conv="fft", fft_pmax=pmax)
    assert eng.info["fft_pmax"] == pmax
    d = eng.forward(w.plan.leaves, w.plan.jaws, w.plan.mu).cpu().numpy().astype(np.float64)
    g = np.random.default_rng(pmax).standard_normal(w.phantom.shape).astype(np.float32)
    dl, dj, dm = (t.cpu().numpy().astype(np.float64)
                  for t in eng.backward(w.plan.leaves, w.plan.jaws, w.plan.mu, g))
    work = eng.work()
    assert eng.status_flags() == 0
    eng.close()
    assert work["fft_slices"] + work["tc_slices"] == 2 * work["active_slices"]
    if pmax <= 32:
        assert work["tc_slices"] > 0
    if pmax >= 96:
        assert work["tc_slices"] == 0 and work["fft_flops"] > 0
    mod = O.Model(w.phantom, w.machine, w.plan)
    _assert_dose(d, mod.dose())
    rl, rj, rm = mod.dose_grad(g.astype(np.float64))
    _assert_grad(dl, rl, "leaves")
    _assert_grad(dj, rj, "jaws")
    _assert_grad(dm, rm, "mu")


def test_fft_size_144_radix9_matches_oracle():
    """Slices whose padded u size falls in (128, 144]: with the size limit at
    128 they overflow to the tensor cores, at 144 they go by FFT (rows of
    72 = 8 x 9, the radix-9 passes; the wider ones stay on the tensor cores);
    dose and gradients of both against the oracle."""
    w = S.small_pelvis(seed=29, n=(16, 160, 160), spacing=2.0, n_cp=2, r_px=44,
                       ptv_radii=(46.0, 40.0, 12.0))
    g = np.random.default_rng(144).standard_normal(w.phantom.shape).astype(np.float32)
    out = {}
    for pmax in (128, 144):
        eng = _engine(w, conv="fft", fft_pmax=pmax)
        assert eng.info["fft_pmax"] == pmax
        d = eng.forward(w.plan.leaves, w.plan.jaws, w.plan.mu).cpu().numpy().astype(np.float64)
        grads = [t.cpu().numpy().astype(np.float64)
                 for t in eng.backward(w.plan.leaves, w.plan.jaws, w.plan.mu, g)]
        out[pmax] = (d, grads, eng.work())
        assert eng.status_flags() == 0
        eng.close()
    assert out[144][2]["tc_slices"] < out[128][2]["tc_slices"]
    assert out[144][2]["fft_slices"] > out[128][2]["fft_slices"]
    mod = O.Model(w.phantom, w.machine, w.plan)
    ref = mod.dose()
    rgrads = mod.dose_grad(g.astype(np.float64))
    for pmax in (128, 144):
        d, grads, _ = out[pmax]
        _assert_dose(d, ref)
        for gg, rr, name in zip(grads, rgrads, ("leaves", "jaws", "mu")):
            _assert_grad(gg, rr, name)


def test_spectrum_memo_changes_no_result():
    """The kernel-spectrum memo: a plan with it (the default) and one without
    give bit-identical doses and gradients over a call sequence that fills it
    (forward), takes from it (adjoint, repeated calls), meets other padded
    sizes (wider jaws: those slices are computed again and stored) and is
    reset."""
    w = S.small_pelvis(seed=31, n=(20, 36, 36), n_cp=5, r_px=6)
    on, off = _engine(w), _engine(w)
    off.set_spectrum_memo(False)
    assert on.info["spectrum_memo_bytes"] > 0 and on.info["spectrum_memo_pmax"] == on.info["fft_pmax"]
    assert off.info["spectrum_memo_bytes"] == 0
    g = np.random.default_rng(31).standard_normal(w.phantom.shape).astype(np.float32)
    wide = w.plan.jaws.copy()
    wide[:, 0] -= 12.0
    wide[:, 1] += 12.0
    seq = [w.plan.jaws, w.plan.jaws, wide, w.plan.jaws, None, w.plan.jaws]
    for jaws in seq:
        if jaws is None:
            on.reset_spectrum_memo()
            continue
        d1 = on.forward(w.plan.leaves, jaws, w.plan.mu).clone()
        d0 = off.forward(w.plan.leaves, jaws, w.plan.mu).clone()
        assert torch.equal(d1, d0)
        for a, b in zip(on.backward(w.plan.leaves, jaws, w.plan.mu, g),
                        off.backward(w.plan.leaves, jaws, w.plan.mu, g)):
            assert torch.equal(a, b)
    assert on.status_flags() == 0
    ref = O.Model(w.phantom, w.machine, w.plan).dose()
    _assert_dose(on.forward(w.plan.leaves, w.plan.jaws, w.plan.mu).cpu().numpy().astype(np.float64), ref)
    on.close()
    off.close()


def test_plan_without_control_points_is_rejected():
    """An arc with no control points is a shape error of the upload (ESHAPE),
    not an empty dose."""
    from paper_2512_18863_gb300 import _lib
    w = S.small_pelvis(n=(16, 24, 24), n_cp=1, r_px=3)
    with pytest.raises(_lib.PdrtError) as e:
        DoseEngine(w.phantom, w.machine, np.zeros(0), w.plan.iso)
    assert e.value.status == 2


def test_plan_of_another_grid_is_rejected():
    """A plan handle is bound to the grid it was uploaded for: forward and
    backward with another grid's handle fail with EINVAL before any launch,
    and the engines stay usable."""
    from paper_2512_18863_gb300 import _lib
    w = S.small_pelvis(n=(16, 24, 24), n_cp=2, r_px=3)
    a, b = _engine(w), _engine(w)
    leaves, jaws, mu = a._params(w.plan.leaves, w.plan.jaws, w.plan.mu)
    out = torch.empty(a.shape, dtype=torch.float32, device=a.device)
    stream = torch.cuda.current_stream().cuda_stream
    with pytest.raises(_lib.PdrtError) as e:
        _lib.pdrt_dose_forward(a._grid, b._plan, leaves.data_ptr(), jaws.data_ptr(),
                               mu.data_ptr(), out.data_ptr(), stream)
    assert e.value.status == 1
    g = torch.ones(a.shape, dtype=torch.float32, device=a.device)
    grads = [torch.empty_like(t) for t in (leaves, jaws, mu)]
    with pytest.raises(_lib.PdrtError) as e:
        _lib.pdrt_dose_backward(b._grid, a._plan, leaves.data_ptr(), jaws.data_ptr(),
                                mu.data_ptr(), g.data_ptr(), *(t.data_ptr() for t in grads), stream)
    assert e.value.status == 1
    da = a.forward(w.plan.leaves, w.plan.jaws, w.plan.mu)
    db = b.forward(w.plan.leaves, w.plan.jaws, w.plan.mu)
    assert torch.equal(da, db) and float(da.max()) > 0
    a.close()
    b.close()


def test_nan_input_is_flagged():
    w = S.small_pelvis(n=(16, 24, 24), n_cp=2, r_px=3)
    eng = _engine(w)
    leaves = w.plan.leaves.copy()
    leaves[1, 5, 0] = np.nan
    eng.forward(leaves, w.plan.jaws, w.plan.mu)
    assert eng.status_flags() & 1
    eng.forward(w.plan.leaves, w.plan.jaws, w.plan.mu)
    assert eng.status_flags() == 0
    eng.close()


def test_forward_and_backward_are_deterministic():
    w = S.small_pelvis(n=(20, 32, 32), n_cp=4, r_px=5)
    eng = _engine(w)
    assert eng.info["tensor_cores"] == 1
    a = eng.forward(w.plan.leaves, w.plan.jaws, w.plan.mu).clone()
    b = eng.forward(w.plan.leaves, w.plan.jaws, w.plan.mu).clone()
    assert torch.equal(a, b)
    g = torch.rand(w.phantom.shape, device=eng.device)
    r1 = [t.clone() for t in eng.backward(w.plan.leaves, w.plan.jaws, w.plan.mu, g)]
    r2 = eng.backward(w.plan.leaves, w.plan.jaws, w.plan.mu, g)
    assert all(torch.equal(x, y) for x, y in zip(r1, r2))
    eng.close()


# ---------------------------------------------------------------------------
# full size (256x256x160, 2 x 178 CPs) in the benchmark's launch configuration
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def c3():
    return S.pelvis_two_arc_256(r_cm=4.0)


def _subplan(w, sel):
    return S.Workload(w.name, w.phantom, w.machine,
                      S.Plan(w.plan.gantry_deg[sel], w.plan.iso, w.plan.leaves[sel],
                             w.plan.jaws[sel], w.plan.mu[sel]))


@pytest.mark.parametrize("r_cm,n_sample", [(2.0, 12), (4.0, 12), (8.0, 8)])
def test_full_size_sampled_against_oracle(r_cm, n_sample):
    """Every kernel radius of the two-arc configuration at full grid size
    (256 x 256 x 160 at 2 mm): n_sample control points spread evenly over
    both arcs (the second arc runs backwards), the GPU in the benchmark's
    launch configuration (tensor cores, default schedule) against the oracle:
    the dose and all three gradient classes of <g, D> for a random g."""
    w = S.pelvis_two_arc_256(r_cm=r_cm)
    assert w.machine.r_px == int(round(r_cm * 5))
    sel = np.unique(np.linspace(3, w.plan.n_cp - 4, n_sample).round().astype(int))
    assert len(sel) == n_sample and sel.min() < 178 <= sel.max()
    sub = _subplan(w, sel)
    eng = _engine(sub)
    assert eng.info["tensor_cores"] == 1
    gpu = eng.forward(sub.plan.leaves, sub.plan.jaws, sub.plan.mu).cpu().numpy().astype(np.float64)
    g = np.random.default_rng(int(r_cm * 10)).standard_normal(sub.phantom.shape).astype(np.float32)
    dl, dj, dm = (t.cpu().numpy().astype(np.float64)
                  for t in eng.backward(sub.plan.leaves, sub.plan.jaws, sub.plan.mu, g))
    cal = eng.cal
    eng.close()
    mod = O.Model(sub.phantom, sub.machine, sub.plan)
    assert abs(cal - mod.cal) <= 1e-5 * mod.cal
    _assert_dose(gpu, mod.dose())
    rl, rj, rm = mod.dose_grad(g.astype(np.float64))
    _assert_grad(dl, rl, "leaves")
    _assert_grad(dj, rj, "jaws")
    _assert_grad(dm, rm, "mu")


def test_full_size_arc_sum_is_linear(c3):
    """The whole 356-CP dose equals the sum of its two arcs (linearity of
    Eq. D_total; holds at any size, checked GPU against GPU)."""
    full = _gpu_dose(c3)
    a = _gpu_dose(_subplan(c3, np.arange(178)))
    b = _gpu_dose(_subplan(c3, np.arange(178, 356)))
    np.testing.assert_allclose(full, a + b, rtol=0, atol=1e-5 * full.max())


def test_full_size_gradient_vs_central_differences(c3):
    """Two-arc plan at full size (356 CPs): the adjoint on 64 random
    differentiable parameters (leaf edges, jaw edges, MUs away from kinks) of
    8 random control points against central differences (0.01 mm / 0.01 MU)
    of L = <g, D>.  D is a sum over control points (Eq. D_total), so the
    difference of L is that of the perturbed control point's own dose: it is
    taken on a one-CP plan (L summed in FP64), which keeps the FP32 rounding
    of the 356-term dose sum out of the 0.01 mm difference."""
    import torch
    from tests.test_oracle_adjoint import _pick_params
    rng = np.random.default_rng(21)
    eng = _engine(c3)
    g = rng.standard_normal(c3.phantom.shape).astype(np.float32)
    grads = dict(zip(("leaves", "jaws", "mu"),
                     (t.cpu().numpy().astype(np.float64)
                      for t in eng.backward(c3.plan.leaves, c3.plan.jaws, c3.plan.mu, g))))
    eng.close()
    scale = {k: np.abs(v).max() for k, v in grads.items()}
    cps = np.sort(rng.choice(c3.plan.n_cp, 8, replace=False))
    sub8 = _subplan(c3, cps)
    picks = _pick_params(sub8, O.Model(sub8.phantom, sub8.machine, sub8.plan), rng, 64)
    assert len(picks) == 64
    h = 0.01
    for j, b in enumerate(cps):
        one = _subplan(c3, np.array([b]))
        e1 = _engine(one)
        gt = torch.tensor(g, device=e1.device, dtype=torch.float64)
        base = {"leaves": one.plan.leaves, "jaws": one.plan.jaws, "mu": one.plan.mu}
        for name, ix in picks:
            if ix[0] != j:
                continue
            ix1 = (0,) + tuple(ix[1:])
            vals = []
            for sgn in (+1, -1):
                p = {k: v.copy() for k, v in base.items()}
                p[name][ix1] += sgn * h
                D = e1.forward(p["leaves"], p["jaws"], p["mu"])
                vals.append(float((D.double() * gt).sum()))
            fd = (vals[0] - vals[1]) / (2 * h)
            an = grads[name][(b,) + tuple(ix[1:])]
            assert abs(fd - an) <= 1e-3 * scale[name], (name, b, ix, fd, an, scale[name])
        e1.close()
