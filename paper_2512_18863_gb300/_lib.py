"""Thin ctypes binding of the C ABI in include/pdrt.h (argument marshalling only).

The Python functions carry the C names.  Device buffers are passed as raw
pointers (int), streams as cudaStream_t values; every non-OK status raises
PdrtError with pdrt_last_error().  There is no fallback: if the library is not
built, load() raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

MAX_PAIRS = 160
MAX_RADIUS_PX = 44
MAX_DEPTH_TABLE = 4096
MAX_HU_POINTS = 32
NUM_KERNELS = 12
FLAG_NAN_INPUT = 1
FLAG_CAPACITY = 2
FLAG_TIMEOUT = 4

STATUS = {0: "PDRT_OK", 1: "PDRT_EINVAL", 2: "PDRT_ESHAPE", 3: "PDRT_ECUDA", 4: "PDRT_ENOMEM",
          5: "PDRT_EDEVICE"}


class PdrtError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class pdrt_machine(C.Structure):
    _fields_ = [("sid_mm", C.c_double), ("n_pairs", C.c_int32),
                ("leaf_bounds_mm", C.c_double * (MAX_PAIRS + 1)), ("tau", C.c_double),
                ("wmin_leaf_mm", C.c_double), ("wmin_jaw_mm", C.c_double),
                ("f_leaf_mm", C.c_double), ("f_jaw_mm", C.c_double), ("eps_mu", C.c_double),
                ("kernel_radius_px", C.c_int32), ("kernel_alpha", (C.c_double * 3) * 3),
                ("kernel_beta", (C.c_double * 3) * 3), ("n_depth", C.c_int32),
                ("depth_step_mm", C.c_double), ("depth_dose", C.c_double * MAX_DEPTH_TABLE),
                ("cal", C.c_double), ("ste", C.c_int32),
                ("pen_fwhm_u_mm", C.c_double), ("pen_fwhm_v_mm", C.c_double),
                ("off_axis", C.c_double * 3), ("collimator_deg", C.c_double)]


class pdrt_plan_info(C.Structure):
    _fields_ = [("nu", C.c_int32), ("nv", C.c_int32), ("nw", C.c_int32),
                ("cu", C.c_double), ("cv", C.c_double), ("cw", C.c_double),
                ("n_cp", C.c_int32), ("chunk_cp", C.c_int32), ("scratch_bytes", C.c_size_t),
                ("tensor_cores", C.c_int32), ("tc_ctas_per_sm", C.c_int32 * 2),
                ("simt_ctas_per_sm", C.c_int32 * 2), ("tc_phase", C.c_int32 * 2),
                ("fft_pmax", C.c_int32), ("fft_ctas_per_sm", C.c_int32 * 2),
                ("spectrum_memo_pmax", C.c_int32), ("spectrum_memo_bytes", C.c_size_t)]


class pdrt_work(C.Structure):
    _fields_ = [("active_slices", C.c_int64), ("support_points", C.c_int64),
                ("region_points", C.c_int64), ("taps", C.c_int64), ("conv_flops", C.c_double),
                ("mma_flops", C.c_double), ("fft_flops", C.c_double), ("fft_slices", C.c_int64),
                ("tc_slices", C.c_int64)]


class pdrt_tune_result(C.Structure):
    _fields_ = [("tensor_cores", C.c_int32), ("chunk_cp", C.c_int32), ("best_ms", C.c_float),
                ("n_candidates", C.c_int32), ("phase", C.c_int32 * 2), ("tc_ctas_per_sm", C.c_int32 * 2),
                ("fft_pmax", C.c_int32)]


class pdrt_profile(C.Structure):
    _fields_ = [("name", C.c_char_p * NUM_KERNELS), ("launches", C.c_int64 * NUM_KERNELS),
                ("total_ms", C.c_double * NUM_KERNELS), ("overflow", C.c_int32)]


_VP = C.c_void_p
_SIG = {
    "pdrt_grid_create": (C.c_int, [C.POINTER(_VP), _VP, C.c_int32, C.c_int32, C.c_int32, C.c_double,
                                   C.c_double, C.c_double, C.POINTER(C.c_double),
                                   C.POINTER(C.c_double), C.c_int32, _VP]),
    "pdrt_grid_destroy": (None, [_VP]),
    "pdrt_plan_upload": (C.c_int, [C.POINTER(_VP), _VP, C.c_int32, C.POINTER(C.c_double),
                                   C.POINTER(C.c_double), C.POINTER(pdrt_machine), C.c_size_t, _VP]),
    "pdrt_plan_destroy": (None, [_VP]),
    "pdrt_dose_forward": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "pdrt_dose_backward": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "pdrt_plan_get_info": (C.c_int, [_VP, C.POINTER(pdrt_plan_info)]),
    "pdrt_plan_set_spectrum_memo": (C.c_int, [_VP, C.c_int32]),
    "pdrt_plan_reset_spectrum_memo": (C.c_int, [_VP, _VP]),
    "pdrt_plan_set_tensor_cores": (C.c_int, [_VP, C.c_int32]),
    "pdrt_plan_status": (C.c_int, [_VP, _VP, C.POINTER(C.c_uint32)]),
    "pdrt_plan_work": (C.c_int, [_VP, _VP, C.POINTER(pdrt_work)]),
    "pdrt_profile_enable": (C.c_int, [_VP, C.c_int32]),
    "pdrt_profile_read": (C.c_int, [_VP, _VP, C.POINTER(pdrt_profile)]),
    "pdrt_cp_dose_static": (C.c_int, [_VP, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double,
                                      C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                      C.c_double, C.POINTER(pdrt_machine), _VP, _VP, _VP, _VP, _VP]),
    "pdrt_calibrate": (C.c_int, [C.POINTER(pdrt_machine), C.c_double, C.c_double, C.c_double,
                                 C.c_double, C.POINTER(C.c_double), _VP]),
    "pdrt_plan_set_chunk": (C.c_int, [_VP, C.c_int32]),
    "pdrt_plan_set_tc_phase": (C.c_int, [_VP, C.c_int32, C.c_int32]),
    "pdrt_plan_set_fft": (C.c_int, [_VP, C.c_int32]),
    "pdrt_plan_autotune": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                                     C.POINTER(pdrt_tune_result)]),
    "pdrt_batch_create": (C.c_int, [C.POINTER(_VP), C.c_int32, C.POINTER(_VP), C.POINTER(_VP),
                                    C.POINTER(_VP), C.POINTER(_VP), C.POINTER(_VP), C.POINTER(_VP),
                                    C.POINTER(_VP), C.POINTER(_VP), C.POINTER(_VP), C.POINTER(_VP),
                                    C.c_int32, _VP]),
    "pdrt_batch_launch": (C.c_int, [_VP, _VP]),
    "pdrt_batch_plan_times": (C.c_int, [_VP, _VP, C.POINTER(C.c_float)]),
    "pdrt_batch_kernels": (C.c_int64, [_VP]),
    "pdrt_batch_pass_cp": (C.c_int32, [_VP, C.c_int32]),
    "pdrt_batch_destroy": (None, [_VP]),
    "pdrt_launch_count": (C.c_int64, []),
    "pdrt_last_error": (C.c_char_p, []),
    # warm-start network (pdrt_cnn.h)
    "pdrt_cnn_param_count": (C.c_int64, []),
    "pdrt_cnn_create": (C.c_int, [C.POINTER(_VP), C.c_int32, _VP]),
    "pdrt_cnn_destroy": (None, [_VP]),
    "pdrt_cnn_set_params": (C.c_int, [_VP, _VP, _VP]),
    "pdrt_cnn_get_params": (C.c_int, [_VP, _VP, _VP]),
    "pdrt_cnn_forward": (C.c_int, [_VP, _VP, C.c_int32, _VP, _VP]),
    "pdrt_cnn_backward": (C.c_int, [_VP, C.c_int32, _VP, _VP, _VP]),
    "pdrt_cnn_train_step": (C.c_int, [_VP, _VP, _VP, C.c_int32, C.c_float, _VP, _VP]),
    "pdrt_cnn_read_activation": (C.c_int, [_VP, C.c_int32, C.c_int32, _VP, _VP]),
    "pdrt_cnn_status": (C.c_int, [_VP, _VP, C.POINTER(C.c_uint32)]),
    "pdrt_bev_project": (C.c_int, [_VP, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double,
                                   C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                   C.c_double, C.c_int32, C.POINTER(C.c_double), C.c_int32,
                                   C.c_double, C.c_double, C.c_double, _VP, _VP]),
}

_lock = threading.Lock()
_handle = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libpdrt.so (building it first if needed and allowed)."""
    global _handle
    with _lock:
        if _handle is None:
            path = _build.LIB
            if build_if_missing:
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"dose-engine library not built: {path} (run build())")
            h = C.CDLL(path)
            for name, (res, args) in _SIG.items():
                f = getattr(h, name)
                f.restype = res
                f.argtypes = args
            _handle = h
    return _handle


def _check(st):
    if st != 0:
        raise PdrtError(st, load().pdrt_last_error().decode())


def _dptr(a):
    return C.c_double(0) if a is None else (C.c_double * len(a))(*[float(x) for x in a])


def pdrt_last_error() -> str:
    return load().pdrt_last_error().decode()


def pdrt_launch_count() -> int:
    return int(load().pdrt_launch_count())


def pdrt_grid_create(hu_dev_ptr, nx, ny, nz, sx, sy, sz, origin_mm, hu_red_pairs, stream):
    out = _VP()
    pts = [float(x) for pair in hu_red_pairs for x in pair]
    _check(load().pdrt_grid_create(C.byref(out), _VP(hu_dev_ptr), int(nx), int(ny), int(nz),
                                   float(sx), float(sy), float(sz), _dptr(origin_mm), _dptr(pts),
                                   len(pts) // 2, _VP(stream)))
    return out.value


def pdrt_grid_destroy(grid):
    load().pdrt_grid_destroy(_VP(grid))


def pdrt_plan_upload(grid, gantry_deg, iso_mm, machine: pdrt_machine, scratch_budget_bytes, stream):
    out = _VP()
    _check(load().pdrt_plan_upload(C.byref(out), _VP(grid), len(gantry_deg), _dptr(gantry_deg),
                                   _dptr(iso_mm), C.byref(machine), int(scratch_budget_bytes),
                                   _VP(stream)))
    return out.value


def pdrt_plan_destroy(plan):
    load().pdrt_plan_destroy(_VP(plan))


def pdrt_dose_forward(grid, plan, leaves_ptr, jaws_ptr, mu_ptr, dose_ptr, stream):
    _check(load().pdrt_dose_forward(_VP(grid), _VP(plan), _VP(leaves_ptr), _VP(jaws_ptr),
                                    _VP(mu_ptr), _VP(dose_ptr), _VP(stream)))


def pdrt_dose_backward(grid, plan, leaves_ptr, jaws_ptr, mu_ptr, dose_grad_ptr, dleaves_ptr,
                       djaws_ptr, dmu_ptr, stream):
    _check(load().pdrt_dose_backward(_VP(grid), _VP(plan), _VP(leaves_ptr), _VP(jaws_ptr),
                                     _VP(mu_ptr), _VP(dose_grad_ptr), _VP(dleaves_ptr),
                                     _VP(djaws_ptr), _VP(dmu_ptr), _VP(stream)))


def pdrt_plan_set_tensor_cores(plan, enable):
    _check(load().pdrt_plan_set_tensor_cores(_VP(plan), 1 if enable else 0))


def pdrt_plan_get_info(plan) -> dict:
    info = pdrt_plan_info()
    _check(load().pdrt_plan_get_info(_VP(plan), C.byref(info)))
    out = {k: getattr(info, k) for k, _ in pdrt_plan_info._fields_}
    out["simt_ctas_per_sm"] = list(out["simt_ctas_per_sm"])
    out["tc_ctas_per_sm"] = list(out["tc_ctas_per_sm"])
    out["tc_phase"] = list(out["tc_phase"])
    out["fft_ctas_per_sm"] = list(out["fft_ctas_per_sm"])
    return out


def pdrt_plan_status(plan, stream) -> int:
    f = C.c_uint32(0)
    _check(load().pdrt_plan_status(_VP(plan), _VP(stream), C.byref(f)))
    return int(f.value)


def pdrt_plan_work(plan, stream) -> dict:
    w = pdrt_work()
    _check(load().pdrt_plan_work(_VP(plan), _VP(stream), C.byref(w)))
    return {k: getattr(w, k) for k, _ in pdrt_work._fields_}


def pdrt_profile_enable(plan, enable):
    _check(load().pdrt_profile_enable(_VP(plan), 1 if enable else 0))


def pdrt_profile_read(plan, stream) -> dict:
    p = pdrt_profile()
    _check(load().pdrt_profile_read(_VP(plan), _VP(stream), C.byref(p)))
    out = {}
    for k in range(NUM_KERNELS):
        out[p.name[k].decode()] = {"launches": int(p.launches[k]), "total_ms": float(p.total_ms[k])}
    out["_overflow"] = bool(p.overflow)
    return out


STATIC_SCRATCH_BYTES = 64 << 20


def pdrt_cp_dose_static(red_dev_ptr, nx, ny, nz, sx, sy, sz, origin_mm, iso_mm, gantry_deg,
                        machine: pdrt_machine, leaves_ptr, jaws_ptr, mu_ptr, dose_ptr, stream):
    """One control point's dose using the library's static scratch (no allocation)."""
    _check(load().pdrt_cp_dose_static(_VP(red_dev_ptr), int(nx), int(ny), int(nz), float(sx),
                                      float(sy), float(sz), _dptr(origin_mm), _dptr(iso_mm),
                                      float(gantry_deg), C.byref(machine), _VP(leaves_ptr),
                                      _VP(jaws_ptr), _VP(mu_ptr), _VP(dose_ptr), _VP(stream)))


def pdrt_calibrate(machine: pdrt_machine, sxy, sz, ref_mu, ref_gy, stream) -> float:
    """Output calibration factor of Sec. 2.4 computed by the library's kernels."""
    cal = C.c_double()
    _check(load().pdrt_calibrate(C.byref(machine), float(sxy), float(sz), float(ref_mu),
                                 float(ref_gy), C.byref(cal), _VP(stream)))
    return cal.value


def pdrt_plan_set_chunk(plan, chunk_cp):
    _check(load().pdrt_plan_set_chunk(_VP(plan), int(chunk_cp)))


def pdrt_plan_autotune(grid, plan, leaves_ptr, jaws_ptr, mu_ptr, dose_ptr, dose_grad_ptr,
                       dleaves_ptr, djaws_ptr, dmu_ptr, stream) -> dict:
    r = pdrt_tune_result()
    _check(load().pdrt_plan_autotune(_VP(grid), _VP(plan), _VP(leaves_ptr), _VP(jaws_ptr),
                                     _VP(mu_ptr), _VP(dose_ptr), _VP(dose_grad_ptr),
                                     _VP(dleaves_ptr), _VP(djaws_ptr), _VP(dmu_ptr), _VP(stream),
                                     C.byref(r)))
    out = {k: getattr(r, k) for k, _ in pdrt_tune_result._fields_}
    for k in ("phase", "tc_ctas_per_sm"):
        out[k] = list(out[k])
    return out


def _ptr_array(values):
    return (_VP * len(values))(*[_VP(x) for x in values])


def pdrt_batch_create(grids, plans, leaves, jaws, mu, dose, dose_grad, dleaves, djaws, dmu,
                      n_branches, stream):
    """All list arguments: one device pointer (int) per plan (None: no adjoint)."""
    out = _VP()
    n = len(plans)
    arr = lambda xs: None if xs is None else _ptr_array([0 if x is None else x for x in xs])
    _check(load().pdrt_batch_create(C.byref(out), n, _ptr_array(grids), _ptr_array(plans),
                                    arr(leaves), arr(jaws), arr(mu), arr(dose), arr(dose_grad),
                                    arr(dleaves), arr(djaws), arr(dmu), int(n_branches),
                                    _VP(stream)))
    return out.value


def pdrt_batch_launch(batch, stream):
    _check(load().pdrt_batch_launch(_VP(batch), _VP(stream)))


def pdrt_batch_plan_times(batch, n, stream):
    ms = (C.c_float * n)()
    _check(load().pdrt_batch_plan_times(_VP(batch), _VP(stream), ms))
    return list(ms)


def pdrt_batch_kernels(batch) -> int:
    return int(load().pdrt_batch_kernels(_VP(batch)))


def pdrt_batch_pass_cp(batch, i) -> int:
    return int(load().pdrt_batch_pass_cp(_VP(batch), int(i)))


def pdrt_batch_destroy(batch):
    load().pdrt_batch_destroy(_VP(batch))


def machine_struct(machine, cal=None) -> pdrt_machine:
    """Fill pdrt_machine from a synth.Machine-like object.  cal overrides the
    machine's output factor; a machine without one (cal None: calibrate) needs
    it given."""
    m = pdrt_machine()
    lb = list(machine.leaf_bounds)
    if len(lb) - 1 > MAX_PAIRS:
        raise ValueError("too many leaf pairs")
    tt = list(machine.t_table)
    if len(tt) > MAX_DEPTH_TABLE:
        raise ValueError("depth-dose table too long")
    m.sid_mm = float(machine.sid)
    m.n_pairs = len(lb) - 1
    for i, x in enumerate(lb):
        m.leaf_bounds_mm[i] = float(x)
    m.tau = float(machine.tau)
    m.wmin_leaf_mm = float(machine.wmin_leaf)
    m.wmin_jaw_mm = float(machine.wmin_jaw)
    m.f_leaf_mm = float(machine.f_leaf)
    m.f_jaw_mm = float(machine.f_jaw)
    m.eps_mu = float(machine.eps_mu)
    m.kernel_radius_px = int(machine.r_px)
    for c in range(3):
        for k in range(3):
            m.kernel_alpha[c][k] = float(machine.alpha[c][k])
            m.kernel_beta[c][k] = float(machine.beta[c][k])
    m.n_depth = len(tt)
    m.depth_step_mm = float(machine.dz_t)
    for i, x in enumerate(tt):
        m.depth_dose[i] = float(x)
    cal = machine.cal if cal is None else cal
    if cal is None:
        raise ValueError("the machine has no output factor: calibrate it (pdrt_calibrate) and pass cal")
    m.cal = float(cal)
    m.ste = int(machine.ste)
    m.pen_fwhm_u_mm = float(getattr(machine, "pen_fwhm_u", 0.0))
    m.pen_fwhm_v_mm = float(getattr(machine, "pen_fwhm_v", 0.0))
    m.off_axis[:] = [float(x) for x in getattr(machine, "off_axis", (1.0, 0.0, 0.0))]
    m.collimator_deg = float(getattr(machine, "collimator_deg", 0.0))
    return m


# ---------------------------------------------------------------------------
# warm-start network (pdrt_cnn.h): argument marshalling only
# ---------------------------------------------------------------------------
CNN_SIDE = 64
CNN_IN_CH = 3
CNN_OUT = 121


def pdrt_cnn_param_count() -> int:
    return int(load().pdrt_cnn_param_count())


def pdrt_cnn_create(batch_max, stream):
    out = _VP()
    _check(load().pdrt_cnn_create(C.byref(out), int(batch_max), _VP(stream)))
    return out.value


def pdrt_cnn_destroy(net):
    if net:
        load().pdrt_cnn_destroy(_VP(net))


def pdrt_cnn_set_params(net, params_dev, stream):
    _check(load().pdrt_cnn_set_params(_VP(net), _VP(params_dev), _VP(stream)))


def pdrt_cnn_get_params(net, params_dev, stream):
    _check(load().pdrt_cnn_get_params(_VP(net), _VP(params_dev), _VP(stream)))


def pdrt_cnn_forward(net, x_dev, n, y_dev, stream):
    _check(load().pdrt_cnn_forward(_VP(net), _VP(x_dev), int(n), _VP(y_dev), _VP(stream)))


def pdrt_cnn_backward(net, n, dy_dev, grads_dev, stream):
    _check(load().pdrt_cnn_backward(_VP(net), int(n), _VP(dy_dev), _VP(grads_dev), _VP(stream)))


def pdrt_cnn_train_step(net, x_dev, target_dev, n, lr, loss_dev, stream):
    _check(load().pdrt_cnn_train_step(_VP(net), _VP(x_dev), _VP(target_dev), int(n), float(lr),
                                      _VP(loss_dev), _VP(stream)))


def pdrt_cnn_read_activation(net, layer, n, dst_dev, stream):
    _check(load().pdrt_cnn_read_activation(_VP(net), int(layer), int(n), _VP(dst_dev), _VP(stream)))


def pdrt_cnn_status(net, stream) -> int:
    f = C.c_uint32(0)
    _check(load().pdrt_cnn_status(_VP(net), _VP(stream), C.byref(f)))
    return int(f.value)


def pdrt_bev_project(masks_dev, nx, ny, nz, spacing, origin, iso, sid, gantry_deg, side, pitch,
                     reach, step, out_dev, stream):
    g = (C.c_double * len(gantry_deg))(*[float(x) for x in gantry_deg])
    _check(load().pdrt_bev_project(_VP(masks_dev), int(nx), int(ny), int(nz), float(spacing[0]),
                                   float(spacing[1]), float(spacing[2]),
                                   (C.c_double * 3)(*[float(x) for x in origin]),
                                   (C.c_double * 3)(*[float(x) for x in iso]), float(sid),
                                   len(gantry_deg), g, int(side), float(pitch), float(reach),
                                   float(step), _VP(out_dev), _VP(stream)))


def pdrt_plan_set_spectrum_memo(plan, enable):
    _check(load().pdrt_plan_set_spectrum_memo(_VP(plan), 1 if enable else 0))


def pdrt_plan_reset_spectrum_memo(plan, stream):
    _check(load().pdrt_plan_reset_spectrum_memo(_VP(plan), _VP(stream)))


def pdrt_plan_set_fft(plan, pmax):
    _check(load().pdrt_plan_set_fft(_VP(plan), int(pmax)))


def pdrt_plan_set_tc_phase(plan, phase_forward, phase_adjoint):
    _check(load().pdrt_plan_set_tc_phase(_VP(plan), int(phase_forward), int(phase_adjoint)))
