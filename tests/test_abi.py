"""The C-ABI library builds for sm_103a, loads, exports every entry point that
include/pdrt.h declares, and rejects bad arguments on the host before it
touches the GPU (no compute calls here)."""
import ctypes as C
import os
import re

import pytest

from paper_2512_18863_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    import glob
    text = "".join(open(f).read() for f in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pdrt_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_entry_point():
    lib = _lib.load()
    names = _declared()
    assert "pdrt_dose_forward" in names and "pdrt_dose_backward" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib._SIG), "binding and header disagree"


def test_host_only_calls():
    assert _lib.pdrt_last_error() == ""
    assert _lib.pdrt_launch_count() >= 0


def _grid_create(**kw):
    args = dict(hu=1, nx=4, ny=4, nz=4, sx=2.0, sy=2.0, sz=2.0, origin=(0, 0, 0),
                pts=((-1000.0, 0.0), (0.0, 1.0)))
    args.update(kw)
    return _lib.pdrt_grid_create(args["hu"], args["nx"], args["ny"], args["nz"], args["sx"],
                                 args["sy"], args["sz"], args["origin"], args["pts"], 0)


@pytest.mark.parametrize("kw,status", [
    (dict(nx=0), 2),
    (dict(sx=2.0, sy=3.0), 1),
    (dict(sz=-1.0), 1),
    (dict(pts=((0.0, 1.0),)), 1),
    (dict(pts=((0.0, 1.0), (-5.0, 0.0))), 1),
    (dict(origin=(0.0, float("nan"), 0.0)), 1),
])
def test_grid_create_rejects_bad_arguments(kw, status):
    with pytest.raises(_lib.PdrtError) as e:
        _grid_create(**kw)
    assert e.value.status == status
    assert _lib.pdrt_last_error() != ""


def test_null_handles_rejected():
    lib = _lib.load()
    assert lib.pdrt_dose_forward(None, None, None, None, None, None, None) == 1
    assert lib.pdrt_dose_backward(None, None, None, None, None, None, None, None, None, None) == 1
    out = C.c_void_p()
    m = _lib.pdrt_machine()
    assert lib.pdrt_plan_upload(C.byref(out), None, 1, None, None, C.byref(m), 0, None) == 1
    info = _lib.pdrt_plan_info()
    assert lib.pdrt_plan_get_info(None, C.byref(info)) == 1
    assert lib.pdrt_plan_set_spectrum_memo(None, 1) == 1
    assert lib.pdrt_plan_set_spectrum_memo(None, 0) == 1
    assert lib.pdrt_plan_reset_spectrum_memo(None, None) == 1


def test_struct_layouts_match_the_header(tmp_path):
    """ctypes mirrors of the header's structs have the C compiler's sizes and
    field offsets (a host C program built from include/pdrt.h prints them)."""
    import subprocess
    structs = {"pdrt_machine": _lib.pdrt_machine, "pdrt_plan_info": _lib.pdrt_plan_info,
               "pdrt_work": _lib.pdrt_work, "pdrt_tune_result": _lib.pdrt_tune_result}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pdrt.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                 text=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == C.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"


def test_network_parameter_count_and_host_checks():
    from oracle import cnn_oracle as N
    from paper_2512_18863_gb300 import warmstart as W
    p = N.init_params(0)
    assert _lib.pdrt_cnn_param_count() == sum(v.size for v in p.values()) == 236601
    assert [k for k, _ in W.param_layout()] == ["W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4",
                                                 "W5", "b5"]
    for k, shp in W.param_layout():
        assert p[k].shape == shp
    with pytest.raises(_lib.PdrtError) as e:
        _lib.pdrt_cnn_create(0, 0)
    assert e.value.status == 1
    with pytest.raises(_lib.PdrtError):
        _lib.pdrt_bev_project(0, 4, 4, 4, (1.0, 1.0, 1.0), (0, 0, 0), (0, 0, 0), 1000.0, [0.0], 64,
                              2.5, 50.0, 1.0, 0, 0)


@pytest.mark.skipif(__import__("torch").cuda.is_available(),
                    reason="host-only check with placeholder device pointers; "
                           "the GPU test of the entry point covers a real device")
def test_static_entry_point_rejects_on_the_host():
    """pdrt_cp_dose_static checks its arguments and its scratch need on the
    host before any CUDA call: NULL buffers are EINVAL, and a grid whose
    scratch exceeds PDRT_STATIC_SCRATCH_BYTES is EINVAL with the size needed."""
    from paper_2512_18863_gb300 import synth as S
    m = _lib.machine_struct(S.machine_model(5, r_px=10))
    fake = 256   # never dereferenced: every call below is rejected on the host
    with pytest.raises(_lib.PdrtError) as e:
        _lib.pdrt_cp_dose_static(0, 64, 64, 64, 2.0, 2.0, 2.0, (-64.0, -64.0, -64.0), (0, 0, 0),
                                 0.0, m, fake, fake, fake, fake, 0)
    assert e.value.status == 1
    with pytest.raises(_lib.PdrtError) as e:
        _lib.pdrt_cp_dose_static(fake, 1024, 1024, 512, 1.0, 1.0, 1.0, (-512.0, -512.0, -256.0),
                                 (0, 0, 0), 30.0, m, fake, fake, fake, fake, 0)
    assert e.value.status == 1
    msg = _lib.pdrt_last_error()
    assert "MiB" in msg and "PDRT_STATIC_SCRATCH_BYTES" in msg
    # a tall, narrow grid (nz > 32767) fits the scratch but not the gather's
    # 16-bit packing of the v bounds: EINVAL before any device work
    with pytest.raises(_lib.PdrtError) as e:
        _lib.pdrt_cp_dose_static(fake, 4, 4, 40000, 2.0, 2.0, 1.0, (-4.0, -4.0, -20000.0),
                                 (0, 0, 0), 0.0, m, fake, fake, fake, fake, 0)
    assert e.value.status == 1 and "32767" in _lib.pdrt_last_error()
