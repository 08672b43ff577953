"""Host-side checks of the C ABI: the library loads, exports what the header
declares, plans steps like the oracle and rejects bad arguments before any
CUDA call.  CPU only (no GPU is touched)."""
import ctypes

import pytest

import paper_1304_6514_gb300 as nvp
from paper_1304_6514_gb300 import _build
from oracle import nievergelt as nv


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return nvp.load_library()


def test_exports_every_declared_function(lib):
    names = nvp.header_functions()
    assert "nv_build_propagators" in names and "nv_compose" in names and "nv_solve" in names
    for name in names:
        assert hasattr(lib, name), name
    assert nvp.version() == 1


@pytest.mark.parametrize("t0,T,S,dt,fixed", [
    (0.0, 0.1, 1024, 1e-5, 0), (0.0, 20.0, 128, 1e-3, 0), (0.0, 1.0, 512, 2e-4, 0),
    (0.0, 0.5, 4, 0.01, 0), (0.0, 0.5, 4, 0.005, 0), (0.0, 10.0, 16, 0.0, 10000),
    (1.5, 7.25, 33, 3e-3, 0), (0.0, 17.3, 211, 1e-3, 0)])
def test_plan_steps_matches_oracle(lib, t0, T, S, dt, fixed):
    m, h = nvp.plan_steps(t0, T, S, dt, fixed)
    mo = nv.steps_per_slice(t0, T, S, dt, fixed)
    assert m == mo
    assert h == nv.step_size(t0, T, S, mo)


def test_plan_steps_rejects(lib):
    with pytest.raises(nvp.NvError) as e:
        nvp.plan_steps(1.0, 0.5, 4, 0.1)
    assert e.value.status == nvp.NV_EINVAL
    with pytest.raises(nvp.NvError):
        nvp.plan_steps(0.0, 1.0, 4, 0.0, 0)


def _expect(status_wanted, fn):
    with pytest.raises(nvp.NvError) as e:
        fn()
    assert e.value.status == status_wanted, (e.value.status, str(e.value))
    assert nvp.last_error()


@pytest.mark.parametrize("case", [
    dict(rhs=("cos_cubic", 2, ()), smp=("pl1d", 64, (-2,), (2,)), msg="dim"),
    dict(rhs=("cos_cubic", 1, ()), smp=("pl1d", 1, (-2,), (2,)), msg="per_dim"),
    dict(rhs=("cos_cubic", 1, ()), smp=("pl1d", 8, (2,), (-2,)), msg="lo<hi"),
    dict(rhs=("vdp", 2, ()), smp=("bilinear2d", 8, (-3, -3), (3, 3)), msg="mu missing"),
    dict(rhs=("vdp", 2, (1.0,)), smp=("pl1d", 8, (-3,), (3,)), msg="map/dim"),
    dict(rhs=("cos_cubic", 1, ()), smp=("affine", 0, (), ()), msg="affine nonlinear"),
    dict(rhs=("heat1d", 600, ()), smp=("affine", 0, (), ()), msg="too big"),
    dict(rhs=("heat1d", 16, (1.0,)), smp=("affine", 0, (), ()), msg="params"),
])
def test_build_rejects_before_launch(lib, case):
    r = nvp.rhs(*case["rhs"])
    s = nvp.samples(*case["smp"])
    st = nvp.steps("rk4", 1e-3)
    _expect(nvp.NV_EINVAL, lambda: nvp.build_propagators(r, 0.0, 1.0, 4, s, st, stream=0))


def test_build_rejects_bad_grid(lib):
    r = nvp.rhs("cos_cubic", 1)
    s = nvp.samples("pl1d", 8, (-2,), (2,))
    _expect(nvp.NV_EINVAL, lambda: nvp.build_propagators(r, 1.0, 0.0, 4, s, nvp.steps("euler", 1e-3), stream=0))
    _expect(nvp.NV_EINVAL, lambda: nvp.build_propagators(r, 0.0, 1.0, 0, s, nvp.steps("euler", 1e-3), stream=0))
    _expect(nvp.NV_EINVAL, lambda: nvp.build_propagators(r, 0.0, 1.0, 4, s, nvp.steps("euler", 0.0), stream=0))
    _expect(nvp.NV_EINVAL, lambda: nvp.build_propagators(
        r, 0.0, 1.0, 4, s, nvp.steps("euler", 1e-3, prec="tf32_refine"), stream=0))


def test_wave_scheme_and_dimension_checks(lib):
    """The leapfrog scheme belongs to the two-level wave state and only to it;
    the wave state has dimension 2(M-1); its maps have no TF32 path."""
    aff = nvp.samples("affine")
    wv = nvp.rhs("wave", 158)
    _expect(nvp.NV_EINVAL, lambda: nvp.build_propagators(wv, 0.0, 1.0, 4, aff, nvp.steps("rk4", 1e-3), stream=0))
    _expect(nvp.NV_EINVAL, lambda: nvp.build_propagators(nvp.rhs("heat1d", 16), 0.0, 1.0, 4, aff,
                                                         nvp.steps("leapfrog", 1e-3), stream=0))
    _expect(nvp.NV_EINVAL, lambda: nvp.build_propagators(nvp.rhs("wave", 157), 0.0, 1.0, 4, aff,
                                                         nvp.steps("leapfrog", 1e-3), stream=0))
    _expect(nvp.NV_EINVAL, lambda: nvp.build_propagators(nvp.rhs("wave", 162), 0.0, 1.0, 4, aff,
                                                         nvp.steps("leapfrog", 1e-3), stream=0))
    _expect(nvp.NV_EINVAL, lambda: nvp.build_propagators(nvp.rhs("wave", 158, (40.0,)), 0.0, 1.0, 4, aff,
                                                         nvp.steps("leapfrog", 1e-3), stream=0))
    _expect(nvp.NV_ENOTSUP, lambda: nvp.build_propagators(wv, 0.0, 1.0, 4, aff,
                                                          nvp.steps("leapfrog", 1e-3, prec="tf32_refine"), stream=0))
    _expect(nvp.NV_EINVAL, lambda: nvp.build_propagators(wv, 0.0, 1.0, 4, nvp.samples("pl1d", 8, (-1,), (1,)),
                                                         nvp.steps("leapfrog", 1e-3), stream=0))


def test_null_handles(lib):
    assert lib.nv_compose(None, None, None, None, None) == nvp.NV_EBADMAP
    assert lib.nv_maps_info(None, None) == nvp.NV_EINVAL
    assert lib.nv_maps_destroy(None) == nvp.NV_OK
    assert lib.nv_tune_set(99, 1) == nvp.NV_EINVAL
    assert lib.nv_tune_set(6, 6) == nvp.NV_EINVAL           # heat step form is 0..5
    assert lib.nv_tune_set(6, 5) == nvp.NV_OK
    assert lib.nv_tune_set(6, 4) == nvp.NV_OK
    assert lib.nv_tune_set(6, -1) == nvp.NV_EINVAL
    assert lib.nv_tune_set(6, 3) == nvp.NV_OK
    assert lib.nv_tune_set(6, 0) == nvp.NV_OK
    assert lib.nv_tune_set(7, 5) == nvp.NV_EINVAL           # phantom barrier participants 0..4
    assert lib.nv_tune_set(7, -1) == nvp.NV_EINVAL
    assert lib.nv_tune_set(8, 3) == nvp.NV_EINVAL           # split-K is 0 or a power of two <= 16
    assert lib.nv_tune_set(8, 32) == nvp.NV_EINVAL
    assert lib.nv_tune_set(9, 3) == nvp.NV_EINVAL           # tiled chain kernel is 0..2
    assert lib.nv_tune_set(9, -1) == nvp.NV_EINVAL
    assert lib.nv_tune_set(9, 1) == nvp.NV_OK
    assert lib.nv_tune_set(9, 0) == nvp.NV_OK
    assert lib.nv_tune_set(15, 3) == nvp.NV_EINVAL          # advection-diffusion build form is 0, 1 or 2
    assert lib.nv_tune_set(15, 2) == nvp.NV_OK
    assert lib.nv_tune_set(15, 1) == nvp.NV_OK
    assert lib.nv_tune_set(15, 0) == nvp.NV_OK
    assert lib.nv_tune_set(14, 2) == nvp.NV_EINVAL          # chain band use is 0 or 1
    assert lib.nv_tune_set(14, -1) == nvp.NV_EINVAL
    assert lib.nv_tune_set(14, 1) == nvp.NV_OK
    assert lib.nv_tune_set(14, 0) == nvp.NV_OK
    assert lib.nv_tune_set(10, 2) == nvp.NV_EINVAL          # refinement schedule is 0 or 1
    assert lib.nv_tune_set(10, 1) == nvp.NV_OK
    assert lib.nv_tune_set(10, 0) == nvp.NV_OK
    assert lib.nv_tune_set(12, -1) == nvp.NV_EINVAL         # withheld slice is >= 0
    assert lib.nv_tune_set(12, 0) == nvp.NV_OK
    assert lib.nv_tune_set(13, -1) == nvp.NV_EINVAL         # skipped step is >= 0
    assert lib.nv_tune_set(13, 0) == nvp.NV_OK
    assert lib.nv_tune_set(16, 4) == nvp.NV_EINVAL          # strip height is 0, 8, 16 or 32
    assert lib.nv_tune_set(16, 8) == nvp.NV_OK
    assert lib.nv_tune_set(16, 0) == nvp.NV_OK
    assert lib.nv_tune_set(17, 5) == nvp.NV_EINVAL          # float32 heat window form is 0..4
    assert lib.nv_tune_set(17, 4) == nvp.NV_OK
    assert lib.nv_tune_set(17, 2) == nvp.NV_OK
    assert lib.nv_tune_set(17, 0) == nvp.NV_OK
    assert lib.nv_tune_set(18, 3) == nvp.NV_EINVAL          # learned iteration-0 form is 0, 1 or 2
    assert lib.nv_tune_set(18, 1) == nvp.NV_OK
    assert lib.nv_tune_set(18, 0) == nvp.NV_OK
    assert lib.nv_tune_set(19, 3) == nvp.NV_EINVAL          # learned correction form is 0, 1 or 2
    assert lib.nv_tune_set(19, 1) == nvp.NV_OK
    assert lib.nv_tune_set(19, 0) == nvp.NV_OK
    assert lib.nv_tune_set(20, -1) == nvp.NV_EINVAL         # float32 learned iterations are 0..1000
    assert lib.nv_tune_set(20, 3) == nvp.NV_OK
    assert lib.nv_tune_set(20, 0) == nvp.NV_OK
    assert lib.nv_alu_rate(0, None, None) == nvp.NV_EINVAL        # no output pointer
    rate = ctypes.c_double(0.0)
    assert lib.nv_alu_rate(3, ctypes.byref(rate), None) == nvp.NV_EINVAL   # float64 or float32 only
    assert lib.nv_mlp_parareal(None, None, 0.0, 1.0, 4, None, 1, 128, None, None, None, None) == nvp.NV_EINVAL
    assert lib.nv_build_propagators(None, 0.0, 1.0, 4, None, None, None, None) == nvp.NV_EINVAL
    h = ctypes.c_void_p()
    assert lib.nv_build_propagators(None, 0.0, 1.0, 4, None, None, ctypes.byref(h), None) == nvp.NV_EINVAL


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes mirrors of the header's structs have the C
    compiler's size and field offsets (a field added on one side only would
    shift every later one)."""
    import os
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    include = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    mirrors = {"nv_rhs": nvp.NvRhs, "nv_samples": nvp.NvSamples, "nv_steps": nvp.NvSteps,
               "nv_maps_desc": nvp.NvMapsDesc}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "nvpit.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", include, str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)


def test_every_tunable_is_documented_in_the_header(lib):
    """The keys nv_tune_set accepts (api.cu) are exactly the keys the header
    documents ("key N:")."""
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    header = open(os.path.join(root, "include", "nvpit.h")).read()
    api = open(os.path.join(root, "paper_1304_6514_gb300", "csrc", "api.cu")).read()
    body = api[api.index("nv_status nv_tune_set("):]
    body = body[:body.index("default:")]
    accepted = {int(k) for k in re.findall(r"case (\d+):", body)}
    documented = {int(k) for k in re.findall(r"\bkey (\d+):", header)}
    assert accepted == documented
    for key in sorted(accepted):
        assert lib.nv_tune_set(key, 0) == nvp.NV_OK, key
