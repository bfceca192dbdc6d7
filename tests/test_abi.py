"""Host-side tests of the C ABI: the library loads, exports what include/poisson.h declares,
and validates descriptors without touching a GPU (poisson_plan_create makes no CUDA call)."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_2104_08863_gb300 import build as b
    b.build()
    from paper_2104_08863_gb300 import _native
    return _native


def _header_functions():
    text = open(os.path.join(ROOT, "include", "poisson.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", text, flags=re.M)))


def test_library_exports_every_declared_symbol(native):
    names = _header_functions()
    assert len(names) >= 10
    lib = ctypes.CDLL(native.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(native.EXPORTS) == names


def _desc(native, nx=32, ny=32, nz=32, faces=None, **kw):
    faces = W.tanh_faces(ny, 1.5) if faces is None else faces
    arr = np.ascontiguousarray(faces, dtype=np.float64)
    d = native.PoissonDesc(nx, ny, nz, 2 * np.pi, np.pi, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           kw.get("precision", 0), kw.get("tridiag", 0), kw.get("pdd_parts", 0),
                           kw.get("fp64_low_modes", 4), kw.get("refine_steps", 1), kw.get("flags", 0))
    return d, arr


def _create(native, d):
    h = ctypes.c_void_p()
    st = native.lib().poisson_plan_create(ctypes.byref(d), ctypes.byref(h))
    if st == 0:
        size = ctypes.c_size_t()
        assert native.lib().poisson_workspace_size(h, ctypes.byref(size)) == 0
        native.lib().poisson_plan_destroy(h)
        return st, size.value
    return st, None


@pytest.mark.parametrize("kw,expect", [
    (dict(nx=31), 1), (dict(nx=2), 1), (dict(nz=1), 1), (dict(ny=1, faces=np.array([-1.0, 1.0])), 1),
    (dict(nx=28), 2), (dict(nz=14), 2), (dict(nx=20), 2),
    (dict(tridiag=2, pdd_parts=5), 2), (dict(tridiag=2, pdd_parts=64, ny=64, faces=W.tanh_faces(64, 1.0)), 2),
    (dict(precision=7), 1), (dict(tridiag=9), 1),
])
def test_plan_rejects_invalid_or_unsupported(native, kw, expect):
    d, _ = _desc(native, **kw)
    st, _ = _create(native, d)
    assert st == expect


def test_plan_rejects_non_monotone_faces(native):
    f = W.tanh_faces(32, 1.5)
    f[5], f[6] = f[6], f[5]
    d, _ = _desc(native, faces=f)
    assert _create(native, d)[0] == 1
    f2 = W.tanh_faces(32, 1.5)
    f2[3] = np.nan
    d, _ = _desc(native, faces=f2)
    assert _create(native, d)[0] == 1


@pytest.mark.parametrize("nx,ny,nz", [(32, 32, 32), (6, 8, 12), (96, 48, 27), (1536, 768, 1024)])
def test_plan_accepts_radix_2_3_sizes_and_reports_workspace(native, nx, ny, nz):
    d, _ = _desc(native, nx=nx, ny=ny, nz=nz, faces=W.tanh_faces(ny, 2.0))
    st, size = _create(native, d)
    assert st == 0
    spectral = ny * nz * (nx // 2 + 1) * 16
    assert size >= spectral


def test_status_strings(native):
    assert native.status_string(0) == "ok"
    assert "invalid" in native.status_string(1)
    assert native.status_string(99) == "unknown status"


def test_entry_points_validate_before_any_device_work(native):
    """Null arguments and a plan without workspace are rejected synchronously (no CUDA call is
    reached), for the solve, its adjoint and the projection."""
    d, _ = _desc(native, precision=2)
    h = ctypes.c_void_p()
    L = native.lib()
    assert L.poisson_plan_create(ctypes.byref(d), ctypes.byref(h)) == 0
    try:
        buf = (ctypes.c_double * 4)()
        p = ctypes.cast(buf, ctypes.c_void_p)
        assert L.poisson_solve_adjoint(None, p, p, None) == native.PS_EINVAL
        assert L.poisson_solve_adjoint(h, None, p, None) == native.PS_EINVAL
        assert L.poisson_solve_adjoint(h, p, None, None) == native.PS_EINVAL
        assert L.poisson_solve_adjoint(h, p, p, None) == native.PS_ENOWORKSPACE
        assert L.poisson_solve(h, p, p, None) == native.PS_ENOWORKSPACE
        assert L.projection_step(h, p, p, p, None, 1e-3, None) == native.PS_ENOWORKSPACE
    finally:
        L.poisson_plan_destroy(h)


def test_selftest_flag_is_accepted_by_the_planner(native):
    d, _ = _desc(native, nx=512, ny=4, nz=16, faces=W.tanh_faces(4, 1.5), precision=2,
                 flags=native.POISSON_SELFTEST_WAIT)
    assert _create(native, d)[0] == 0


def test_slab_chain_configuration_is_validated_on_the_host(native):
    """poisson_plan_set_chain accepts only the FP32 scan-PDD path with tile-aligned slab widths;
    single-stream configurations make no CUDA call."""
    L = native.lib()

    def plan(**kw):
        d, arr = _desc(native, **kw)
        h = ctypes.c_void_p()
        assert L.poisson_plan_create(ctypes.byref(d), ctypes.byref(h)) == 0
        return h, arr

    f96 = W.tanh_faces(96, 2.0)
    h64, _ = plan(nx=96, ny=96, nz=64, faces=f96, precision=0, pdd_parts=8)
    h32, _ = plan(nx=96, ny=96, nz=64, faces=f96, precision=1, pdd_parts=16)
    hreg, _ = plan(nx=96, ny=96, nz=64, faces=f96, precision=1, pdd_parts=48)   # register kernel
    try:
        assert L.poisson_plan_set_chain(h64, 32, 1) == native.PS_EUNSUPPORTED
        assert L.poisson_plan_set_chain(hreg, 32, 1) == native.PS_EUNSUPPORTED
        assert L.poisson_plan_set_chain(h32, 32, 1) == native.PS_OK      # z tile 32, 16 systems per CTA
        assert L.poisson_plan_set_chain(h32, 16, 1) == native.PS_EUNSUPPORTED
        assert L.poisson_plan_set_chain(h32, 48, 1) == native.PS_EUNSUPPORTED
        assert L.poisson_plan_set_chain(h32, 32, 3) == native.PS_EINVAL
        assert L.poisson_plan_set_chain(h32, -1, 1) == native.PS_EINVAL
        assert L.poisson_plan_set_chain(h32, 0, 1) == native.PS_OK
        assert L.poisson_plan_set_chain(None, 32, 1) == native.PS_EINVAL
    finally:
        for h in (h64, h32, hreg):
            L.poisson_plan_destroy(h)
