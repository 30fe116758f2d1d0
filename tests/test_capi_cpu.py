"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports every
entry point that include/iesh.h declares, and rejects invalid arguments before
touching the device."""
import ctypes
import os
import re

import pytest

import iesh_inputs as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2212_00518_gb300 import iesh
    from paper_2212_00518_gb300 import build as B
    B.build()
    return iesh.load()


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(iesh2?_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(lib):
    names = _declared("iesh.h")
    assert "iesh_run" in names and "iesh_create" in names and "iesh2_run" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_2212_00518_gb300 import iesh
    assert sorted(iesh.EXPORTS) == _declared("iesh.h")


def test_status_strings(lib):
    from paper_2212_00518_gb300 import iesh
    assert lib.iesh_status_string(0) == b"IESH_OK"
    assert lib.iesh_status_string(1) == b"IESH_EINVAL"
    for code, name in iesh.STATUS_NAMES.items():
        assert lib.iesh_status_string(code) == name.encode()


def test_invalid_options_rejected_without_device(lib):
    from paper_2212_00518_gb300 import iesh
    md = iesh.model_struct(W.double_well(20))
    for kw in (dict(prop_tol=1.0), dict(prop_tol=-1e-3), dict(traj_base=-1),
               dict(norm_tol=float("nan"))):
        opt = iesh._Options(iesh.PREC_FP64, 0, 0, 0, 0.0)
        for k, v in kw.items():
            setattr(opt, k, v)
        h = ctypes.c_void_p()
        rc = lib.iesh_create(ctypes.byref(h), ctypes.byref(md), ctypes.byref(opt), 16, None)
        assert rc == 1, (kw, rc)
        assert lib.iesh_last_error(h)
        lib.iesh_destroy(h)
    # entry points refuse a null context
    for fn in ("iesh_checkpoint_bytes", "iesh_checkpoint_save", "iesh_checkpoint_load",
               "iesh_observables", "iesh_check"):
        f = getattr(lib, fn)
        args = [0 if t is ctypes.c_size_t else None for t in f.argtypes]
        assert f(*args) == 1, fn


def test_invalid_models_rejected_without_device(lib):
    from paper_2212_00518_gb300 import iesh
    opt = iesh._Options(iesh.PREC_FP64, 0, 0, 0, 0.0)
    for bad in (dict(M=0), dict(M=300), dict(Ne=0), dict(Ne=21), dict(mass=-1.0),
                dict(Gamma=-1.0)):
        md = W.double_well(20)
        md.update(bad)
        h = ctypes.c_void_p()
        rc = lib.iesh_create(ctypes.byref(h), ctypes.byref(iesh.model_struct(md)),
                             ctypes.byref(opt), 16, None)
        assert rc == 1, (bad, rc)
        assert lib.iesh_last_error(h)
        lib.iesh_destroy(h)
    # null arguments
    assert lib.iesh_create(None, None, None, 1, None) == 1
    assert lib.iesh_run(None, 1.0, 1, 0) == 1
    assert lib.iesh_destroy(None) == 0


def test_invalid_two_orbital_models_rejected_without_device(lib):
    from paper_2212_00518_gb300 import two
    for bad in (dict(M=1), dict(M=255), dict(Ne=0), dict(Ne=22), dict(mass=0.0),
                dict(band=(0.5, -0.5))):
        md = W.two_orbital(20)
        md.update(bad)
        h = ctypes.c_void_p()
        rc = lib.iesh2_create(ctypes.byref(h), ctypes.byref(two.model_struct(md)), 0, 16, 0, None)
        assert rc == 1, (bad, rc)
        assert lib.iesh2_last_error(h)
        lib.iesh2_destroy(h)
    md = W.two_orbital(20)
    md["theta"] = md["theta"].copy()
    md["theta"][14] = 0.0
    h = ctypes.c_void_p()
    assert lib.iesh2_create(ctypes.byref(h), ctypes.byref(two.model_struct(md)), 0, 16, 0, None) == 1
    lib.iesh2_destroy(h)
    h = ctypes.c_void_p()
    assert lib.iesh2_create(ctypes.byref(h), ctypes.byref(two.model_struct(W.two_orbital(20))), 7, 16, 0,
                            None) == 1
    lib.iesh2_destroy(h)
    assert lib.iesh2_create(None, None, 0, 1, 0, None) == 1


@pytest.mark.parametrize("N", [2, 21, 61, 101, 129, 201, 256])
def test_tuner_shapes_within_documented_limits(N):
    """The autotuner proposes only propagator shapes that iesh_set_kernel_shape
    accepts by its documented limits: mixed (4, G) with G * ceil(N/4) <= 256
    threads and 8 Np (8G + 1) + 192 Np bytes of shared memory (two buffers
    and the ring of W rows) within 110 KiB for G > 1, or (32, G) with
    G * ceil(ceil(N/4)/2) <= 256 and the same bytes within 220 KiB; FP64
    (ept, G) with ept in {1, 2} and G * N <= 1024."""
    from paper_2212_00518_gb300 import tuning
    from paper_2212_00518_gb300 import iesh as I
    Np = -(-N // 4) * 4
    for Ne in (1, N // 2, N - 1):
        if Ne < 1:
            continue
        mixed = tuning.cheb_candidates(N, Ne, precision=I.PREC_MIXED)
        assert mixed and all(ept in (4, 32) for ept, _ in mixed)
        for ept, G in mixed:
            nq = -(-N // 4)
            rows, cap = (nq, 110) if ept == 4 else (-(-nq // 2), 220)
            assert G * rows <= 256
            assert G == 1 or 8 * Np * (8 * G + 1) + 192 * Np <= cap * 1024
        fp64 = tuning.cheb_candidates(N, Ne, precision=I.PREC_FP64)
        assert fp64 and all(ept in (1, 2) and G * N <= 1024 for ept, G in fp64)
