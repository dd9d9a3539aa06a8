"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/cjt.h declares; its argument checks and the binding's buffer checks
refuse bad input before any device call (no compute calls here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1602_02618_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(os.path.join(ROOT, "include", "cjt.h")).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cjt_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cjt_plan", "cjt_forward", "cjt_inverse", "cjt_execute_batched", "cjt_destroy",
                     "cjt_strerror", "cjt_sync", "cjt_execute_host"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    lib.cjt_strerror.restype = ctypes.c_char_p
    assert lib.cjt_strerror(0) == b"success"
    assert b"alpha" in lib.cjt_strerror(-2)
    lib.cjt_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.cjt_version()


def test_binding_names_match_header():
    from paper_1602_02618_gb300 import cjt
    assert sorted(cjt.EXPORTED) == declared_functions()


def header_struct_fields(name):
    """Field names of `typedef struct { ... } name;` in include/cjt.h, in order."""
    text = open(os.path.join(ROOT, "include", "cjt.h")).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    m = re.search(r"typedef\s+struct\s*\{([^}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        ctype, names = re.match(r"(\w+)\s+(.*)", decl).groups()
        fields += [(n.strip(), ctype) for n in names.split(",")]
    return fields


@pytest.mark.parametrize("name", ["cjt_plan_opts", "cjt_plan_info"])
def test_binding_structs_match_header(name):
    """The ctypes structures of the binding list the header's fields in the header's order,
    with the same C types, so that options and plan summaries cross the ABI intact."""
    import ctypes as ct
    from paper_1602_02618_gb300 import cjt
    ctypes_of = {"int": ct.c_int, "double": ct.c_double, "int64_t": ct.c_int64}
    want = [(n, ctypes_of[t]) for n, t in header_struct_fields(name)]
    got = list(getattr(cjt, name)._fields_)
    assert got == want


def test_without_a_device_calls_fail_loudly():
    """With no usable GPU the library reports errors instead of computing anything on the
    host: argument errors first (before any device call), then CJT_ECUDA with the CUDA
    runtime's message; no handle is returned and nothing crashes."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1602_02618_gb300 import cjt
    lib = cjt.load()
    h = ctypes.c_void_p()
    o = cjt.default_opts()
    assert lib.cjt_plan(ctypes.byref(h), 64, 0.9, 2.0, ctypes.byref(o), None) == cjt.CJT_EDOMAIN
    assert lib.cjt_plan(ctypes.byref(h), -1, 0.1, -0.3, ctypes.byref(o), None) == cjt.CJT_EINVAL
    assert lib.cjt_plan(None, 64, 0.1, -0.3, ctypes.byref(o), None) == cjt.CJT_EINVAL
    assert lib.cjt_cheb_coeffs_noalloc(64, None, None, None) == cjt.CJT_EINVAL
    assert lib.cjt_plan(ctypes.byref(h), 64, 0.1, -0.3, ctypes.byref(o), None) == cjt.CJT_ECUDA
    assert h.value is None
    assert lib.cjt_last_cuda_error()
    with pytest.raises(cjt.CJTError) as e:
        cjt.Plan(64, 0.1, -0.3, stream=0)      # the default stream, named without torch
    assert e.value.code == cjt.CJT_ECUDA
    assert lib.cjt_sync(None) == cjt.CJT_ECUDA
    assert lib.cjt_error_bound(None, cjt.CJT_FWD, None) == cjt.CJT_EINVAL
    assert lib.cjt_get_partition(None, cjt.CJT_FWD, 0, None, None) == cjt.CJT_EINVAL
    assert lib.cjt_fft_set_config(cjt.CJT_FP64, 40, 4, 0, 12) == cjt.CJT_EINVAL
    assert lib.cjt_fft_set_config(cjt.CJT_FP64, 16, 4, 0, 14) == cjt.CJT_EINVAL
    assert lib.cjt_fft_time(cjt.CJT_FP64, 16, 1, 1, None, None) == cjt.CJT_EINVAL
    assert lib.cjt_batch_launch_host(None, None, None, None) == cjt.CJT_EINVAL
    assert lib.cjt_batch_set_profiling(None, 1) == cjt.CJT_EINVAL
    assert lib.cjt_batch_get_profile(None, None, None, 0) == cjt.CJT_EINVAL


# one bad value per option; cjt_plan checks them all before it touches the device
_BAD_OPTIONS = [dict(M=21), dict(M=-1), dict(eps=1.5), dict(eps=-1e-3), dict(precision=7), dict(directions=4),
                dict(directions=-1), dict(ratio=1.0), dict(ratio=-0.1), dict(seg_len=48), dict(seg_len=16),
                dict(seg_len=1 << 21), dict(use_asy=2), dict(use_asy=-2), dict(rec_store=2), dict(expansion=3),
                dict(expansion=-1), dict(grid=2), dict(grid=-2), dict(overlap=4), dict(overlap=-1),
                dict(seg_whole=-1), dict(seg_whole=(1 << 23) + 1)]


@pytest.mark.parametrize("bad", _BAD_OPTIONS, ids=lambda d: "%s=%s" % next(iter(d.items())))
def test_bad_option_values_are_refused(bad):
    """Every option outside its documented range returns CJT_EINVAL and no handle, on a
    machine with or without a GPU (the checks run before any device call)."""
    from paper_1602_02618_gb300 import cjt
    lib = cjt.load()
    o = cjt.default_opts()
    for k, v in bad.items():
        setattr(o, k, v)
    h = ctypes.c_void_p()
    assert lib.cjt_plan(ctypes.byref(h), 64, 0.1, -0.3, ctypes.byref(o), None) == cjt.CJT_EINVAL
    assert h.value is None


def test_ultraspherical_expansion_needs_equal_parameters():
    from paper_1602_02618_gb300 import cjt
    lib = cjt.load()
    o = cjt.default_opts()
    o.expansion = cjt.CJT_EXPANSION_ULTRASPHERICAL
    h = ctypes.c_void_p()
    assert lib.cjt_plan(ctypes.byref(h), 64, 0.1, -0.3, ctypes.byref(o), None) == cjt.CJT_EINVAL
    assert h.value is None


def test_binding_refuses_buffers_that_do_not_fit():
    """The binding checks the caller's buffers before it calls the library: host arrays
    too small, of another dtype, non-contiguous or read-only, and a workspace that is not a
    CUDA tensor, are refused, so that the library never writes past a host array nor gets
    a host address for device memory."""
    torch = pytest.importorskip("torch")
    from paper_1602_02618_gb300 import cjt

    class FakePlan:
        N = 7
        handle = ctypes.c_void_p()

    with pytest.raises(ValueError):
        cjt.cjt_execute_host(FakePlan(), cjt.CJT_FWD, np.zeros(8), out=np.zeros(7))
    with pytest.raises(TypeError):
        cjt.cjt_execute_host(FakePlan(), cjt.CJT_FWD, np.zeros(8), out=np.zeros(8, dtype=np.float32))
    with pytest.raises(TypeError):
        cjt.cjt_execute_host(FakePlan(), cjt.CJT_FWD, np.zeros(8), out=np.zeros(16)[::2])
    ro = np.zeros(8)
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        cjt.cjt_execute_host(FakePlan(), cjt.CJT_FWD, np.zeros(8), out=ro)
    for fn in (cjt.cjt_forward_ws, cjt.cjt_inverse_ws):
        with pytest.raises(TypeError, match="workspace"):
            fn(FakePlan(), torch.zeros(8, dtype=torch.float64), torch.zeros(8, dtype=torch.float64),
               torch.zeros(64, dtype=torch.uint8))
    b = cjt.Batch.__new__(cjt.Batch)          # a batch whose inputs span 10 values
    b._h, b.total = ctypes.c_void_p(), 10
    with pytest.raises(ValueError):
        b.launch_host(np.zeros(9), np.zeros(10))
    with pytest.raises(ValueError):
        b.launch_host(np.zeros(10), np.zeros(9))
