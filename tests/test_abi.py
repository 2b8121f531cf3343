"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and rejects bad arguments with the documented status codes
before it touches a device."""

import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tn():
    import __graft_entry__ as g
    g.build()
    from paper_2312_05233_gb300 import tnep
    return tnep


def header_symbols():
    src = open(os.path.join(ROOT, "include", "tnep.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tnep_[a-z_0-9]+)\s*\(", src)))


def test_header_and_library_exports(tn):
    syms = header_symbols()
    assert len(syms) >= 11
    lib = tn.lib()
    for s in syms:
        assert hasattr(lib, s), f"libtnep.so does not export {s}"
    assert sorted(tn.EXPORTED) == sorted(syms)


def _desc(tn, **over):
    import synth
    hp = synth.HyperParams(n_types=2, rank=1)
    p = synth.model_params(hp, np.random.default_rng(0))
    m = tn.Model.from_hyper(hp, p)
    for k, v in over.items():
        setattr(m, k, v)
    return m


def _create_status(tn, models, n_types=2, cut=(6.0, 4.0)):
    try:
        ctx = tn.tnep_create(models, n_types, cut)
    except tn.TnepError as e:
        return e.status
    ctx.close()
    return 0


def test_create_validation(tn):
    assert _create_status(tn, []) == 1
    assert _create_status(tn, [_desc(tn)], n_types=0) == 1
    assert _create_status(tn, [_desc(tn)], n_types=9) == 1
    assert _create_status(tn, [_desc(tn)], cut=(4.0, 6.0)) == 1
    assert _create_status(tn, [_desc(tn, rank=3)]) == 1
    assert _create_status(tn, [_desc(tn, n_hidden=65)]) == 1
    bad = _desc(tn)
    bad.params = bad.params[:-1]
    assert _create_status(tn, [bad]) == 1
    assert _create_status(tn, [_desc(tn, l_max=6)]) in (1, 7)
    assert _create_status(tn, [_desc(tn, mlp_precision=3)]) == 1
    assert _create_status(tn, [_desc(tn, mlp_precision=1, n_hidden=40)]) == 7


def test_create_without_gpu_reports_no_device(tn):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    assert _create_status(tn, [_desc(tn)]) == 9


def test_null_context_and_spectrum_validation(tn):
    lib = tn.lib()
    assert lib.tnep_eval(None, 1, 1, None, None, None, None, None) == 1
    assert lib.tnep_set_option(None, 0, 1.0) == 1
    v = C.c_double()
    assert lib.tnep_get_option(None, 0, C.byref(v)) == 1
    assert lib.tnep_output_dim(None, 0) == 0
    s = np.zeros((10, 3))
    f = np.zeros(6)
    sp = np.zeros(6)
    # C must match the kind, T >= 2, dt > 0, 1 <= max_lag < T
    assert lib.tnep_spectrum(s.ctypes.data, 10, 9, 1.0, 0, 5, 1, f.ctypes.data, sp.ctypes.data, None, None) == 1
    assert lib.tnep_spectrum(s.ctypes.data, 1, 3, 1.0, 0, 5, 1, f.ctypes.data, sp.ctypes.data, None, None) == 1
    assert lib.tnep_spectrum(s.ctypes.data, 10, 3, 0.0, 0, 5, 1, f.ctypes.data, sp.ctypes.data, None, None) == 1
    assert lib.tnep_spectrum(s.ctypes.data, 10, 3, 1.0, 0, 10, 1, f.ctypes.data, sp.ctypes.data, None, None) == 1
    assert lib.tnep_spectrum(s.ctypes.data, 10, 3, 1.0, 7, 5, 1, f.ctypes.data, sp.ctypes.data, None, None) == 1
    assert "kind" in lib.tnep_last_error().decode()


def test_snes_validation(tn):
    lib = tn.lib()
    buf = np.zeros(64)
    # population size 2..1024, dim >= 1, device buffers only
    assert lib.tnep_snes_normals(1, 0, 1, 8, buf.ctypes.data, None) == 1
    assert lib.tnep_snes_normals(1, 0, 1025, 8, buf.ctypes.data, None) == 1
    assert lib.tnep_snes_normals(1, 0, 4, 0, buf.ctypes.data, None) == 1
    assert lib.tnep_snes_normals(1, -1, 4, 8, buf.ctypes.data, None) == 1
    assert lib.tnep_snes_normals(1, 0, 4, 8, buf.ctypes.data, None) == 1  # host pointer
    assert "device" in lib.tnep_last_error().decode()
    assert lib.tnep_snes_update(4, 8, buf.ctypes.data, buf.ctypes.data, buf.ctypes.data, buf.ctypes.data,
                                1.0, 0.0, None) == 1
    cfg = tn.SnesConfig(8, 0.0, 0.0, 0.0, 0.0, 1)
    h = C.c_void_p()
    assert lib.tnep_snes_create(None, 0, C.byref(cfg), buf.ctypes.data, buf.ctypes.data, 1, None, None, None,
                                None, None, C.byref(h)) == 1
    assert lib.tnep_snes_run(None, 1, None) == 1
    assert lib.tnep_snes_info(None, buf.ctypes.data) == 1


def test_raman_validation(tn):
    lib = tn.lib()
    s = np.zeros((10, 9))
    f = np.zeros(6)
    L = np.zeros((6, 81))
    assert lib.tnep_raman_tensor(s.ctypes.data, 1, 1.0, 0, 1, f.ctypes.data, L.ctypes.data, None) == 1
    assert lib.tnep_raman_tensor(s.ctypes.data, 10, 0.0, 5, 1, f.ctypes.data, L.ctypes.data, None) == 1
    assert lib.tnep_raman_tensor(s.ctypes.data, 10, 1.0, 10, 1, f.ctypes.data, L.ctypes.data, None) == 1
    assert lib.tnep_raman_tensor(None, 10, 1.0, 5, 1, f.ctypes.data, L.ctypes.data, None) == 1
    v = np.zeros(3)
    assert lib.tnep_raman_polarized(L.ctypes.data, 5, 0, v.ctypes.data, v.ctypes.data, f.ctypes.data, None) == 1
    assert lib.tnep_raman_porto_map(L.ctypes.data, 5, 1, v.ctypes.data, 3, f.ctypes.data, f.ctypes.data,
                                    None) == 1
    assert "axis" in lib.tnep_last_error().decode()


def test_noalloc_wrapper_checks_buffers_before_any_call(tn):
    """The C entry point cannot see buffer lengths, so the binding checks
    them: outputs shorter than M + 1, a series that is not 2-D, not float64
    or not contiguous, and a series not in CUDA memory are all refused before
    the library is called (CPU tensors here: nothing reaches a device)."""
    import torch
    s = torch.zeros((100, 3), dtype=torch.float64)
    ok = torch.zeros(51, dtype=torch.float64)
    short = torch.zeros(50, dtype=torch.float64)
    with pytest.raises(tn.TnepError) as e:
        tn.tnep_spectrum_noalloc(s, 1.0, tn.TNEP_SPECTRUM_IR, short, ok)
    assert e.value.status == 1 and "freq_out" in str(e.value)
    with pytest.raises(tn.TnepError) as e:
        tn.tnep_spectrum_noalloc(s, 1.0, tn.TNEP_SPECTRUM_IR, ok, ok, short)
    assert e.value.status == 1 and "acf_out" in str(e.value)
    with pytest.raises(tn.TnepError) as e:  # max_lag 70 needs 71 elements
        tn.tnep_spectrum_noalloc(s, 1.0, tn.TNEP_SPECTRUM_IR, ok, ok, max_lag=70)
    assert e.value.status == 1 and "71" in str(e.value)
    with pytest.raises(tn.TnepError):
        tn.tnep_spectrum_noalloc(s.reshape(-1), 1.0, tn.TNEP_SPECTRUM_IR, ok, ok)
    with pytest.raises(TypeError):
        tn.tnep_spectrum_noalloc(s.float(), 1.0, tn.TNEP_SPECTRUM_IR, ok, ok)
    with pytest.raises(TypeError):
        tn.tnep_spectrum_noalloc(torch.zeros((3, 100), dtype=torch.float64).t(), 1.0, tn.TNEP_SPECTRUM_IR, ok, ok)
    with pytest.raises(tn.TnepError) as e:  # sizes fine, but host memory
        tn.tnep_spectrum_noalloc(s, 1.0, tn.TNEP_SPECTRUM_IR, ok, ok)
    assert e.value.status == 1 and "CUDA" in str(e.value)
