"""The allocation-free spectrum entry point against the allocating one.

tnep_spectrum_noalloc serves callers that cannot call cudaMalloc (an MD
engine that owns all device memory, or one computing spectra inside its
time-step loop, where allocation would synchronise the device).  It keeps its
scratch in one static device array shared by every call, so this test checks
two calls in a row, with different inputs, each against tnep_spectrum with
the tolerance of the spectrum parity tests.  The file sorts last so that a
run stopping at the first failure has already run every other test.
"""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    import __graft_entry__ as g
    g.build()
    from paper_2312_05233_gb300 import tnep
    return tnep


def _run_noalloc(tn, series, kind, max_lag):
    M = max_lag if max_lag > 0 else series.shape[0] // 2
    dev = torch.device("cuda")
    s = torch.from_numpy(series).to(dev)
    f = torch.empty(M + 1, dtype=torch.float64, device=dev)
    p = torch.empty(M + 1, dtype=torch.float64, device=dev)
    a = torch.empty(M + 1, dtype=torch.float64, device=dev)
    tn.tnep_spectrum_noalloc(s, 0.5, kind, f, p, a, max_lag=max_lag)
    torch.cuda.synchronize()
    return f.cpu().numpy(), p.cpu().numpy(), a.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_twice(tn):
    rng = np.random.default_rng(7)
    cases = [(tn.TNEP_SPECTRUM_RAMAN_ANISO, rng.normal(size=(700, 9)), 300),
             (tn.TNEP_SPECTRUM_IR, rng.normal(size=(400, 3)) + 5.0, 0)]
    for kind, series, max_lag in cases:  # two calls in a row on the shared scratch
        f, S, A = _run_noalloc(tn, series, kind, max_lag)
        fr, Sr, Ar = tn.tnep_spectrum(series, 0.5, kind, max_lag=max_lag, want_acf=True)
        np.testing.assert_allclose(A, Ar, rtol=1e-11, atol=1e-13 * np.abs(Ar).max())
        np.testing.assert_allclose(f, fr, rtol=1e-13)
        np.testing.assert_allclose(S, Sr, rtol=1e-9, atol=1e-11 * np.abs(Sr).max())


def test_noalloc_rejects_oversized_series(tn):
    dev = torch.device("cuda")
    T = tn.TNEP_NOALLOC_MAX_T + 1
    s = torch.zeros((T, 3), dtype=torch.float64, device=dev)
    f = torch.empty(T // 2 + 1, dtype=torch.float64, device=dev)
    p = torch.empty(T // 2 + 1, dtype=torch.float64, device=dev)
    with pytest.raises(tn.TnepError) as e:
        tn.tnep_spectrum_noalloc(s, 1.0, tn.TNEP_SPECTRUM_IR, f, p)
    assert e.value.status == 1 and "TNEP_NOALLOC_MAX_T" in str(e.value)
