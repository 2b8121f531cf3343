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


def test_noalloc_where_the_allocating_path_takes_the_fourier_route(tn):
    """At T = 20,000 (Raman aniso, M = T/2) tnep_spectrum correlates through
    the float64 FFT while the allocation-free entry point keeps the direct
    time-origin sums; both must agree within the Fourier-route tolerance of
    the long-series parity tests."""
    rng = np.random.default_rng(11)
    T = 20_000
    t = np.arange(T)
    series = rng.normal(size=(T, 9)) + np.cos(0.003 * t)[:, None] * rng.normal(size=9) + 2.0
    f, S, A = _run_noalloc(tn, series, tn.TNEP_SPECTRUM_RAMAN_ANISO, 0)
    fr, Sr, Ar = tn.tnep_spectrum(series, 0.5, tn.TNEP_SPECTRUM_RAMAN_ANISO, want_acf=True)
    np.testing.assert_allclose(A, Ar, rtol=0, atol=1e-12 * np.abs(Ar).max())
    np.testing.assert_allclose(f, fr, rtol=1e-13)
    np.testing.assert_allclose(S, Sr, rtol=0, atol=1e-10 * np.abs(Sr).max())


@pytest.mark.parametrize("kind,C", [(0, 3), (2, 9)])
def test_noalloc_at_its_layout_bound_against_oracle(tn, kind, C):
    """T = TNEP_NOALLOC_MAX_T and max_lag = T - 1 fill the static scratch to
    its bound (signal T*C, ACF M+1, cosine table 2M).  The ACF is compared
    at every lag and the spectrum at 64 frequencies with the FP64 oracle."""
    import oracle
    rng = np.random.default_rng(12 + kind)
    T = tn.TNEP_NOALLOC_MAX_T
    t = np.arange(T)
    series = rng.normal(size=(T, C)) + np.cos(0.01 * t)[:, None] * rng.normal(size=C)
    f, S, A = _run_noalloc(tn, series, kind, T - 1)
    Cr = oracle.acf(series, T - 1, kind)
    np.testing.assert_allclose(A, Cr, rtol=0, atol=1e-11 * np.abs(Cr).max())
    ks = np.unique(np.concatenate([[0, 1, T - 2, T - 1], rng.integers(0, T, 60)]))
    fr, Sr = oracle.spectrum(series, 0.5, kind, max_lag=T - 1, k_sel=ks)
    np.testing.assert_allclose(f[ks], fr, rtol=1e-13)
    np.testing.assert_allclose(S[ks], Sr, rtol=0, atol=1e-9 * np.abs(Sr).max())


def test_noalloc_rejects_oversized_series(tn):
    dev = torch.device("cuda")
    T = tn.TNEP_NOALLOC_MAX_T + 1
    s = torch.zeros((T, 3), dtype=torch.float64, device=dev)
    f = torch.empty(T // 2 + 1, dtype=torch.float64, device=dev)
    p = torch.empty(T // 2 + 1, dtype=torch.float64, device=dev)
    with pytest.raises(tn.TnepError) as e:
        tn.tnep_spectrum_noalloc(s, 1.0, tn.TNEP_SPECTRUM_IR, f, p)
    assert e.value.status == 1 and "TNEP_NOALLOC_MAX_T" in str(e.value)
