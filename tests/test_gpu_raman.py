"""Polarized Raman tail (Sec. II.G, Eqs. 7-8) through the C ABI against the
FP64 oracle: the lineshape tensor element by element, the polarization
contraction and the Porto orientation map, from tiny to the BaZrO3-length
series (500 ps at 5 fs)."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
DT = 5.0


@pytest.fixture(scope="module")
def tn():
    import __graft_entry__ as g
    g.build()
    from paper_2312_05233_gb300 import tnep
    return tnep


def _series(T, seed, symmetric=True):
    return synth.tensor_series(T, np.random.default_rng(synth.seed_for(7, seed)), symmetric=symmetric)


def _close(got, ref, rel=1e-10):
    np.testing.assert_allclose(got, ref, rtol=0, atol=rel * np.abs(ref).max())


@pytest.mark.parametrize("T,M,sym,sub", [(3000, 500, True, True), (3000, 7, False, True), (777, 776, True, False),
                                         (2, 1, False, True), (1000, 513, False, False),
                                         # long enough for the Fourier route (81 T M > 1e9)
                                         (20000, 3001, False, True), (8193, 8192, True, False)])
def test_tensor_matches_oracle(tn, T, M, sym, sub):
    a = _series(T, T + M, sym)
    f, L = tn.tnep_raman_tensor(a, DT, M, sub)
    fo, Lo = oracle.raman_tensor(a, DT, M, sub)
    np.testing.assert_allclose(f, fo, rtol=1e-14)
    _close(L, Lo.reshape(M + 1, 9, 9))


def test_polarized_and_porto_match_oracle(tn):
    a = _series(2000, 1)
    _, L = tn.tnep_raman_tensor(a, DT, 300)
    _, Lo = oracle.raman_tensor(a, DT, 300)
    rng = np.random.default_rng(3)
    n, e = rng.normal(size=(17, 3)), rng.normal(size=(17, 3))
    _close(tn.tnep_raman_polarized(L, n, e), oracle.raman_polarized(Lo, n, e))
    th = np.linspace(0, np.pi, 37)
    for axis in (0, 1, 2):
        par, crs = tn.tnep_raman_porto_map(L, th, axis)
        eps, npar, ncr = oracle.porto_vectors(th, axis)
        _close(par, oracle.raman_polarized(Lo, npar, eps))
        _close(crs, oracle.raman_polarized(Lo, ncr, eps))


def test_bazro3_length_series(tn):
    # 500 ps at 5 fs: T = 100,000 samples, lags up to 10 ps
    T, M = 100_000, 2000
    a = _series(T, 5)
    f, L = tn.tnep_raman_tensor(a, DT, M)
    _, Lo = oracle.raman_tensor(a, DT, M)
    _close(L, Lo.reshape(M + 1, 9, 9), rel=1e-9)
    # the isotropic averages of the GPU's own polarized spectra reproduce its
    # iso / aniso spectra (12 icosahedron vertices: a spherical 5-design)
    phi = (1 + 5 ** 0.5) / 2
    V = []
    for s1 in (1, -1):
        for s2 in (1, -1):
            V += [(0, s1, s2 * phi), (s1, s2 * phi, 0), (s2 * phi, 0, s1)]
    V = np.array(V) / np.linalg.norm(V[0])
    par = tn.tnep_raman_polarized(L, V, V).mean(0)
    _, iso = tn.tnep_spectrum(a, DT, tn.TNEP_SPECTRUM_RAMAN_ISO, M)
    _, aniso = tn.tnep_spectrum(a, DT, tn.TNEP_SPECTRUM_RAMAN_ANISO, M)
    _close(par, iso + 2.0 / 15.0 * aniso, rel=1e-9)
