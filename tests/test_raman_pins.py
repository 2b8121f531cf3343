"""Pins of the polarized Raman oracle (Sec. II.G, Eqs. 7-8) against the
independently pinned iso / aniso spectra, the isotropic-average identities
of Raman scattering and exact closed forms."""

import numpy as np
import pytest

import oracle
import synth

DT = 5.0


def _series(T=600, seed=1, symmetric=True):
    return synth.tensor_series(T, np.random.default_rng(synth.seed_for(7, seed)), symmetric=symmetric)


def _icosahedron():
    phi = (1 + 5 ** 0.5) / 2
    v = []
    for s1 in (1, -1):
        for s2 in (1, -1):
            v += [(0, s1, s2 * phi), (s1, s2 * phi, 0), (s2 * phi, 0, s1)]
    v = np.array(v, float)
    return v / np.linalg.norm(v, axis=1)[:, None]


def test_single_elements_equal_scalar_spectra():
    a = _series(T=400, symmetric=False)
    _, L = oracle.raman_tensor(a, DT, max_lag=120)
    e = np.eye(3)
    for i, j in [(0, 0), (1, 2), (2, 1), (0, 2)]:
        # the iso spectrum of c(t) I is the plain spectrum of the scalar c(t)
        c = a.reshape(-1, 3, 3)[:, i, j]
        _, ref = oracle.spectrum(np.einsum("t,ab->tab", c, np.eye(3)).reshape(-1, 9), DT,
                                 oracle.KIND_RAMAN_ISO, max_lag=120)
        got = oracle.raman_polarized(L, e[i], e[j])[0]
        np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_isotropic_averages_give_iso_and_aniso():
    # The 12 icosahedron vertices are a spherical 5-design, so their mean is
    # the exact isotropic average of the degree-4 intensities:
    #   parallel <(e.a e)^2> = gamma^2 + 2/15 Tr(beta^2)
    #   crossed  <(n.a e)^2> = Tr(beta^2) / 10   (n uniform on the circle orthogonal to e)
    a = _series(T=500)
    _, L = oracle.raman_tensor(a, DT, max_lag=150)
    V = _icosahedron()
    par = oracle.raman_polarized(L, V, V).mean(0)
    ns, es = [], []
    for v in V:
        t = np.cross(v, [0.3, 0.5, 0.7]); t /= np.linalg.norm(t)
        u = np.cross(v, t)
        for k in range(4):
            th = 0.5 * np.pi * k
            ns.append(np.cos(th) * t + np.sin(th) * u)
            es.append(v)
    cr = oracle.raman_polarized(L, np.array(ns), np.array(es)).mean(0)
    _, iso = oracle.spectrum(a, DT, oracle.KIND_RAMAN_ISO, max_lag=150)
    _, aniso = oracle.spectrum(a, DT, oracle.KIND_RAMAN_ANISO, max_lag=150)
    scale = np.abs(iso).max() + np.abs(aniso).max()
    np.testing.assert_allclose(par, iso + 2.0 / 15.0 * aniso, rtol=0, atol=1e-10 * scale)
    np.testing.assert_allclose(cr, aniso / 10.0, rtol=0, atol=1e-10 * scale)


def test_rotating_sample_and_light_together_changes_nothing():
    a = _series(T=300, seed=2)
    R = synth.random_rotation(np.random.default_rng(4))
    ar = np.einsum("ij,tjk,lk->til", R, a.reshape(-1, 3, 3), R).reshape(-1, 9)
    _, L = oracle.raman_tensor(a, DT, max_lag=90)
    _, Lr = oracle.raman_tensor(ar, DT, max_lag=90)
    rng = np.random.default_rng(5)
    n, e = rng.normal(size=(6, 3)), rng.normal(size=(6, 3))
    got = oracle.raman_polarized(Lr, n @ R.T, e @ R.T)
    ref = oracle.raman_polarized(L, n, e)
    np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())


def test_single_tensor_mode_spectra_are_proportional():
    # alpha(t) = A f(t): every polarization sees (n.A eps)^2 times one spectrum
    rng = np.random.default_rng(6)
    A = rng.normal(size=(3, 3))
    f = synth.tensor_series(400, rng)[:, 0]
    a = (f[:, None, None] * A).reshape(-1, 9)
    _, L = oracle.raman_tensor(a, DT, max_lag=100)
    n, e = rng.normal(size=(4, 3)), rng.normal(size=(4, 3))
    sp = oracle.raman_polarized(L, n, e)
    w = np.einsum("og,gd,od->o", n, A, e) ** 2
    base = sp[0] / w[0]
    for o in range(1, 4):
        np.testing.assert_allclose(sp[o], w[o] * base, rtol=1e-9, atol=1e-12 * np.abs(sp).max())


def test_tensor_symmetry_and_porto_period():
    a = _series(T=200, seed=3, symmetric=False)
    _, L = oracle.raman_tensor(a, DT, max_lag=60)
    Lf = L.reshape(L.shape[0], 9, 9)
    np.testing.assert_allclose(Lf, Lf.transpose(0, 2, 1), rtol=0, atol=1e-14 * np.abs(Lf).max())
    th = np.array([0.3, 0.3 + np.pi, 1.1])
    eps, npar, ncr = oracle.porto_vectors(th)
    assert np.allclose(np.einsum("oi,oi->o", eps, ncr), 0) and np.allclose(np.linalg.norm(eps, axis=1), 1)
    sp = oracle.raman_polarized(L, npar, eps)
    np.testing.assert_allclose(sp[0], sp[1], rtol=1e-12, atol=1e-14 * np.abs(sp).max())
