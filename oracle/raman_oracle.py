"""FP64 CPU oracle of the polarized Raman tail -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and ``bench.py`` may import this
module; it shares no code with the CUDA kernels.

Sec. II.G: the Stokes cross-section for observed polarization n and incoming
polarization eps is sum_{gamma delta mu nu} n_gamma n_mu L_{gamma delta mu nu}(omega)
eps_delta eps_nu (Eq. 7), with the lineshape tensor L the Fourier transform of
<alpha_{gamma delta}(0) alpha_{mu nu}(t)> (Eq. 8).  Readings (the paper is
silent on the estimator):

* correlation of components p = (gamma, delta), q = (mu, nu), tau = 0..M:
      C_pq(tau) = 1/(T - tau) sum_{t=0}^{T-1-tau} a_p(t) a_q(t + tau),
  each component's mean removed first when asked (as for the iso / aniso
  spectra);
* only the part of L that any polarization contraction sees is kept: the
  weights n_gamma eps_delta n_mu eps_nu are symmetric under p <-> q, so the
  contraction takes S_pq = (C_pq + C_qp) / 2, which is even in t and has the
  real cosine transform
      L_pq(nu_k) = dt [S_pq(0) + 2 sum_{tau=1}^{M} S_pq(tau) cos(pi k tau / M)],
  nu_k = k / (2 M dt), the same transform as the iso / aniso spectra;
* spectrum for one (n, eps): sum_pq w_p w_q L_pq with w = vec(n eps^T).
  Parallel / crossed polarization in Porto notation, Z(XX)Z-bar and
  Z(XY)Z-bar (Sec. IV, BaZrO3), are eps = X, n = X or n = Y of the crystal
  frame seen by the laser; rotating the crystal by R turns them into R^T X,
  R^T Y.
"""

from __future__ import annotations

import numpy as np

from .tnep_oracle import WAVENUMBER_PER_INV_FS

__all__ = ["raman_correlations", "raman_tensor", "raman_polarized", "porto_vectors"]


def raman_correlations(series, max_lag=None, subtract_mean=True):
    """S [M+1][9][9]: symmetrised component cross-correlations (row-major 3x3)."""
    a = np.asarray(series, dtype=np.float64).reshape(len(series), 9)
    T = a.shape[0]
    M = T // 2 if max_lag is None else int(max_lag)
    if subtract_mean:
        a = a - a.mean(0)
    C = np.stack([a[:T - t].T @ a[t:] / (T - t) for t in range(M + 1)])
    return 0.5 * (C + C.transpose(0, 2, 1))


def raman_tensor(series, dt_fs, max_lag=None, subtract_mean=True):
    """(frequency in cm^-1 [M+1], L [M+1][3][3][3][3]) -- Eq. 8, real symmetric part."""
    S = raman_correlations(series, max_lag, subtract_mean)
    M = S.shape[0] - 1
    k = np.arange(M + 1)
    tau = np.arange(1, M + 1)
    nu = k / (2.0 * M * dt_fs) if M > 0 else np.zeros(1)
    cos = np.cos(np.pi * np.outer(k, tau) / max(M, 1))
    L = dt_fs * (S[0][None] + 2.0 * np.einsum("kt,tpq->kpq", cos, S[1:]))
    return nu * WAVENUMBER_PER_INV_FS, L.reshape(M + 1, 3, 3, 3, 3)


def raman_polarized(L, n, eps):
    """Eq. 7 for each (n_o, eps_o): spec [O][M+1]."""
    n = np.atleast_2d(np.asarray(n, dtype=np.float64))
    eps = np.atleast_2d(np.asarray(eps, dtype=np.float64))
    return np.einsum("og,od,om,on,kgdmn->ok", n, eps, n, eps, L)


def porto_vectors(thetas, axis=2):
    """Polarization vectors of Z(XX)Z-bar and Z(XY)Z-bar for a crystal turned
    by theta about its `axis` (the laser direction): rows of eps, n_par, n_cross."""
    th = np.asarray(thetas, dtype=np.float64)
    c, s = np.cos(th), np.sin(th)
    i, j = [(1, 2), (2, 0), (0, 1)][axis]
    eps = np.zeros((len(th), 3))
    ncr = np.zeros((len(th), 3))
    eps[:, i], eps[:, j] = c, -s   # R(theta)^T X in the crystal frame
    ncr[:, i], ncr[:, j] = s, c    # R(theta)^T Y
    return eps, eps.copy(), ncr
