"""FP64 CPU oracle of the training loop -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and ``bench.py`` may import this
module; it imports nothing from the product package and shares no code with
the CUDA kernels.

The paper trains TNEP models with the separable natural evolution strategy
(SNES, Sec. II.D) on a loss made of the RMSE of the tensor plus L1 and L2
regularization terms (Sec. II.D, the dipole and polarizability losses).  It
defers both the optimiser and the regularization terms to the cited
references; the readings used here are:

* loss of a parameter vector z of dimension d:
      L(z) = RMSE(z) + lambda1 * (1/d) sum_i |z_i| + lambda2 * sqrt((1/d) sum_i z_i^2)
  (the regularization form of the NEP papers).
* one SNES generation (Schaul, Glasmachers and Schmidhuber 2011; Wierstra
  et al. 2014), population size lambda:
      s_k ~ N(0, I_d),  z_k = mu + sigma * s_k                 k = 1..lambda
      rank the z_k by L ascending (ties: lower k first), rank 1 = best
      u_r = max(0, ln(lambda/2 + 1) - ln r) / sum_j max(0, ln(lambda/2 + 1) - ln j) - 1/lambda
      grad_mu    = sum_k u_{r(k)} s_k
      grad_sigma = sum_k u_{r(k)} (s_k^2 - 1)
      mu    <- mu + eta_mu * sigma * grad_mu
      sigma <- sigma * exp(eta_sigma / 2 * grad_sigma)
  with the published defaults eta_mu = 1, eta_sigma = (3 + ln d) / (5 sqrt d).
* the normal samples come from the counter-based generator Philox4x64-10
  (Salmon, Moraes, Dror and Shaw 2011) and the Box-Muller transform:
  block b (parameters 4b..4b+3) of individual k at generation g uses counter
  (b, k, g, 0) and key (seed, 0); each 64-bit output x gives
  u = (floor(x / 2^12) + 1/2) 2^-52 in (0, 1); outputs (x0, x1) and (x2, x3)
  give the pairs sqrt(-2 ln u_a) (cos 2 pi u_b, sin 2 pi u_b).
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "philox4x64_10", "snes_normals", "snes_utilities", "default_eta_sigma", "regularization",
    "snes_update", "snes_generation", "PHILOX_M", "PHILOX_W",
]

# Philox4x64 multipliers and Weyl key increments (Salmon et al. 2011, Table 2 and Sec. 5).
PHILOX_M = (0xD2E7470EE14C6C93, 0xCA5A826395121157)
PHILOX_W = (0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B)
_M32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo(a, b):
    """High and low 64-bit words of the 128-bit product a * b (uint64 arrays)."""
    a0, a1 = a & _M32, a >> _S32
    b0, b1 = b & _M32, b >> _S32
    p00, p01, p10, p11 = a0 * b0, a0 * b1, a1 * b0, a1 * b1
    mid = (p00 >> _S32) + (p01 & _M32) + (p10 & _M32)
    hi = p11 + (p01 >> _S32) + (p10 >> _S32) + (mid >> _S32)
    return hi, a * b


def philox4x64_10(ctr, key):
    """Philox4x64 with 10 rounds.  ctr: uint64 [..., 4]; key: two uint64.
    Returns uint64 [..., 4]."""
    c = [np.asarray(ctr[..., w], dtype=np.uint64).copy() for w in range(4)]
    k0, k1 = np.uint64(key[0]), np.uint64(key[1])
    m0, m1 = np.uint64(PHILOX_M[0]), np.uint64(PHILOX_M[1])
    w0, w1 = np.uint64(PHILOX_W[0]), np.uint64(PHILOX_W[1])
    with np.errstate(over="ignore"):
        for r in range(10):
            hi0, lo0 = _mulhilo(m0, c[0])
            hi1, lo1 = _mulhilo(m1, c[2])
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
            k0 = k0 + w0
            k1 = k1 + w1
    return np.stack(c, axis=-1)


def _uniform(x):
    return ((x >> np.uint64(12)).astype(np.float64) + 0.5) * 2.0 ** -52


def snes_normals(seed, generation, n_pop, dim):
    """Standard normals s [n_pop][dim] of one generation (see the module notes)."""
    nb = (dim + 3) // 4
    ctr = np.zeros((n_pop, nb, 4), dtype=np.uint64)
    ctr[:, :, 0] = np.arange(nb, dtype=np.uint64)[None, :]
    ctr[:, :, 1] = np.arange(n_pop, dtype=np.uint64)[:, None]
    ctr[:, :, 2] = np.uint64(generation)
    x = philox4x64_10(ctr, (np.uint64(seed), np.uint64(0)))
    u = _uniform(x)
    out = np.empty((n_pop, nb, 4))
    for pair in range(2):
        rad = np.sqrt(-2.0 * np.log(u[..., 2 * pair]))
        ang = 2.0 * np.pi * u[..., 2 * pair + 1]
        out[..., 2 * pair] = rad * np.cos(ang)
        out[..., 2 * pair + 1] = rad * np.sin(ang)
    return out.reshape(n_pop, nb * 4)[:, :dim]


def snes_utilities(n_pop):
    """Rank-based utilities u_r, r = 1..n_pop (index 0 = best)."""
    r = np.arange(1, n_pop + 1, dtype=np.float64)
    w = np.maximum(0.0, np.log(n_pop / 2.0 + 1.0) - np.log(r))
    return w / w.sum() - 1.0 / n_pop


def default_eta_sigma(dim):
    return (3.0 + np.log(dim)) / (5.0 * np.sqrt(dim))


def regularization(z, lambda1, lambda2):
    """L1 and L2 terms of the loss for each row of z [..., d]."""
    z = np.asarray(z, dtype=np.float64)
    d = z.shape[-1]
    return lambda1 * np.abs(z).sum(-1) / d + lambda2 * np.sqrt((z * z).sum(-1) / d)


def _ranks(loss):
    """rank[k] in 1..P of individual k (ascending loss, ties by index)."""
    order = np.argsort(np.asarray(loss), kind="stable")
    rank = np.empty(len(order), dtype=np.int64)
    rank[order] = np.arange(1, len(order) + 1)
    return rank


def snes_update(mu, sigma, s, loss, eta_mu, eta_sigma):
    """One SNES update of (mu, sigma) from the samples s [P][d] and their losses [P]."""
    s = np.asarray(s, dtype=np.float64)
    util = snes_utilities(len(loss))[_ranks(loss) - 1]
    g_mu = util @ s
    g_sigma = util @ (s * s - 1.0)
    mu_new = mu + eta_mu * sigma * g_mu
    sigma_new = sigma * np.exp(0.5 * eta_sigma * g_sigma)
    return mu_new, sigma_new


def snes_generation(mu, sigma, generation, seed, n_pop, rmse_fn, lambda1=0.0, lambda2=0.0, eta_mu=1.0,
                    eta_sigma=None):
    """One generation: sample, evaluate rmse_fn(z) for every individual, add
    the regularization, update.  Returns (mu, sigma, loss [P], rmse [P])."""
    d = len(mu)
    if eta_sigma is None:
        eta_sigma = default_eta_sigma(d)
    s = snes_normals(seed, generation, n_pop, d)
    z = mu[None, :] + sigma[None, :] * s
    rmse = np.array([rmse_fn(z[k]) for k in range(n_pop)])
    loss = rmse + regularization(z, lambda1, lambda2)
    mu_new, sigma_new = snes_update(mu, sigma, s, loss, eta_mu, eta_sigma)
    return mu_new, sigma_new, loss, rmse
