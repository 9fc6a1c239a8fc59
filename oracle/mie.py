"""Mie series for a PEC sphere (oracle pin; textbook closed form, not from the paper).

Scattering amplitudes (Bohren-Huffman form, perfect-conductor limit):
  a_n = psi_n'(x)/xi_n'(x),  b_n = psi_n(x)/xi_n(x),  x = k a,
  psi_n = x j_n(x), xi_n = x h_n^(1)(x),
  S1 = sum_n (2n+1)/(n(n+1)) (a_n pi_n + b_n tau_n),
  S2 = sum_n (2n+1)/(n(n+1)) (a_n tau_n + b_n pi_n),
with pi_n = P_n^1(cos T)/sin T, tau_n = dP_n^1/dT, T the scattering angle.
Bistatic RCS: E-plane sigma = 4 pi |S2|^2/k^2, H-plane sigma = 4 pi |S1|^2/k^2.
|S|^2 does not depend on the time convention.
"""
from __future__ import annotations

import numpy as np
from scipy.special import spherical_jn, spherical_yn


def pec_sphere_rcs(ka: float, k: float, scat_angle: np.ndarray, nmax: int | None = None):
    """(sigma_E_plane, sigma_H_plane) at scattering angles T (radians from forward)."""
    x = float(ka)
    if nmax is None:
        nmax = int(x + 4.0 * x ** (1.0 / 3.0) + 10)
    n = np.arange(1, nmax + 1)
    jn = spherical_jn(n, x)
    jnp = spherical_jn(n, x, derivative=True)
    yn = spherical_yn(n, x)
    ynp = spherical_yn(n, x, derivative=True)
    psi = x * jn
    dpsi = jn + x * jnp
    hn = jn + 1j * yn
    dhn = jnp + 1j * ynp
    xi = x * hn
    dxi = hn + x * dhn
    a = dpsi / dxi
    b = psi / xi
    mu = np.cos(np.atleast_1d(scat_angle))
    S1 = np.zeros(mu.shape, dtype=np.complex128)
    S2 = np.zeros(mu.shape, dtype=np.complex128)
    pi_prev = np.zeros_like(mu)
    pi_cur = np.ones_like(mu)
    for i, nn in enumerate(n):
        if nn == 1:
            pi_n = np.ones_like(mu)
        else:
            pi_n = ((2 * nn - 1) / (nn - 1)) * mu * pi_cur - (nn / (nn - 1)) * pi_prev
        tau_n = nn * mu * pi_n - (nn + 1) * (pi_cur if nn > 1 else np.zeros_like(mu))
        c = (2 * nn + 1) / (nn * (nn + 1))
        S1 += c * (a[i] * pi_n + b[i] * tau_n)
        S2 += c * (a[i] * tau_n + b[i] * pi_n)
        if nn > 1:
            pi_prev = pi_cur
        pi_cur = pi_n
    return 4 * np.pi * np.abs(S2) ** 2 / k ** 2, 4 * np.pi * np.abs(S1) ** 2 / k ** 2
