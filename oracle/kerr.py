"""Single-mode quartic (Kerr) oscillator of Fig. 2 (oracle; test infrastructure only).

H = (Lam / 2) a^dag a^dag a a.  Starting from the coherent state |z>:
  exact quantum   <a(t)> = z exp(|z|^2 (exp(-i Lam t) - 1))
  TWA trajectory  alpha(t) = alpha0 exp(-i Lam (|alpha0|^2 - 1) t)
(the Weyl symbol of a^dag a^dag a a is |alpha|^4 - 2|alpha|^2 + 1/2, whose
derivative d/d alpha* gives the -1 in the frequency).  For alpha0 drawn from
the coherent-state Wigner function (complex Gaussian around z with
E|alpha0 - z|^2 = s, s = 1/2) the TWA ensemble mean has the closed form
  <alpha(t)> = e^{i th} z / (1 + i th s)^2 exp(-i th |z|^2 / (1 + i th s)),  th = Lam t,
from the Gaussian integral E[alpha exp(-lam |alpha|^2)].
"""
from __future__ import annotations

import numpy as np


def exact_mean(z: complex, lam: float, t):
    t = np.asarray(t, dtype=np.float64)
    return z * np.exp(abs(z) ** 2 * (np.exp(-1j * lam * t) - 1.0))


def twa_trajectory(alpha0, lam: float, t: float):
    return alpha0 * np.exp(-1j * lam * (np.abs(alpha0) ** 2 - 1.0) * t)


def twa_mean_closed_form(z: complex, lam: float, t, s: float = 0.5):
    th = lam * np.asarray(t, dtype=np.float64)
    den = 1.0 + 1j * th * s
    return np.exp(1j * th) * z / den ** 2 * np.exp(-1j * th * abs(z) ** 2 / den)
