"""Exact Fock-space evolution of the lattice Schroedinger-Poisson Hamiltonian (oracle).

Test infrastructure only (see ``oracle/__init__``).

The quantum Hamiltonian of Eq. eqn_Ham, restricted to the M cells of a 1D
periodic lattice, in number units b_g = sqrt(n dx) psi_g:
    H = sum_gh T_gh a_g^dag a_h + 1/2 sum_gh K_gh a_g^dag a_h^dag a_h a_g
with
    T_gh = (1/M) sum_k (hbar k^2 / 2) exp(i k (x_g - x_h))          (kinetic term)
    K_gh = C G_gh / (n dx hbar),  G_gh = (1/M) sum_{k != 0} (-1/k^2) exp(i k (x_g - x_h))
(the lattice Green's function of the Poisson equation with the k = 0 mode
removed).  Its mean-field limit is exactly the lattice form of Eq. mft_normed,
so the TWA of this Hamiltonian is the oracle's split-step evolution of sampled
fields.  The Weyl symbol of the quartic term differs from the classical one by
-1/2 sum_g K_gg |alpha_g|^2 (because sum_h K_gh = 0), a global phase that
leaves every a^dag a moment unchanged.

The initial state is the coherent state of Eq. eqn_coherentStates with
amplitudes z_g = sqrt(n dx) psi_cl(x_g).  H conserves the particle number, so
each N-sector (dimension C(N+M-1, M-1)) is evolved separately with
scipy.sparse.linalg.expm_multiply, for N up to ``n_max``.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sps
from scipy.sparse.linalg import expm_multiply


def lattice_operators(M: int, L: float, hbar: float, C: float, n_tot: float):
    """(T, K) matrices of the module docstring (real symmetric M x M)."""
    dx = L / M
    x = np.arange(M) * dx
    k = 2.0 * np.pi * np.fft.fftfreq(M, d=dx)
    d = x[:, None] - x[None, :]
    E = np.exp(1j * k[None, None, :] * d[:, :, None])
    T = (E * (0.5 * hbar * k ** 2)[None, None, :]).sum(-1).real / M
    ginv = np.zeros(M)
    ginv[k != 0] = -1.0 / k[k != 0] ** 2
    G = (E * ginv[None, None, :]).sum(-1).real / M
    K = C * G / (n_tot * dx * hbar)
    return T, K


def _basis(N: int, M: int) -> np.ndarray:
    """All occupation vectors of M sites with total N (rows), in a fixed order."""
    if M == 1:
        return np.array([[N]], dtype=np.int64)
    parts = []
    for first in range(N, -1, -1):
        rest = _basis(N - first, M - 1)
        parts.append(np.concatenate([np.full((len(rest), 1), first, dtype=np.int64), rest], axis=1))
    return np.concatenate(parts, axis=0)


def _keys(states: np.ndarray, base: int) -> np.ndarray:
    return states @ (base ** np.arange(states.shape[1], dtype=np.int64))


def _lowering(states_hi: np.ndarray, states_lo: np.ndarray, h: int, base: int):
    """Sparse a_h from the N sector (columns) to the N-1 sector (rows)."""
    keys_lo = _keys(states_lo, base)
    order = np.argsort(keys_lo)
    src = np.nonzero(states_hi[:, h] > 0)[0]
    tgt_keys = _keys(states_hi[src], base) - base ** h
    pos = order[np.searchsorted(keys_lo, tgt_keys, sorter=order)]
    vals = np.sqrt(states_hi[src, h].astype(np.float64))
    return sps.csr_matrix((vals, (pos, src)), shape=(len(states_lo), len(states_hi)))


def _coherent_sector(states: np.ndarray, z: np.ndarray) -> np.ndarray:
    """Sector component of the coherent state exp(-|z|^2/2) prod_g z_g^n_g / sqrt(n_g!)."""
    lg = np.vectorize(math.lgamma)
    logc = (states * np.log(z.astype(np.complex128) + 0j)[None, :]).sum(1) - 0.5 * lg(states + 1.0).sum(1)
    return np.exp(logc - 0.5 * np.sum(np.abs(z) ** 2))


def mode_occupations(psi_cl: np.ndarray, L: float, hbar: float, C: float, n_tot: float,
                     times, n_max: int = 40):
    """Exact <a_k^dag a_k> and Var(a_k^dag a_k) at ``times`` for the coherent initial state.

    a_k = M^{-1/2} sum_g exp(-i k x_g) a_g (unitary DFT, the same convention as the
    oracle's moments).  Returns (nk_mean, nk_var, total_prob) with arrays of
    shape (len(times), M); total_prob is the norm captured by N <= n_max.
    """
    M = psi_cl.size
    dx = L / M
    base = n_max + 2
    z = math.sqrt(n_tot * dx) * psi_cl.astype(np.complex128)
    T, K = lattice_operators(M, L, hbar, C, n_tot)
    times = np.asarray(times, dtype=np.float64)
    x = np.arange(M) * dx
    k = 2.0 * np.pi * np.fft.fftfreq(M, d=dx)
    U = np.exp(-1j * np.outer(k, x)) / math.sqrt(M)      # a_k = sum_g U[k, g] a_g
    nk = np.zeros((len(times), M))
    nk2 = np.zeros((len(times), M))
    prob = np.zeros(len(times))
    states_lo = _basis(0, M)
    prob += np.sum(np.abs(_coherent_sector(states_lo, z)) ** 2)
    for N in range(1, n_max + 1):
        states = _basis(N, M)
        c0 = _coherent_sector(states, z)
        A = [_lowering(states, states_lo, h, base) for h in range(M)]
        n = states.astype(np.float64)
        diag = n @ np.diag(T) + 0.5 * np.einsum("sg,gh,sh->s", n, K, n) - 0.5 * n @ np.diag(K)
        H = sps.diags(diag).tocsr()
        for g in range(M):
            for h in range(M):
                if g != h:
                    H = H + T[g, h] * (A[g].T @ A[h])
        H = H.tocsc()
        Ak = [sum(U[kk, h] * A[h] for h in range(M)).tocsr() for kk in range(M)]
        for ti, t in enumerate(times):
            ct = c0 if t == 0.0 else expm_multiply(-1j * t * H, c0)
            prob[ti] += np.sum(np.abs(ct) ** 2)
            for kk in range(M):
                uk = Ak[kk] @ ct
                nk[ti, kk] += np.vdot(uk, uk).real
                v = Ak[kk].conj().T @ uk
                nk2[ti, kk] += np.vdot(v, v).real
        states_lo = states
    return nk, nk2 - nk ** 2, prob
