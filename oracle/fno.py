"""FP64 reference of the Fourier-neural-operator surrogate (oracle; test infrastructure only).

The surrogate maps per-mode features of a TWA run (on the grid of Fourier modes of the field) to
the ensemble-averaged correction spectrum <n_k> - n_k^cl.  It is not part of the paper; the
network follows the standard Fourier neural operator:

  h_0 = P x + p                                  (pointwise lift, C_in -> W channels)
  z_l = Re F^-1[ R_l . F_trunc[h_l] ] + W_l h_l + b_l        l = 0..L-1
  h_{l+1} = gelu(z_l)  (l < L-1),  h_L = z_{L-1}
  y = Q h_L + q                                  (pointwise projection, W -> C_out)

F_trunc is the unitary ("ortho") 3D DFT restricted to the frequencies |m_a| < modes on every axis
(m in {0..modes-1} U {N-modes..N-1}); F^-1 is its adjoint (zero-padded unitary inverse).  R_l holds
one complex W x W matrix per retained mode.  gelu(x) = x Phi(x) with the exact normal CDF.

Parameters are one flat float vector, in this order: P (W x C_in), p (W); per layer R (modes^3 of
2*modes per axis, W, W, re/im interleaved), W_l (W x W), b_l (W); Q (C_out x W), q (C_out).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def kept(n: int, modes: int) -> np.ndarray:
    return np.concatenate([np.arange(modes), np.arange(n - modes, n)])


def param_shapes(W: int, c_in: int, c_out: int, modes: int, layers: int):
    M = (2 * modes) ** 3
    shapes = [("P", (W, c_in)), ("p", (W,))]
    for l in range(layers):
        shapes += [(f"R{l}", (M, W, W, 2)), (f"W{l}", (W, W)), (f"b{l}", (W,))]
    shapes += [("Q", (c_out, W)), ("q", (c_out,))]
    return shapes


def unpack(theta: np.ndarray, W, c_in, c_out, modes, layers):
    out, o = {}, 0
    for name, sh in param_shapes(W, c_in, c_out, modes, layers):
        n = int(np.prod(sh))
        out[name] = theta[o:o + n].reshape(sh)
        o += n
    assert o == theta.size
    return out


def num_params(W, c_in, c_out, modes, layers):
    return sum(int(np.prod(sh)) for _, sh in param_shapes(W, c_in, c_out, modes, layers))


def _gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def _gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def _dft_trunc(h, n, modes):
    """Unitary DFT over the last three axes, restricted to the kept frequencies (complex)."""
    k = kept(n, modes)
    s = np.fft.fftn(h, axes=(-3, -2, -1), norm="ortho")
    return s[..., k[:, None, None], k[None, :, None], k[None, None, :]]


def _idft_trunc(s, n, modes):
    """Adjoint of _dft_trunc: zero-pad the kept frequencies and take the unitary inverse DFT."""
    k = kept(n, modes)
    full = np.zeros(s.shape[:-3] + (n, n, n), dtype=np.complex128)
    full[..., k[:, None, None], k[None, :, None], k[None, None, :]] = s
    return np.fft.ifftn(full, axes=(-3, -2, -1), norm="ortho")


def forward(theta, x, W, c_in, c_out, modes, layers, keep=False):
    """x: (B, C_in, N, N, N) -> y: (B, C_out, N, N, N)."""
    p = unpack(theta, W, c_in, c_out, modes, layers)
    n = x.shape[-1]
    h = np.einsum("oc,bc...->bo...", p["P"], x) + p["p"][None, :, None, None, None]
    cache = {"x": x, "h": [], "s": [], "z": []}
    for l in range(layers):
        R = p[f"R{l}"][..., 0] + 1j * p[f"R{l}"][..., 1]              # (M, W_out, W_in)
        s = _dft_trunc(h, n, modes)                                    # (B, W, m, m, m)
        B = s.shape[0]
        sf = s.reshape(B, W, -1)                                       # (B, W, M)
        mixed = np.einsum("moc,bcm->bom", R, sf).reshape(s.shape)
        u = _idft_trunc(mixed, n, modes).real
        z = u + np.einsum("oc,bc...->bo...", p[f"W{l}"], h) + p[f"b{l}"][None, :, None, None, None]
        cache["h"].append(h)
        cache["s"].append(sf)
        cache["z"].append(z)
        h = _gelu(z) if l < layers - 1 else z
    cache["h"].append(h)
    y = np.einsum("oc,bc...->bo...", p["Q"], h) + p["q"][None, :, None, None, None]
    return (y, cache) if keep else y


def backward(theta, cache, dy, W, c_in, c_out, modes, layers):
    """Gradient of a real scalar loss L with dL/dy = dy; returns (dtheta flat, dx)."""
    p = unpack(theta, W, c_in, c_out, modes, layers)
    g = {name: np.zeros(sh) for name, sh in param_shapes(W, c_in, c_out, modes, layers)}
    n = dy.shape[-1]
    hL = cache["h"][layers]
    g["Q"] = np.einsum("boxyz,bcxyz->oc", dy, hL)
    g["q"] = dy.sum(axis=(0, 2, 3, 4))
    dh = np.einsum("oc,bo...->bc...", p["Q"], dy)
    for l in reversed(range(layers)):
        z = cache["z"][l]
        dz = dh * _gelu_grad(z) if l < layers - 1 else dh
        h = cache["h"][l]
        g[f"W{l}"] = np.einsum("boxyz,bcxyz->oc", dz, h)
        g[f"b{l}"] = dz.sum(axis=(0, 2, 3, 4))
        dh = np.einsum("oc,bo...->bc...", p[f"W{l}"], dz)
        # spectral branch: u = Re(A* (R . A h)) with A the truncated unitary DFT
        B = dz.shape[0]
        dmixed = _dft_trunc(dz.astype(np.complex128), n, modes).reshape(B, W, -1)   # A dz (adjoint of A*)
        R = p[f"R{l}"][..., 0] + 1j * p[f"R{l}"][..., 1]
        sf = cache["s"][l]
        dR = np.einsum("bom,bcm->moc", dmixed, np.conj(sf))
        g[f"R{l}"] = np.stack([dR.real, dR.imag], axis=-1)
        ds = np.einsum("moc,bom->bcm", np.conj(R), dmixed).reshape((B, W) + (2 * modes,) * 3)
        dh = dh + _idft_trunc(ds, n, modes).real
    g["P"] = np.einsum("boxyz,bcxyz->oc", dh, cache["x"])
    g["p"] = dh.sum(axis=(0, 2, 3, 4))
    dx = np.einsum("oc,bo...->bc...", p["P"], dh)
    flat = np.concatenate([g[name].ravel() for name, _ in param_shapes(W, c_in, c_out, modes, layers)])
    return flat, dx


def mse(y, t):
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


def shell_average(field: np.ndarray, n: int, nbins: int = None):
    """Average of a mode-grid field over shells of integer |m| (FFT index order on every axis)."""
    m = np.fft.fftfreq(n, d=1.0 / n)
    r = np.sqrt(m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2)
    idx = np.rint(r).astype(int)
    nb = nbins or idx.max() + 1
    s = np.bincount(idx.ravel(), weights=field.ravel(), minlength=nb)[:nb]
    c = np.bincount(idx.ravel(), minlength=nb)[:nb]
    return s / np.maximum(c, 1)
