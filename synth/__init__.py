"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 5).

This module is shared by the tests, the oracle-timing leg of ``bench.py`` and the GPU parity
tests.  It only builds initial Wigner functions and request parameters; it holds none of the
arithmetic of the time step itself (no spline, no FFT convolution, no Strang composition).

Contents
  * ``gaussian_packets``: sums of separable Gaussians w exp(-ax|x-x0|^2 - ak|k-k0|^2), the
    wavepackets of Sec. 5.1-5.4 (for example pi^-3 exp(-(x1-1)^2/2 - ... - 2|k|^2)).
  * ``wigner_1s``: the hydrogen 1s Wigner function by the discrete Fourier sum of Sec. 5.2 with
    phi_1s = exp(-|x|) / (2 sqrt(2) pi^2) and dy = 2 pi / (N_k dk).
  * ``SplitMix64``: the published SplitMix64 generator (Steele, Lea, Flood 2014; constants as in
    Vigna's public-domain reference), for seeded request streams and mixtures.
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64: state += 0x9E3779B97F4A7C15; z = mix(state)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        """The next 64-bit output."""
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        """53-bit double in [lo, hi)."""
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def randint(self, lo: int, hi: int) -> int:
        """Integer in [lo, hi] (inclusive), by rejection-free multiply-shift on 53 bits."""
        return lo + int(self.uniform() * (hi - lo + 1))


def axes(nx, nk, x_lo, x_hi, lk):
    """The x-node arrays per dimension (ends included) and the k-nodes (j - N_k/2) dk."""
    xs = [x_lo[d] + np.arange(nx[d]) * ((x_hi[d] - x_lo[d]) / (nx[d] - 1)) for d in range(3)]
    ks = (np.arange(nk) - nk / 2) * (2.0 * lk / nk)
    return xs, ks


def gaussian_packets(nx, nk, x_lo, x_hi, lk, packets, dtype=np.float64) -> np.ndarray:
    """f(x,k) = sum_p w_p exp(-ax_p |x - x0_p|^2 - ak_p |k - k0_p|^2), array [x1,x2,x3,k1,k2,k3].

    packets: iterable of dicts with keys w, x0 (3), k0 (3), ax, ak."""
    xs, ks = axes(nx, nk, x_lo, x_hi, lk)
    f = np.zeros(tuple(nx) + (nk,) * 3, dtype=np.float64)
    for p in packets:
        gx = [np.exp(-p["ax"] * (xs[d] - p["x0"][d]) ** 2) for d in range(3)]
        gk = [np.exp(-p["ak"] * (ks - p["k0"][d]) ** 2) for d in range(3)]
        X = gx[0][:, None, None] * gx[1][None, :, None] * gx[2][None, None, :]
        K = gk[0][:, None, None] * gk[1][None, :, None] * gk[2][None, None, :]
        f += p["w"] * X[:, :, :, None, None, None] * K[None, None, None]
    return f.astype(dtype)


def packet(x0, k0, ax=0.5, ak=2.0, w=None):
    """Minimum-uncertainty packet; default is the unit-mass form pi^-3 exp(-|x-x0|^2/2-2|k-k0|^2)
    of Sec. 5.3-5.4.  The unit-mass weight for general (ax, ak) is (ax ak)^{3/2} / pi^3."""
    if w is None:
        w = (ax * ak) ** 1.5 / math.pi ** 3
    return {"w": w, "x0": tuple(map(float, x0)), "k0": tuple(map(float, k0)),
            "ax": float(ax), "ak": float(ak)}


def two_packet_mixture(seed: int, center_box=3.0, k_box=1.0):
    """Statistical mixture of two unit-mass packets with seeded centres in [-3,3]^3 and momenta in
    [-1,1]^3 (weights 1/2 each)."""
    g = SplitMix64(seed)
    out = []
    for _ in range(2):
        x0 = [g.uniform(-center_box, center_box) for _ in range(3)]
        k0 = [g.uniform(-k_box, k_box) for _ in range(3)]
        p = packet(x0, k0)
        p["w"] *= 0.5
        out.append(p)
    return out


def phi_1s(r: np.ndarray) -> np.ndarray:
    """phi_1s = exp(-|x|) / (2 sqrt(2) pi^2) (Sec. 5.2)."""
    return np.exp(-r) / (2.0 * math.sqrt(2.0) * math.pi ** 2)


def wigner_1s(nx, nk, x_lo, x_hi, lk, n_y: int = 64, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Hydrogen 1s Wigner function by the discrete Fourier sum of Sec. 5.2:

      f(x, k_zeta) = sum_{eta in [-Ny/2, Ny/2)^3} phi(x - eta dy/2) phi(x + eta dy/2)
                     e^{-i zeta.eta dk dy} dy^3,     dy = 2 pi / (N_k dk),  k_zeta = zeta dk.

    Because dk dy = 2 pi / N_k the phase is periodic in eta with period N_k, so the sum is a fold
    of the N_y^3 samples into N_k^3 bins followed by an N_k^3 DFT (real, since the summand is
    even in eta).  Requires N_y to be a multiple of N_k."""
    assert n_y % nk == 0 and (n_y // 2) % nk == 0
    xs, ks = axes(nx, nk, x_lo, x_hi, lk)
    dk = 2.0 * lk / nk
    dy = 2.0 * math.pi / (nk * dk)
    eta = np.arange(-n_y // 2, n_y // 2) * dy
    f = np.zeros(tuple(nx) + (nk,) * 3)
    zeta = np.round(ks / dk).astype(np.int64)        # zeta = j - N_k/2
    rep = n_y // nk
    for i1, x1 in enumerate(xs[0]):
        for i2, x2 in enumerate(xs[1]):
            for i3, x3 in enumerate(xs[2]):
                a1 = x1 - center[0]
                a2 = x2 - center[1]
                a3 = x3 - center[2]
                # |x - y/2| and |x + y/2| on the separable sample grid
                m1 = (a1 - eta / 2) ** 2
                p1 = (a1 + eta / 2) ** 2
                m2 = (a2 - eta / 2) ** 2
                p2 = (a2 + eta / 2) ** 2
                m3 = (a3 - eta / 2) ** 2
                p3 = (a3 + eta / 2) ** 2
                rm = np.sqrt(m1[:, None, None] + m2[None, :, None] + m3[None, None, :])
                rp = np.sqrt(p1[:, None, None] + p2[None, :, None] + p3[None, None, :])
                rho = phi_1s(rm) * phi_1s(rp)
                # fold eta -> eta mod N_k; eta index i corresponds to eta = i - Ny/2 == i (mod N_k)
                P = rho.reshape(rep, nk, rep, nk, rep, nk).sum(axis=(0, 2, 4))
                F = np.fft.fftn(P)                    # sum_r P_r e^{-2 pi i zeta.r / N_k}
                f[i1, i2, i3] = np.real(F[np.ix_(zeta % nk, zeta % nk, zeta % nk)]) * dy ** 3
    return f
