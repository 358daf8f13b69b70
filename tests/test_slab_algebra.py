"""CPU pins of the index algebra that the slab phase of the table-form Coulomb kernel relies on
(Sec. 4.1: twofold zero padding): a padded length-2N transform split by frequency parity into two
N-point transforms, the i sigma product between forward and inverse passes, and the split-half
combine, in which a (-1)^j modulation of the parity-1 inverse input shifts that lane's output by
N/2 so each lane of a pair keeps a contiguous half.  Written with numpy FFTs, independent of the
oracle and of the CUDA sources; checked against the direct 2-D padded convolution."""
import numpy as np
import pytest


def _twist(n, N, conj):
    return np.exp((1 if conj else -1) * 1j * np.pi * n / N)


def _ifft(x):
    return np.fft.ifft(x) * len(x)   # unnormalised inverse, as the register FFT


def _direct(G, sig):
    """Crop of IFFT2_{2N}(i S . FFT2_{2N}(pad G)), S the parity-major symbol mapped back."""
    N = G.shape[0]
    P = np.zeros((2 * N, 2 * N), complex)
    P[:N, :N] = G
    x = np.arange(2 * N)
    S = sig[(x[:, None] & 1) * N + x[:, None] // 2, (x[None, :] & 1) * N + x[None, :] // 2]
    return (np.fft.ifft2(1j * S * np.fft.fft2(P)) * (2 * N) ** 2)[:N, :N]


def _slab(G, sig, split):
    """The lane-level steps: B1 rows along k2 (both parities), B2 columns along k1 with the symbol
    (interleaved or split-half combine), B3 rows back."""
    N = G.shape[0]
    n = np.arange(N)
    s = sig.copy()
    if split:   # the table's sign pattern: (-1)^j on the parity-1 runs
        s[N:, :] *= ((-1.0) ** n)[:, None]
    V = np.zeros((N, 2, N), complex)
    for r in range(N):
        for h in range(2):
            V[r, h] = np.fft.fft(G[r] * (_twist(n, N, False) if h else 1))
    half = N // 2
    for rho in range(2):
        for c in range(N):
            regs = []
            for h in range(2):
                X = np.fft.fft(V[:, rho, c] * (_twist(n, N, False) if h else 1))
                y = _ifft(1j * s[h * N:(h + 1) * N, rho * N + c] * X)
                if h:   # conjugate twist; with split, register n holds index (n + N/2) mod N
                    y = y * _twist((n + half) % N if split else n, N, True)
                regs.append(y)
            if split:
                k = np.arange(half)
                for h in range(2):
                    V[k + h * half, rho, c] = regs[h][k] + regs[1 - h][k + half]
            else:
                V[:, rho, c] = regs[0] + regs[1]
    out = np.zeros_like(G)
    for r in range(N):
        out[r] = sum(_ifft(V[r, h]) * (_twist(n, N, True) if h else 1) for h in range(2))
    return out


@pytest.mark.parametrize("N", [8, 16, 32])
@pytest.mark.parametrize("split", [False, True])
def test_slab_steps_equal_the_direct_padded_convolution(N, split):
    rng = np.random.default_rng(N + 100 * split)
    G = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    sig = rng.standard_normal((2 * N, 2 * N))
    ref = _direct(G, sig)
    got = _slab(G, sig, split)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_split_without_the_sign_pattern_is_wrong():
    """The planted mistake: the split combine on a table without (-1)^j gives a wrong slab."""
    N = 8
    rng = np.random.default_rng(3)
    G = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    sig = rng.standard_normal((2 * N, 2 * N))
    ref = _direct(G, sig)
    n = np.arange(N)
    # _slab's split path applies (-1)^j itself; a symbol already carrying it cancels that, so the
    # split combine runs on a table without the sign pattern
    cancelled = sig.copy()
    cancelled[N:, :] *= ((-1.0) ** n)[:, None]
    got = _slab(G, cancelled, True)
    assert np.max(np.abs(got - ref)) > 1e-3 * np.max(np.abs(ref))
