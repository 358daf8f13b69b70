"""CPU pins of the index algebra of the packed single-precision Coulomb kernel (the table form of
Theta^T, Sec. 4.1: twofold zero padding), written with numpy FFTs and independent of the oracle and
of the CUDA sources.  The steps are emulated with the kernel's own data layouts:

  * k3: the real line twisted by e^{-i pi n/(2N)} and transformed (negacyclic embedding: the kept
    frequencies are nu3 = 2j + 1/2), two neighbouring lines (k2 = 2m, 2m + 1) packed into one
    spectrum quad (Re z_2m, Re z_2m+1, Im z_2m, Im z_2m+1);
  * k2 and k1: a zero-padded length-2N transform held as the pair (E, O) = (x, x e^{-i pi n/N}),
    whose N-point FFTs are the even and odd output frequencies, stored in the slab buffer as
    quads (Re E, Re O, Im E, Im O) with the halves swapped for quad indices with bit 3 set; the
    cropped inverse y_n = IFFT(E)_n + e^{+i pi n/N} IFFT(O)_n;
  * the symbol sigma (spectrum i sigma, tabulated as quads over xi1) multiplied as a real factor,
    the factor i applied at the end: Re[e^{i phi} i y] = -(sin phi Re y + cos phi Im y);

and checked against the direct linear convolution Theta_p = sum_q S_{p-q} u_q of a random real odd
kernel S on (-N, N)^3 with random real u on [0, N)^3."""
import numpy as np
import pytest


def _fft(x):
    return np.fft.fft(x)


def _ifft(x):
    return np.fft.ifft(x) * len(x)   # unnormalised inverse, as the register FFT


def _sigma_table(S, N):
    """sigma = (2/(2N)^3) Im S-hat on (xi1, xi2, j) with xi1, xi2 in [0, 2N) (circular, length 2N)
    and nu3 = 2j + 1/2 (negacyclic), as the quads [j][q][c][e] (xi1 = 4q + e, xi2 = c)."""
    L = 2 * N
    m = np.arange(-N + 1, N)
    xi = np.arange(L)
    nu = 2 * np.arange(N) + 0.5
    E1 = np.exp(-2j * np.pi * np.outer(xi, m) / L)          # [xi1][m1]
    E3 = np.exp(-2j * np.pi * np.outer(nu, m) / L)          # [j][m3]
    Sh = np.einsum("am,bn,jp,mnp->jab", E1, E1, E3, S)      # [j][xi1][xi2]
    assert np.max(np.abs(Sh.real)) <= 1e-9 * np.max(np.abs(Sh))   # odd real S: imaginary
    sig = 2.0 / L ** 3 * Sh.imag
    return sig.reshape(N, L // 4, 4, L).transpose(0, 1, 3, 2).copy()   # [j][q][c][e]


def _v_store(row, jj, E, O):
    q = np.array([E.real, O.real, E.imag, O.imag])
    row[4 * jj:4 * jj + 4] = np.roll(q, 2) if jj & 8 else q


def _v_load(row, jj):
    q = row[4 * jj:4 * jj + 4]
    if jj & 8:
        q = np.roll(q, 2)
    return q[0] + 1j * q[2], q[1] + 1j * q[3]


def _theta_packed(u, S, N, swizzle=True):
    """One application of Theta^T through the packed kernel's steps."""
    L = 2 * N
    n = np.arange(N)
    tw = np.exp(-1j * np.pi * n / N)          # the O twist
    tq = np.exp(-1j * np.pi * n / (2 * N))    # the k3 (negacyclic) twist
    sig = _sigma_table(S, N)
    G = np.zeros((N, N, N // 2, 4))           # [j][k1][m] quads
    for k1 in range(N):
        for m in range(N // 2):
            za = _fft(u[k1, 2 * m] * tq)
            zb = _fft(u[k1, 2 * m + 1] * tq)
            G[:, k1, m] = np.stack([za.real, zb.real, za.imag, zb.imag], axis=1)
    RS = 4 * N + 4
    for j in range(N):
        V = np.zeros((N, RS))
        for r in range(N):                    # B1: rows along k2
            x = np.empty(N, complex)
            x[0::2] = G[j, r, :, 0] + 1j * G[j, r, :, 2]
            x[1::2] = G[j, r, :, 1] + 1j * G[j, r, :, 3]
            E, O = _fft(x), _fft(x * tw)
            for jj in range(N):
                _v_store(V[r], jj, E[jj], O[jj])
        for c in range(L):                    # B2: columns along k1
            jc, h = c >> 1, c & 1
            ore = 4 * jc + (2 if (jc & 8) and swizzle else 0) + h
            oim = ore ^ 2
            x = V[:, ore] + 1j * V[:, oim]
            E, O = _fft(x), _fft(x * tw)
            s_even = sig[j, :, c, :].reshape(-1)[0::2]   # xi1 = 2i
            s_odd = sig[j, :, c, :].reshape(-1)[1::2]    # xi1 = 2i + 1
            y = _ifft(E * s_even) + np.conj(tw) * _ifft(O * s_odd)
            V[:, ore], V[:, oim] = y.real, y.imag
        for r in range(N):                    # B3: rows back along k2
            pairs = [_v_load(V[r], jj) for jj in range(N)]
            E = np.array([p[0] for p in pairs])
            O = np.array([p[1] for p in pairs])
            y = _ifft(E) + np.conj(tw) * _ifft(O)
            G[j, r, :, 0], G[j, r, :, 1] = y[0::2].real, y[1::2].real
            G[j, r, :, 2], G[j, r, :, 3] = y[0::2].imag, y[1::2].imag
    th = np.zeros((N, N, N))
    phi = np.pi * n / (2 * N)
    for k1 in range(N):                       # k3 inverse, the deferred factor i, real part
        for m in range(N // 2):
            ya = _ifft(G[:, k1, m, 0] + 1j * G[:, k1, m, 2])
            yb = _ifft(G[:, k1, m, 1] + 1j * G[:, k1, m, 3])
            th[k1, 2 * m] = -(np.sin(phi) * ya.real + np.cos(phi) * ya.imag)
            th[k1, 2 * m + 1] = -(np.sin(phi) * yb.real + np.cos(phi) * yb.imag)
    return th


def _direct(u, S, N):
    """Theta_p = sum_q S_{p-q} u_q (S indexed by m + N - 1)."""
    out = np.zeros((N, N, N))
    for q1 in range(N):
        for q2 in range(N):
            for q3 in range(N):
                out += u[q1, q2, q3] * S[N - 1 - q1:2 * N - 1 - q1, N - 1 - q2:2 * N - 1 - q2,
                                         N - 1 - q3:2 * N - 1 - q3]
    return out


def _case(N, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((2 * N - 1,) * 3)
    S = A - A[::-1, ::-1, ::-1]               # real and odd: S_{-m} = -S_m
    u = rng.standard_normal((N,) * 3)
    return u, S


@pytest.mark.parametrize("N", [8, 16])
def test_packed_steps_equal_the_direct_linear_convolution(N):
    u, S = _case(N, 100 + N)
    ref = _direct(u, S, N)
    got = _theta_packed(u, S, N)
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_swizzle_mismatch_is_caught():
    """The planted mistake: the column pass reading the slab buffer without the half swap of the
    quads with bit 3 set (which the row passes apply) gives a wrong result."""
    N = 16
    u, S = _case(N, 7)
    ref = _direct(u, S, N)
    got = _theta_packed(u, S, N, swizzle=False)
    assert np.max(np.abs(got - ref)) > 1e-3 * np.max(np.abs(ref))
