"""FP64 CPU oracle for one Strang step of the CHASM scheme (Xiong, Zhang, Shao, arXiv 2205.02380).

TEST INFRASTRUCTURE ONLY.  This module is imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The product path (the
CUDA library and its Python binding) never imports, links or executes anything here, and this
module imports nothing from the product path.

Everything is plain numpy/scipy in float64.  Library primitives used as single steps: ``numpy.fft``
(the FFTs the paper itself prescribes), ``numpy.linalg.inv/solve`` (the dense inverse of the spline
matrix and the LU solve of step (5) of the PMBC procedure), ``scipy.special.sici`` (the sine
integral Si of Eq. 4.3).  No blocking, fusion or reordering beyond what the cited equations state.

Layout: a Wigner function is an array f[x1, x2, x3, k1, k2, k3] (x first, k last).

Grid readings (stated once, used everywhere):
  * x-grid: N_x points per dimension including both ends, x_j = lo + j h, h = (hi-lo)/(N_x-1);
    the paper's "N+1 grid points" with N = N_x - 1 (Sec. 2.2).
  * k-grid: k_j = (j - N_k/2) dk, dk = 2 L_k / N_k, j = 0..N_k-1 (Sec. 5.2, k_zeta = zeta dk).
  * Strang step S(dt) = A(dt/2) P(dt) A(dt/2); P for the Coulomb case is the 4-term Taylor
    (Horner) approximation of exp(dt Theta^T); for a quadratic potential P is the exact k-shift.
  * LPC1 step (the paper's one-stage Lawson predictor-corrector): one advection of f and of
    Theta[f] by the full dt and two applications of Theta (lpc1_step).
  * Sign of the Coulomb operator follows Eq. 2.3 (its classical limit is +(1/hbar) grad V . grad_k f,
    as in Eq. 5.1): Theta = -(2 Z / (pi^2 hbar)) Im[e^{2 i xt.k} Phi], Phi = T * (f e^{-2 i xt.k}).

Parity pins: every public function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` against closed forms, library routines, invariants or brute force.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.special import sici

# --------------------------------------------------------------------------------------------
# Grids
# --------------------------------------------------------------------------------------------


def x_nodes(n: int, lo: float, hi: float) -> np.ndarray:
    """x_j = lo + j h, j = 0..n-1, both ends included (Sec. 2.2: N+1 points, N = n-1)."""
    if n == 1:
        return np.array([float(lo)])
    return lo + np.arange(n, dtype=np.float64) * ((hi - lo) / (n - 1))


def k_nodes(nk: int, lk: float) -> np.ndarray:
    """k_j = (j - N_k/2) dk with dk = 2 L_k / N_k (Sec. 5.2: k_zeta = zeta dk)."""
    dk = 2.0 * lk / nk
    return (np.arange(nk, dtype=np.float64) - nk / 2) * dk


@dataclass
class Problem:
    """A 6-D uniform grid, a potential and the physical constants hbar, m.

    nuclei: list of (position[3], charge Z) for V = -sum Z/|x - x_A| (Sec. 2.1);
    if empty, the harmonic potential V = kappa/2 |x - c|^2 (Sec. 5.1) is used.
    """
    nx: tuple
    nk: int
    x_lo: tuple
    x_hi: tuple
    lk: float
    hbar: float = 1.0
    m: float = 1.0
    nuclei: list = field(default_factory=list)
    kappa: float = 0.0
    center: tuple = (0.0, 0.0, 0.0)
    n_nb: int = 20

    def xs(self, d: int) -> np.ndarray:
        """x-nodes of dimension d, ends included (Sec. 3: N + 1 points)."""
        return x_nodes(self.nx[d], self.x_lo[d], self.x_hi[d])

    def hs(self, d: int) -> float:
        """x-spacing of dimension d."""
        return (self.x_hi[d] - self.x_lo[d]) / (self.nx[d] - 1)

    def ks(self) -> np.ndarray:
        """k-nodes (j - N_k/2) dk, the same in every dimension (Sec. 4.1, k_zeta = zeta dk)."""
        return k_nodes(self.nk, self.lk)

    @property
    def dk(self) -> float:
        """k-spacing 2 L_k / N_k."""
        return 2.0 * self.lk / self.nk

    @property
    def shape(self) -> tuple:
        """Shape of f: (nx1, nx2, nx3, N_k, N_k, N_k), k3 fastest."""
        return tuple(self.nx) + (self.nk,) * 3

    def potential(self) -> np.ndarray:
        """V(x) on the x-grid, shape (nx1, nx2, nx3)."""
        X = np.meshgrid(self.xs(0), self.xs(1), self.xs(2), indexing="ij")
        if self.nuclei:
            V = np.zeros(tuple(self.nx))
            for pos, Z in self.nuclei:
                r = np.sqrt(sum((X[d] - pos[d]) ** 2 for d in range(3)))
                V -= Z / r
            return V
        return 0.5 * self.kappa * sum((X[d] - self.center[d]) ** 2 for d in range(3))


# --------------------------------------------------------------------------------------------
# Cubic B-splines and the PMBC-closed spline transform (Sec. 2.2, Sec. 3.1)
# --------------------------------------------------------------------------------------------


def bspline(t: np.ndarray) -> np.ndarray:
    """B_nu(x) as a function of t = (x - x_nu)/h, piecewise as written in Eq. 2.9.

    Pieces: [x_{nu-2}, x_{nu-1}], [x_{nu-1}, x_nu], [x_nu, x_{nu+1}], [x_{nu+1}, x_{nu+2}]."""
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros_like(t)
    p1 = (t >= -2) & (t < -1)
    p2 = (t >= -1) & (t < 0)
    p3 = (t >= 0) & (t < 1)
    p4 = (t >= 1) & (t <= 2)
    u = t + 2.0  # (x - x_{nu-2})/h
    out[p1] = u[p1] ** 3 / 6.0
    u = t + 1.0  # (x - x_{nu-1})/h
    out[p2] = -u[p2] ** 3 / 2.0 + u[p2] ** 2 / 2.0 + u[p2] / 2.0 + 1.0 / 6.0
    u = 1.0 - t  # (x_{nu+1} - x)/h
    out[p3] = -u[p3] ** 3 / 2.0 + u[p3] ** 2 / 2.0 + u[p3] / 2.0 + 1.0 / 6.0
    u = 2.0 - t  # (x_{nu+2} - x)/h
    out[p4] = u[p4] ** 3 / 6.0
    return out


def natural_matrix(n: int, h: float) -> np.ndarray:
    """A-tilde: the (N+3)x(N+3) spline matrix with natural end rows (Eqs. 2.11, 2.13, 2.14).

    Unknowns eta_{-1..N+1} at array index nu+1; rows: natural(left), three-term rows i=0..N,
    natural(right)."""
    N = n - 1
    A = np.zeros((N + 3, N + 3))
    A[0, 0:3] = np.array([1.0, -2.0, 1.0]) / h**2
    for i in range(N + 1):
        A[i + 1, i:i + 3] = [1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0]
    A[N + 2, N:N + 3] = np.array([1.0, -2.0, 1.0]) / h**2
    return A


def hermite_matrix(n: int, h: float) -> np.ndarray:
    """A: the (N+3)x(N+3) spline matrix with Hermite end rows s'(x_0)=phi_L, s'(x_N)=phi_R
    (Eqs. 2.11, 2.12, 2.14)."""
    N = n - 1
    A = np.zeros((N + 3, N + 3))
    A[0, 0] = -1.0 / (2 * h)
    A[0, 2] = 1.0 / (2 * h)
    for i in range(N + 1):
        A[i + 1, i:i + 3] = [1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0]
    A[N + 2, N] = -1.0 / (2 * h)
    A[N + 2, N + 2] = 1.0 / (2 * h)
    return A


def pmbc_end_stencils(n: int, h: float, n_nb: int):
    """PMBC closure of the global natural spline on a single patch (Eq. 3.5).

    Returns (c_plus, c_minus), each of length J = min(n_nb, N)+1:
      phi_L = sum_j c_plus[j]  * phi(x_j),       c+_{j,0} = (-bt_{-1,j}  + bt_{1,j}) / 2h
      phi_R = sum_j c_minus[j] * phi(x_{N-j}),   c-_{j,p} = (-bt_{N-1,N-j} + bt_{N+1,N-j}) / 2h
    with bt = inverse of the natural matrix (dense FP64 inverse).  Stencil taps that would fall
    outside [0, N] are dropped."""
    N = n - 1
    bt = np.linalg.inv(natural_matrix(n, h))
    J = min(n_nb, N) + 1
    j = np.arange(J)
    # row index of eta_i is i+1; column index of phi_j is j+1
    c_plus = (-bt[0, j + 1] + bt[2, j + 1]) / (2 * h)
    c_minus = (-bt[N, N - j + 1] + bt[N + 2, N - j + 1]) / (2 * h)
    return c_plus, c_minus


def spline_coeffs_1d(phi: np.ndarray, axis: int, h: float, n_nb: int) -> np.ndarray:
    """eta along one axis: PMBC closure (Eq. 3.5) then the Hermite-closed solve A eta = rhs
    (step (5) of Sec. 3.1.2).  Output has N+3 entries (eta_{-1..N+1}) along ``axis``."""
    phi = np.moveaxis(np.asarray(phi, dtype=np.float64), axis, 0)
    n = phi.shape[0]
    N = n - 1
    cp, cm = pmbc_end_stencils(n, h, n_nb)
    J = cp.shape[0]
    flat = phi.reshape(n, -1)
    phi_L = np.tensordot(cp, flat[0:J], axes=(0, 0))
    phi_R = np.tensordot(cm, flat[N - np.arange(J)], axes=(0, 0))
    rhs = np.vstack([phi_L[None], flat, phi_R[None]])
    eta = np.linalg.solve(hermite_matrix(n, h), rhs)
    eta = eta.reshape((N + 3,) + phi.shape[1:])
    return np.moveaxis(eta, 0, axis)


def pmbc_patch_closures(phi: np.ndarray, h: float, n_nb: int, p: int) -> np.ndarray:
    """The closure values of p patches along axis 0 of phi (n = N+1 nodes, N = p M), steps (1)-(4)
    of Sec. 3.1.2: entry b = 0 is phi_L of the first patch and b = p phi_R of the last (Eq. 3.5,
    global natural ends), entry b = 1..p-1 is phi_R^{(b)} = phi_L^{(b+1)} at the shared node
    s = b M, c_{0,b} phi(x_s) + sum_{j=1}^{n_nb} (c-_{j,b} phi(x_{s-j}) + c+_{j,b} phi(x_{s+j}))
    (Eq. 3.4 with the coefficients of the inverse natural matrix, reading A7), taps outside [0, N]
    dropped.  Shape (p+1,) + phi.shape[1:]."""
    n = phi.shape[0]
    N = n - 1
    M = N // p
    bt = np.linalg.inv(natural_matrix(n, h))
    cp, cm = pmbc_end_stencils(n, h, n_nb)
    J = cp.shape[0]
    out = np.zeros((p + 1,) + phi.shape[1:])
    out[0] = np.tensordot(cp, phi[0:J], axes=(0, 0))
    out[p] = np.tensordot(cm, phi[N - np.arange(J)], axes=(0, 0))
    for b in range(1, p):
        sn = b * M
        # rows of eta_{s-1}, eta_{s+1} are s, s+2; the column of phi_j is j+1
        def c(j):
            return (-bt[sn, j + 1] + bt[sn + 2, j + 1]) / (2 * h)
        acc = c(sn) * phi[sn]
        for j in range(1, n_nb + 1):
            if sn - j >= 0:
                acc = acc + c(sn - j) * phi[sn - j]
            if sn + j <= N:
                acc = acc + c(sn + j) * phi[sn + j]
        out[b] = acc
    return out


def advect_1d_patches(phi: np.ndarray, axis: int, h: float, n_nb: int, alpha: np.ndarray,
                      k_axis: int, p: int) -> np.ndarray:
    """A along one axis with p patches (Sec. 3.1.2): closures from pmbc_patch_closures, each patch
    solves its own Hermite-closed system of M+3 unknowns (step (5)), and the value at node j is
    the local spline of the patch that contains the foot x_j - alpha h (interpolation and
    correction of Sec. 3.1.3: at an exact shared node the left patch, feet beyond the ends use
    the end patches, reading A10); local coefficients outside [-1, M+1] are zero."""
    phi = np.moveaxis(np.asarray(phi, dtype=np.float64), (axis, k_axis), (0, 1))
    n = phi.shape[0]
    N = n - 1
    M = N // p
    cl = pmbc_patch_closures(phi, h, n_nb, p)
    A = hermite_matrix(M + 1, h)
    etas = []
    for l in range(p):
        rhs = np.concatenate([cl[l][None], phi[l * M:(l + 1) * M + 1], cl[l + 1][None]])
        etas.append(np.linalg.solve(A, rhs.reshape(M + 3, -1)).reshape((M + 3,) + phi.shape[1:]))
    out = np.zeros_like(phi)
    for kk, a in enumerate(np.asarray(alpha, dtype=np.float64)):
        for j in range(n):
            t = j - a                                   # foot in units of h from x_0
            l = min(max(int(math.ceil(t / M)) - 1, 0), p - 1)
            tl = t - l * M
            base = math.floor(tl)
            for nu in range(int(base) - 1, int(base) + 3):
                if -1 <= nu <= M + 1:
                    out[j, kk] += etas[l][nu + 1, kk] * bspline(np.array(tl - nu))
    return np.moveaxis(out, (0, 1), (axis, k_axis))


def advect_patches(f: np.ndarray, prob: Problem, tau: float, p: tuple) -> np.ndarray:
    """A(tau) with p[d] patches per x-dimension: the 1-D patch transform along x1, x2, x3 in turn
    (the sum-factorised form of Eq. 3.10; the oracle checks this identity at p = 1 against the
    64-term sum)."""
    g = np.asarray(f, dtype=np.float64)
    ks = prob.ks()
    for d in range(3):
        alpha = prob.hbar * ks * tau / (prob.m * prob.hs(d))
        out = np.empty_like(g)
        for kd in range(prob.nk):
            sl = [slice(None)] * 6
            sl[3 + d] = slice(kd, kd + 1)
            sub = g[tuple(sl)]
            out[tuple(sl)] = advect_1d_patches(sub, d, prob.hs(d), prob.n_nb, alpha[kd:kd + 1],
                                               3 + d, p[d])
        g = out
    return g


def spline_coeffs_3d(f: np.ndarray, prob: Problem) -> np.ndarray:
    """Tensor-product coefficients eta_{nu1 nu2 nu3}(k) by 1-D solves along x1, x2, x3 in turn
    (Eq. 3.9).  Shape (nx1+2, nx2+2, nx3+2, Nk, Nk, Nk)."""
    eta = f
    for d in range(3):
        eta = spline_coeffs_1d(eta, d, prob.hs(d), prob.n_nb)
    return eta


def _feet_taps(n: int, h: float, alpha: np.ndarray):
    """For nodes j=0..n-1 and shifts alpha[k] (in units of h), the four B-splines that are
    nonzero at the foot y = x_j - alpha h: indices nu and values B_nu(y) from Eq. 2.9.

    Returns (nu[j, k, 4], w[j, k, 4])."""
    j = np.arange(n, dtype=np.float64)[:, None]
    s = j - alpha[None, :]                 # foot position in units of h, relative to x_0
    base = np.floor(s)
    nus = base[..., None] + np.array([-1.0, 0.0, 1.0, 2.0])
    w = bspline(s[..., None] - nus)
    return nus.astype(np.int64), w


def advect(f: np.ndarray, prob: Problem, tau: float, kaxes=None) -> np.ndarray:
    """A(tau): f(x - hbar k tau / m, k) by the tensor-product cubic spline (Eqs. 2.6, 3.10).

    eta from spline_coeffs_3d; then, per output point, the literal 4x4x4 = 64-term sum
    sum_{nu1,nu2,nu3} eta * prod_d B_{nu_d}(x_{j_d} - alpha_d h_d), alpha_d = hbar k_d tau/(m h_d).
    Coefficients with nu outside [-1, N+1] are zero (ghost splines).

    kaxes: optional (k1 values, k2 values, k3 values) of the last three axes of f, for inputs
    that hold a subset of the k-grid (each k is independent in A); default the full k-grid."""
    eta = spline_coeffs_3d(f, prob)
    if kaxes is None:
        kaxes = (prob.ks(),) * 3
    kn = [len(kaxes[d]) for d in range(3)]
    taps = []
    pad = 0
    for d in range(3):
        alpha = prob.hbar * np.asarray(kaxes[d], dtype=np.float64) * tau / (prob.m * prob.hs(d))
        nu, w = _feet_taps(prob.nx[d], prob.hs(d), alpha)
        taps.append((nu, w))
        pad = max(pad, int(np.max(np.abs(nu))) + 2)
    # zero-pad eta so every nu in range maps to a zero ghost; array index of nu is nu + 1 + pad
    eta_p = np.pad(eta, [(pad, pad)] * 3 + [(0, 0)] * 3)
    n1, n2, n3 = prob.nx
    m1, m2, m3 = kn
    K1 = np.arange(m1).reshape(1, 1, 1, m1, 1, 1)
    K2 = np.arange(m2).reshape(1, 1, 1, 1, m2, 1)
    K3 = np.arange(m3).reshape(1, 1, 1, 1, 1, m3)
    out = np.zeros(tuple(prob.nx) + tuple(kn))
    (nu1, w1), (nu2, w2), (nu3, w3) = taps
    for a in range(4):
        I1 = (nu1[:, :, a] + 1 + pad).reshape(n1, 1, 1, m1, 1, 1)
        W1 = w1[:, :, a].reshape(n1, 1, 1, m1, 1, 1)
        for b in range(4):
            I2 = (nu2[:, :, b] + 1 + pad).reshape(1, n2, 1, 1, m2, 1)
            W2 = w2[:, :, b].reshape(1, n2, 1, 1, m2, 1)
            for c in range(4):
                I3 = (nu3[:, :, c] + 1 + pad).reshape(1, 1, n3, 1, 1, m3)
                W3 = w3[:, :, c].reshape(1, 1, n3, 1, 1, m3)
                out += W1 * W2 * W3 * eta_p[I1, I2, I3, K1, K2, K3]
    return out


def advect_1d(phi: np.ndarray, axis: int, h: float, n_nb: int, alpha: np.ndarray,
              k_axis: int) -> np.ndarray:
    """1-D version of A: spline along ``axis`` and evaluation at x_j - alpha h, where alpha is
    indexed by the array axis ``k_axis``.  Used by the tests to check the 64-term sum against
    three successive 1-D passes."""
    eta = spline_coeffs_1d(phi, axis, h, n_nb)
    n = phi.shape[axis]
    nu, w = _feet_taps(n, h, alpha)
    pad = int(np.max(np.abs(nu))) + 2
    eta = np.moveaxis(eta, (axis, k_axis), (0, 1))
    eta = np.pad(eta, [(pad, pad)] + [(0, 0)] * (eta.ndim - 1))
    out = np.zeros((n,) + eta.shape[1:])
    kk = np.arange(len(alpha))
    for c in range(4):
        idx = nu[:, :, c] + 1 + pad           # (n, nk)
        g = eta[idx, kk[None, :]]             # (n, nk, ...)
        out += w[:, :, c].reshape(w.shape[:2] + (1,) * (eta.ndim - 2)) * g
    return np.moveaxis(out, (0, 1), (axis, k_axis))


# --------------------------------------------------------------------------------------------
# Truncated kernel method for the Coulomb operator (Sec. 4)
# --------------------------------------------------------------------------------------------


def c_n_alpha(n: int, a: float) -> float:
    """c_{n,alpha} = pi^{n/2} 2^alpha Gamma(alpha/2) / Gamma((n-alpha)/2) (Eq. 2.4)."""
    return math.pi ** (n / 2) * 2.0 ** a * math.gamma(a / 2) / math.gamma((n - a) / 2)


def si(x: np.ndarray) -> np.ndarray:
    """Sine integral Si(x) = int_0^x sin t / t dt (scipy.special.sici)."""
    return sici(np.asarray(x, dtype=np.float64))[0]


def truncated_kernel_hat(xi_abs: np.ndarray, D: float) -> np.ndarray:
    """U_D-hat(xi) = 4 pi Si(|xi| D) / |xi|, with the limit 4 pi D at xi = 0 (Eq. 4.3)."""
    xi_abs = np.asarray(xi_abs, dtype=np.float64)
    out = np.empty_like(xi_abs)
    z = xi_abs == 0.0
    out[z] = 4.0 * math.pi * D
    out[~z] = 4.0 * math.pi * si(xi_abs[~z] * D) / xi_abs[~z]
    return out


def tkm_diameter(lk: float) -> float:
    """D = diam of Omega = [-L_k, L_k]^3 = 2 sqrt(3) L_k (Eq. 4.2)."""
    return 2.0 * math.sqrt(3.0) * lk


def tkm_tensor(nk: int, lk: float) -> np.ndarray:
    """The convolution tensor T_p of Eq. 4.7 for p in [-(N_k-1), N_k-1]^3.

    T_p = (3N_k)^{-3} sum_{n in I} U_D-hat(xi_n) e^{2 pi i p.n/(3N_k)}, xi_n = 2 pi n / (6 L_k),
    I = {-3N_k/2 .. 3N_k/2 - 1}^3 (Eq. 4.8), evaluated as one backward FFT of length (3N_k)^3 as
    the paper prescribes.  Returned array has shape (2N_k-1)^3, index p + N_k - 1; real part."""
    M = 3 * nk
    n = np.arange(-M // 2, M // 2)
    xi = 2.0 * math.pi * n / (6.0 * lk)
    XI = np.sqrt(xi[:, None, None] ** 2 + xi[None, :, None] ** 2 + xi[None, None, :] ** 2)
    U = truncated_kernel_hat(XI, tkm_diameter(lk))
    # place mode n at FFT slot n mod M; numpy.fft.ifftn carries the (3N_k)^{-3} factor
    U = np.fft.ifftshift(U)
    Tfull = np.fft.ifftn(U)
    p = np.arange(-(nk - 1), nk)
    T = Tfull[np.ix_(p % M, p % M, p % M)]
    return T.real.copy()


def tkm_tensor_direct(nk: int, lk: float, p: tuple) -> complex:
    """Brute-force evaluation of Eq. 4.7 at one index p (tests only)."""
    M = 3 * nk
    n = np.arange(-M // 2, M // 2)
    xi = 2.0 * math.pi * n / (6.0 * lk)
    XI = np.sqrt(xi[:, None, None] ** 2 + xi[None, :, None] ** 2 + xi[None, None, :] ** 2)
    U = truncated_kernel_hat(XI, tkm_diameter(lk))
    ph = np.exp(2j * math.pi * (p[0] * n[:, None, None] + p[1] * n[None, :, None]
                                + p[2] * n[None, None, :]) / M)
    return complex(np.sum(U * ph) / M**3)


def tkm_convolve(fs: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Phi_p = sum_{q} T_{p-q} fs_q over the last three axes (Eq. 4.6), computed with twofold
    zero padding: circular convolution of length 2N_k, T placed at slots p mod 2N_k and zero at
    the unused slot N_k."""
    nk = fs.shape[-1]
    L = 2 * nk
    Tc = np.zeros((L, L, L))
    p = np.arange(-(nk - 1), nk) % L
    Tc[np.ix_(p, p, p)] = T
    That = np.fft.fftn(Tc)
    pad = np.zeros(fs.shape[:-3] + (L, L, L), dtype=np.complex128)
    pad[..., :nk, :nk, :nk] = fs
    out = np.fft.ifftn(np.fft.fftn(pad, axes=(-3, -2, -1)) * That, axes=(-3, -2, -1))
    return out[..., :nk, :nk, :nk]


def tkm_convolve_direct(fs: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Brute-force Eq. 4.6 (O(N_k^6)); tests only."""
    nk = fs.shape[-1]
    out = np.zeros(fs.shape, dtype=np.complex128)
    idx = np.arange(nk)
    for p1 in range(nk):
        for p2 in range(nk):
            for p3 in range(nk):
                Tsub = T[np.ix_(p1 - idx + nk - 1, p2 - idx + nk - 1, p3 - idx + nk - 1)]
                out[..., p1, p2, p3] = np.sum(Tsub * fs, axis=(-3, -2, -1))
    return out


def theta_coulomb_point(fk: np.ndarray, xt: np.ndarray, Z: float, hbar: float, ks: np.ndarray,
                        T: np.ndarray, direct: bool = False) -> np.ndarray:
    """Theta^T for one nucleus at spatial points with offsets xt = x - x_A.

    fk: (..., Nk, Nk, Nk) real; xt: (..., 3).  Following Eqs. 4.1, 4.5, 4.6 with the Eq. 2.3 sign:
      fs = f e^{-2 i xt.k};  Phi = T * fs;  Theta = -(2 Z/(pi^2 hbar)) Im[e^{2 i xt.k} Phi].
    (The prefactor 2/c_{3,1} = 1/pi^2.)"""
    ph = 2.0 * (xt[..., 0, None, None, None] * ks[:, None, None]
                + xt[..., 1, None, None, None] * ks[None, :, None]
                + xt[..., 2, None, None, None] * ks[None, None, :])
    fs = fk * np.exp(-1j * ph)
    Phi = tkm_convolve_direct(fs, T) if direct else tkm_convolve(fs, T)
    pref = 2.0 / c_n_alpha(3, 1)  # = 1/pi^2
    return -(2.0 * Z * pref / hbar) * np.imag(np.exp(1j * ph) * Phi)


def theta_coulomb(f: np.ndarray, prob: Problem, T: np.ndarray | None = None,
                  x_batch: int = 64, xpts: np.ndarray | None = None) -> np.ndarray:
    """Theta^T[f] on the whole grid: sum over nuclei of theta_coulomb_point (Sec. 4).

    xpts: optional (n, 3) positions of the leading axis of f (shape (n, Nk, Nk, Nk)), for
    inputs that hold a subset of the x points (Theta is local in x); default the full x-grid."""
    if T is None:
        T = tkm_tensor(prob.nk, prob.lk)
    ks = prob.ks()
    nk = prob.nk
    if xpts is None:
        X = np.stack(np.meshgrid(prob.xs(0), prob.xs(1), prob.xs(2), indexing="ij"), axis=-1)
        Xf = X.reshape(-1, 3)
    else:
        Xf = np.asarray(xpts, dtype=np.float64).reshape(-1, 3)
    fx = f.reshape(-1, nk, nk, nk)
    out = np.zeros_like(fx)
    for pos, Z in prob.nuclei:
        xt = Xf - np.asarray(pos, dtype=np.float64)
        for s in range(0, fx.shape[0], x_batch):
            out[s:s + x_batch] += theta_coulomb_point(fx[s:s + x_batch], xt[s:s + x_batch], Z,
                                                      prob.hbar, ks, T)
    return out.reshape(f.shape)


def pflow_coulomb(f: np.ndarray, prob: Problem, dt: float, T: np.ndarray | None = None,
                  xpts: np.ndarray | None = None) -> np.ndarray:
    """P(dt) for the Coulomb case: the 4-term Taylor approximation of exp(dt Theta^T) in Horner
    form, u <- f + (dt/s) Theta^T[u] for s = 4, 3, 2, 1 starting from u = f."""
    if T is None:
        T = tkm_tensor(prob.nk, prob.lk)
    u = f
    for s in (4, 3, 2, 1):
        u = f + (dt / s) * theta_coulomb(u, prob, T, xpts=xpts)
    return u


def _kshift_factors(prob: Problem, d: int, dt: float) -> np.ndarray:
    """Per (x_d index, k_d mode in FFT order) factor of the exact k-shift by
    s = dt kappa (x_d - c_d)/hbar (Eq. 5.1): e^{i xi_m s}, xi_m = pi m / L_k, m in [-N_k/2, N_k/2),
    with cos(xi s) at the Nyquist mode so the result stays real."""
    nk = prob.nk
    m = np.fft.fftfreq(nk, d=1.0 / nk)          # integer modes in FFT order, -N/2 at slot N/2
    xi = math.pi * m / prob.lk
    s = dt * prob.kappa * (prob.xs(d) - prob.center[d]) / prob.hbar   # shift per x_d
    fac = np.exp(1j * xi[None, :] * s[:, None])
    fac[:, nk // 2] = np.cos(xi[nk // 2] * s)
    return fac


def pflow_harmonic(f: np.ndarray, prob: Problem, dt: float) -> np.ndarray:
    """P(dt) for V = kappa/2 |x - c|^2: Theta = (1/hbar) grad V . grad_k f exactly (Eq. 5.1), so
    the flow is the shift f(x, k + dt kappa (x - c)/hbar).  Applied spectrally per k-axis on the
    periodic k-grid (factors from _kshift_factors)."""
    nk = prob.nk
    F = np.fft.fftn(f, axes=(3, 4, 5))
    for d in range(3):
        shape = [1] * 6
        shape[d] = prob.nx[d]
        shape[3 + d] = nk
        F = F * _kshift_factors(prob, d, dt).reshape(shape)
    return np.real(np.fft.ifftn(F, axes=(3, 4, 5)))


def strang_step_plane(g: np.ndarray, prob: Problem, d: int, dt: float, p: int = 1) -> np.ndarray:
    """One Strang step of the quadratic-potential scheme on the (x_d, k_d) plane, g[i, j] at
    (x_{d,i}, k_j).

    For V = kappa/2 |x - c|^2 both substeps act on each pair (x_d, k_d) separately: A(tau) is the
    product over d of 1-D spline interpolations along x_d with shifts set by k_d (Eqs. 3.9, 3.10)
    and P(dt) the product over d of shifts along k_d by dt kappa (x_d - c_d)/hbar (Eq. 5.1).  A
    product f = prod_d g_d(x_d, k_d) is therefore mapped factor by factor, and this function is
    the factor map (it calls the same 1-D spline and k-shift as the 6-D step).  p > 1: the x_d
    axis is split into p PMBC patches (Sec. 3.1.2-3.1.3), as advect_patches does in 6-D."""
    def a_half(gg):
        alpha = prob.hbar * prob.ks() * (0.5 * dt) / (prob.m * prob.hs(d))
        if p > 1:
            return advect_1d_patches(gg, 0, prob.hs(d), prob.n_nb, alpha, 1, p)
        return advect_1d(gg, 0, prob.hs(d), prob.n_nb, alpha, 1)
    g = a_half(g)
    g = np.real(np.fft.ifft(np.fft.fft(g, axis=1) * _kshift_factors(prob, d, dt), axis=1))
    return a_half(g)


def pflow(f: np.ndarray, prob: Problem, dt: float, T=None) -> np.ndarray:
    """P(dt): the Coulomb Taylor-4 flow when the problem has nuclei, else the exact k-shift."""
    if prob.nuclei:
        return pflow_coulomb(f, prob, dt, T)
    return pflow_harmonic(f, prob, dt)


def strang_step(f: np.ndarray, prob: Problem, dt: float, T=None) -> np.ndarray:
    """S(dt) = A(dt/2) P(dt) A(dt/2) (Sec. 2.2, Strang splitting)."""
    f = advect(f, prob, 0.5 * dt)
    f = pflow(f, prob, dt, T)
    return advect(f, prob, 0.5 * dt)


def run(f: np.ndarray, prob: Problem, dt: float, nsteps: int) -> np.ndarray:
    """nsteps Strang steps (T computed once)."""
    T = tkm_tensor(prob.nk, prob.lk) if prob.nuclei else None
    for _ in range(nsteps):
        f = strang_step(f, prob, dt, T)
    return f


# --------------------------------------------------------------------------------------------
# LPC1: the one-stage Lawson predictor-corrector (Sec. 2.2)
# --------------------------------------------------------------------------------------------


def theta_harmonic(f: np.ndarray, prob: Problem) -> np.ndarray:
    """Theta for V = kappa/2 |x - c|^2: (1/hbar) grad V . grad_k f = sum_d kappa (x_d - c_d)/hbar
    df/dk_d (Eq. 5.1).  The k-derivative is spectral on the periodic k-grid, i xi_m with
    xi_m = pi m / L_k, and 0 at the Nyquist mode: the rate at s = 0 of the shift used by
    pflow_harmonic (whose Nyquist factor cos(xi s) has zero derivative there)."""
    nk = prob.nk
    m = np.fft.fftfreq(nk, d=1.0 / nk)
    ixi = 1j * math.pi * m / prob.lk
    ixi[nk // 2] = 0.0
    out = np.zeros_like(f)
    for d in range(3):
        deriv = np.real(np.fft.ifft(np.fft.fft(f, axis=3 + d) * ixi.reshape(
            [nk if a == 3 + d else 1 for a in range(6)]), axis=3 + d))
        rate = prob.kappa * (prob.xs(d) - prob.center[d]) / prob.hbar
        out += deriv * rate.reshape([prob.nx[d] if a == d else 1 for a in range(6)])
    return out


def theta(f: np.ndarray, prob: Problem, T=None) -> np.ndarray:
    """Theta_V[f] for the problem's potential (Coulomb: Sec. 4; quadratic: Eq. 5.1)."""
    if prob.nuclei:
        return theta_coulomb(f, prob, T)
    return theta_harmonic(f, prob)


def lpc1_combine(f: np.ndarray, adv, th, dt: float) -> np.ndarray:
    """The LPC1 combination (Sec. 2.2) for the advection map adv = A(dt), g -> g(A_dt(x, k)) with
    A_dt(x, k) = (x - hbar k dt / m, k), and the operator th = Theta_V:
      predictor  f~ = f(A_dt) + dt Theta_V[f](A_dt)
      corrector  f' = f(A_dt) + dt/2 Theta_V[f~] + dt/2 Theta_V[f](A_dt)."""
    g = adv(f)
    h = adv(th(f))
    ft = g + dt * h
    return g + 0.5 * dt * th(ft) + 0.5 * dt * h


def lpc1_step(f: np.ndarray, prob: Problem, dt: float, T=None) -> np.ndarray:
    """One LPC1 step on the 6-D grid: lpc1_combine with the advection of Sec. 3 and theta."""
    if prob.nuclei and T is None:
        T = tkm_tensor(prob.nk, prob.lk)
    return lpc1_combine(f, lambda u: advect(u, prob, dt), lambda u: theta(u, prob, T), dt)


def lpc1_step_plane(g: np.ndarray, prob: Problem, d: int, dt: float) -> np.ndarray:
    """One LPC1 step of the quadratic-potential problem on the (x_d, k_d) plane, g[i, j] at
    (x_{d,i}, k_j): the 1-D spline advection along x_d (Eqs. 3.9, 3.10) and
    Theta g = kappa (x_d - c_d)/hbar dg/dk spectrally along k (Eq. 5.1), combined by
    lpc1_combine (the 1-D harmonic oscillator of Sec. 5.1 in its own phase plane)."""
    nk = prob.nk
    m = np.fft.fftfreq(nk, d=1.0 / nk)
    ixi = 1j * math.pi * m / prob.lk
    ixi[nk // 2] = 0.0
    rate = prob.kappa * (prob.xs(d) - prob.center[d]) / prob.hbar
    alpha = prob.hbar * prob.ks() * dt / (prob.m * prob.hs(d))

    def th(gg):
        return rate[:, None] * np.real(np.fft.ifft(np.fft.fft(gg, axis=1) * ixi[None, :], axis=1))

    def adv(gg):
        return advect_1d(gg, 0, prob.hs(d), prob.n_nb, alpha, 1)

    return lpc1_combine(g, adv, th, dt)


def run_lpc1(f: np.ndarray, prob: Problem, dt: float, nsteps: int) -> np.ndarray:
    """nsteps LPC1 steps (Sec. 2.2; T computed once)."""
    T = tkm_tensor(prob.nk, prob.lk) if prob.nuclei else None
    for _ in range(nsteps):
        f = lpc1_step(f, prob, dt, T)
    return f


# --------------------------------------------------------------------------------------------
# Diagnostics (Sec. 5)
# --------------------------------------------------------------------------------------------


def cell_volume(prob: Problem) -> float:
    return prob.hs(0) * prob.hs(1) * prob.hs(2) * prob.dk ** 3


def mass(f: np.ndarray, prob: Problem) -> float:
    """Total mass: the integral replaced by the grid sum times h1 h2 h3 dk^3 (Sec. 5)."""
    return float(np.sum(f) * cell_volume(prob))


def energy(f: np.ndarray, prob: Problem) -> float:
    """Energy: sum (hbar^2 |k|^2 / 2m + V(x)) f times the cell volume."""
    ks = prob.ks()
    K2 = ks[:, None, None] ** 2 + ks[None, :, None] ** 2 + ks[None, None, :] ** 2
    kin = np.einsum("abcijk,ijk->", f, K2) * prob.hbar**2 / (2 * prob.m)
    pot = np.einsum("abcijk,abc->", f, prob.potential())
    return float((kin + pot) * cell_volume(prob))


def reduced_wigner(f: np.ndarray, prob: Problem, j: int) -> np.ndarray:
    """W_j(x, k) = integral of f over the other two x and the other two k coordinates (Sec. 5),
    on the grid: the sum over those indices times their cell volume; shape (nx_j, N_k)."""
    others = [d for d in range(3) if d != j]
    vol = prob.hs(others[0]) * prob.hs(others[1]) * prob.dk ** 2
    return np.sum(f, axis=tuple(others) + tuple(3 + d for d in others)) * vol


def marginal_x12(f: np.ndarray, prob: Problem) -> np.ndarray:
    """P(x1, x2) = integral of f over x3 and k (Sec. 5); shape (nx_1, nx_2)."""
    return np.sum(f, axis=(2, 3, 4, 5)) * prob.hs(2) * prob.dk ** 3


def expectations(f: np.ndarray, prob: Problem) -> np.ndarray:
    """<x_d> and <k_d>, d = 1..3: the f-weighted grid averages sum(x_d f) / sum(f) and
    sum(k_d f) / sum(f) (the averaged position and momentum of Sec. 5.3)."""
    tot = np.sum(f)
    out = np.zeros(6)
    for d in range(3):
        shape = [1] * 6
        shape[d] = prob.nx[d]
        out[d] = np.sum(f * prob.xs(d).reshape(shape)) / tot
        shape = [1] * 6
        shape[3 + d] = prob.nk
        out[3 + d] = np.sum(f * prob.ks().reshape(shape)) / tot
    return out


def errors(f_ref: np.ndarray, f_num: np.ndarray, prob):
    """(eps_inf, eps_2) of Sec. 5: the largest |f_ref - f_num| over the grid, and the square root
    of the integral of (f_ref - f_num)^2 with the integral as the grid sum times the cell volume.
    prob is a Problem (cell h1 h2 h3 dk^3) or the cell volume itself (e.g. dk^3 for a function of k
    alone, as in Example 4.1)."""
    vol = cell_volume(prob) if isinstance(prob, Problem) else float(prob)
    d = f_ref - f_num
    return float(np.max(np.abs(d))), float(np.sqrt(np.sum(d * d) * vol))


def mass_error(f_num: np.ndarray, f_ref0: np.ndarray, prob: Problem) -> float:
    """eps_mass of Sec. 5: |integral of (f_num(t) - f_ref(0))|, the integral as the grid sum times
    the cell volume."""
    return float(abs(np.sum(f_num - f_ref0)) * cell_volume(prob))


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    """||a - b||_2 / ||b||_2."""
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


# --------------------------------------------------------------------------------------------
# Exact solutions for the quadratic potential (Sec. 5.1)
# --------------------------------------------------------------------------------------------


def harmonic_rotation(x, k, t, kappa, hbar=1.0, m=1.0):
    """Backward characteristics of Eq. 5.2 for V = kappa/2 |x|^2 (omega of the paper = kappa/m):
    returns (x(t), k(t)) such that f(x, k, t) = f0(x(t), k(t))."""
    w = math.sqrt(kappa / m)
    c, s = math.cos(w * t), math.sin(w * t)
    return c * x - (hbar / (m * w)) * s * k, (m * w / hbar) * s * x + c * k


def strang_discrete_map(x, k, dt, nsteps, kappa, hbar=1.0, m=1.0):
    """Feet of the exact Strang composition (a o p o a)^n, a: x -> x - hbar k dt/(2m),
    p: k -> k + dt kappa x / hbar, applied backwards from (x, k): f_n(x,k) = f0(feet)."""
    for _ in range(nsteps):
        x = x - hbar * k * dt / (2 * m)
        k = k + dt * kappa * x / hbar
        x = x - hbar * k * dt / (2 * m)
    return x, k
