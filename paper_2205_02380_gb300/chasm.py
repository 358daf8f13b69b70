"""ctypes binding of libchasm (include/chasm.h): argument marshalling only.

Every computation happens in the CUDA library; this module converts Python values and torch
tensors (device memory, streams) into the C structs and pointers of the ABI and turns negative
status codes into ``ChasmError``.  Importing it fails loudly if libchasm.so has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libchasm.so")

OK, PENDING = 0, 1
THETA_AUTO, THETA_TABLE, THETA_MODULATED = 0, 1, 2
STRANG, LPC1 = 0, 1
EINVAL, ENOMEM, ECUDA, EUNSTABLE, EBUSY, EAGAIN, ETIMEOUT, ENOTFOUND, ECANCELED = (
    -1, -2, -3, -4, -5, -6, -7, -8, -9)
FP32_MIXED, FP64 = 0, 1


class ChasmError(RuntimeError):
    """A negative status of the C ABI with chasm_last_error's message; .code is the status."""

    def __init__(self, code: int, msg: str):
        super().__init__(f"chasm error {code}: {msg}")
        self.code = code


class Grid(C.Structure):
    """chasm_grid (include/chasm.h)."""
    _fields_ = [("nx", C.c_int32 * 3), ("nk", C.c_int32 * 3)]


class Box(C.Structure):
    _fields_ = [("x_lo", C.c_double * 3), ("x_hi", C.c_double * 3), ("k_half", C.c_double * 3)]


class Nucleus(C.Structure):
    _fields_ = [("pos", C.c_double * 3), ("charge", C.c_double)]


class Potential(C.Structure):
    _fields_ = [("nuc", C.POINTER(Nucleus)), ("n_nuc", C.c_int32), ("harm_kappa", C.c_double),
                ("harm_center", C.c_double * 3)]


class Options(C.Structure):
    """chasm_options (include/chasm.h); fill with chasm_options_default first."""
    _fields_ = [("precision", C.c_int32), ("n_nb", C.c_int32), ("patches", C.c_int32 * 3),
                ("use_graphs", C.c_int32), ("cuda_stream", C.c_void_p), ("theta_form", C.c_int32),
                ("integrator", C.c_int32)]


class Gaussian(C.Structure):
    _fields_ = [("w", C.c_double), ("x0", C.c_double * 3), ("k0", C.c_double * 3),
                ("ax", C.c_double), ("ak", C.c_double)]


class Request(C.Structure):
    _fields_ = [("grid", Grid), ("box", Box), ("nuclei", Nucleus * 8), ("n_nuc", C.c_int32),
                ("harm_kappa", C.c_double), ("harm_center", C.c_double * 3),
                ("hbar", C.c_double), ("m", C.c_double), ("precision", C.c_int32),
                ("n_nb", C.c_int32), ("dt", C.c_double), ("nsteps", C.c_int32),
                ("packets", Gaussian * 4), ("n_packets", C.c_int32),
                ("f0_host", C.c_void_p), ("f_out_host", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("mass", C.c_double), ("energy", C.c_double),
                ("queue_ms", C.c_double), ("run_ms", C.c_double), ("latency_ms", C.c_double),
                ("cells", C.c_int64), ("nsteps", C.c_int32)]


# (name, restype, argtypes) for every function of include/chasm.h
_SIGS = [
    ("chasm_options_default", C.c_int, [C.POINTER(Options)]),
    ("chasm_create", C.c_int, [C.POINTER(Grid), C.POINTER(Box), C.POINTER(Potential), C.c_double,
                               C.c_double, C.POINTER(Options), C.POINTER(C.c_void_p)]),
    ("chasm_destroy", C.c_int, [C.c_void_p]),
    ("chasm_last_error", C.c_char_p, [C.c_void_p]),
    ("chasm_workspace_bytes", C.c_size_t, [C.POINTER(Grid), C.POINTER(Potential), C.POINTER(Options)]),
    ("chasm_num_cells", C.c_int64, [C.c_void_p]),
    ("chasm_f_bytes", C.c_size_t, [C.c_void_p]),
    ("chasm_set_stream", C.c_int, [C.c_void_p, C.c_void_p]),
    ("chasm_sync", C.c_int, [C.c_void_p]),
    ("chasm_launch_count", C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    ("chasm_step", C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_int32]),
    ("chasm_advect", C.c_int, [C.c_void_p, C.c_void_p, C.c_double]),
    ("chasm_pflow", C.c_int, [C.c_void_p, C.c_void_p, C.c_double]),
    ("chasm_theta", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("chasm_tkm_convolve", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("chasm_mass", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    ("chasm_energy", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    ("chasm_moments", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("chasm_reduced_wigner", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_double)]),
    ("chasm_marginal_x12", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    ("chasm_expectations", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    ("chasm_fma_peaks", C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("chasm_fma_peak_f32x2", C.c_int, [C.POINTER(C.c_double)]),
    ("chasm_fft_pk_rate", C.c_int, [C.POINTER(C.c_double)]),
    ("chasm_moments_noalloc", C.c_int, [C.c_void_p, C.POINTER(Grid), C.POINTER(Box), C.POINTER(Potential),
                                        C.c_double, C.c_double, C.c_int32, C.c_void_p,
                                        C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("chasm_init_gaussians", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Gaussian), C.c_int32]),
    ("chasm_init_hydrogen_1s", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_double)]),
    ("chasm_tkm_tensor", C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    ("chasm_run_host", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int32,
                                 C.POINTER(C.c_double)]),
    ("chasm_server_create", C.c_int, [C.c_size_t, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_void_p)]),
    ("chasm_submit", C.c_int, [C.c_void_p, C.POINTER(Request), C.POINTER(C.c_uint64)]),
    ("chasm_poll", C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(Result)]),
    ("chasm_wait", C.c_int, [C.c_void_p, C.c_uint64, C.c_double, C.POINTER(Result)]),
    ("chasm_cancel", C.c_int, [C.c_void_p, C.c_uint64]),
    ("chasm_server_stats", C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                     C.POINTER(C.c_size_t)]),
    ("chasm_server_destroy", C.c_int, [C.c_void_p]),
]

_lib = None


def lib() -> C.CDLL:
    """The loaded libchasm.  Raises if the library was not built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                              "(python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, handle=None) -> int:
    if rc < 0:
        msg = lib().chasm_last_error(handle)
        raise ChasmError(rc, msg.decode() if msg else "")
    return rc


def _ptr(t) -> int:
    """Device pointer of a torch tensor (must be contiguous) or an int address."""
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def make_grid(nx, nk) -> Grid:
    """chasm_grid: nx points per x-dimension (an int or three ints), N_k points per k-dimension."""
    nx = list(nx) if hasattr(nx, "__len__") else [nx] * 3
    return Grid((C.c_int32 * 3)(*nx), (C.c_int32 * 3)(nk, nk, nk))


def make_box(x_lo, x_hi, lk) -> Box:
    """chasm_box: x in [x_lo, x_hi] per dimension (ends included), k in [-lk, lk)."""
    x_lo = list(x_lo) if hasattr(x_lo, "__len__") else [x_lo] * 3
    x_hi = list(x_hi) if hasattr(x_hi, "__len__") else [x_hi] * 3
    return Box((C.c_double * 3)(*x_lo), (C.c_double * 3)(*x_hi), (C.c_double * 3)(lk, lk, lk))


def make_gaussian(w, x0, k0, ax, ak) -> Gaussian:
    """chasm_gaussian: w exp(-ax |x - x0|^2 - ak |k - k0|^2)."""
    return Gaussian(w, (C.c_double * 3)(*x0), (C.c_double * 3)(*k0), ax, ak)


class Solver:
    """One chasm_handle: a grid, a box and a potential, in FP32-mixed or FP64 form.

    Stream ordering with PyTorch: the handle issues its work on its own CUDA stream (a torch
    stream created here unless ``stream`` gives a cudaStream_t).  Every call first makes that
    stream wait for torch's current stream and afterwards makes torch's current stream wait for
    it, so tensors written by torch before a call are complete when the kernels read them and the
    results are visible to torch work issued after the call (device-side dependencies only)."""

    def __init__(self, nx, nk, x_lo, x_hi, lk, nuclei=(), kappa=0.0, center=(0.0, 0.0, 0.0),
                 hbar=1.0, m=1.0, precision=FP32_MIXED, n_nb=20, use_graphs=True, stream=None,
                 theta_form=THETA_AUTO, integrator=STRANG, patches=(1, 1, 1)):
        L = lib()
        self._tstream = None
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    self._tstream = torch.cuda.Stream()
                    stream = self._tstream.cuda_stream
            except ImportError:
                pass
        self._nuc = (Nucleus * max(1, len(nuclei)))(
            *[Nucleus((C.c_double * 3)(*p), z) for p, z in nuclei])
        self.grid = make_grid(nx, nk)
        self.box = make_box(x_lo, x_hi, lk)
        self.pot = Potential(self._nuc if nuclei else None, len(nuclei), kappa,
                             (C.c_double * 3)(*center))
        opt = Options()
        L.chasm_options_default(C.byref(opt))
        opt.precision = precision
        opt.n_nb = n_nb
        opt.use_graphs = 1 if use_graphs else 0
        opt.cuda_stream = stream if stream is not None else None
        opt.theta_form = theta_form
        opt.integrator = integrator
        opt.patches = (C.c_int32 * 3)(*patches)
        self.opt = opt
        h = C.c_void_p()
        _check(L.chasm_create(C.byref(self.grid), C.byref(self.box), C.byref(self.pot), hbar, m,
                              C.byref(opt), C.byref(h)))
        self.h = h
        self.precision = precision
        nxx = list(nx) if hasattr(nx, "__len__") else [nx] * 3
        self.shape = tuple(nxx) + (nk,) * 3

    def close(self):
        """chasm_destroy: frees the handle's workspace (idempotent)."""
        if getattr(self, "h", None):
            lib().chasm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # --- stream ordering with torch ---
    def _enter(self):
        if self._tstream is not None:
            import torch
            self._tstream.wait_stream(torch.cuda.current_stream())

    def _leave(self):
        if self._tstream is not None:
            import torch
            torch.cuda.current_stream().wait_stream(self._tstream)

    def _call(self, fn, *args):
        self._enter()
        try:
            _check(fn(self.h, *args), self.h)
        finally:
            self._leave()

    # --- calls ---
    def num_cells(self) -> int:
        """N_x1 N_x2 N_x3 N_k^3."""
        return lib().chasm_num_cells(self.h)

    def f_bytes(self) -> int:
        """Bytes of f in this handle's precision."""
        return lib().chasm_f_bytes(self.h)

    def set_stream(self, stream_ptr):
        """chasm_set_stream: issue later work on the cudaStream_t stream_ptr."""
        _check(lib().chasm_set_stream(self.h, stream_ptr), self.h)

    def sync(self):
        """chasm_sync: wait for the handle's stream."""
        self._call(lib().chasm_sync)

    def launch_count(self) -> int:
        """chasm_launch_count: kernels issued by step / advect / pflow since creation."""
        n = C.c_int64(0)
        self._call(lib().chasm_launch_count, C.byref(n))
        return n.value

    def step(self, f, dt, nsteps=1):
        """chasm_step: nsteps time steps of size dt on f in place (Strang or LPC1, as created);
        raises ChasmError(EUNSTABLE) when dt exceeds the stability bound."""
        self._call(lib().chasm_step, _ptr(f), dt, nsteps)

    def advect(self, f, tau):
        """chasm_advect: the spatial advection A(tau) alone, in place."""
        self._call(lib().chasm_advect, _ptr(f), tau)

    def pflow(self, f, dt):
        """chasm_pflow: the potential flow P(dt) alone, in place."""
        self._call(lib().chasm_pflow, _ptr(f), dt)

    def theta(self, u, out):
        """chasm_theta: out = Theta^T[u] (the Coulomb operator, or kappa (x - c)/hbar . grad_k u)."""
        self._call(lib().chasm_theta, _ptr(u), _ptr(out))

    def tkm_convolve(self, g, phi):
        """chasm_tkm_convolve: phi = T * g per x point (the TKM convolution of Sec. 4)."""
        self._call(lib().chasm_tkm_convolve, _ptr(g), _ptr(phi))

    def moments(self, f):
        """chasm_moments: (mass, energy) of f, FP64, bitwise reproducible."""
        m, e = C.c_double(), C.c_double()
        self._call(lib().chasm_moments, _ptr(f), C.byref(m), C.byref(e))
        return m.value, e.value

    def mass(self, f) -> float:
        """chasm_mass: h1 h2 h3 dk^3 sum f."""
        m = C.c_double()
        self._call(lib().chasm_mass, _ptr(f), C.byref(m))
        return m.value

    def energy(self, f) -> float:
        """chasm_energy: h1 h2 h3 dk^3 sum (hbar^2 |k|^2 / 2m + V(x)) f."""
        e = C.c_double()
        self._call(lib().chasm_energy, _ptr(f), C.byref(e))
        return e.value

    def reduced_wigner(self, f, j):
        """W_j as a (nx[j], N_k) float64 numpy array."""
        import numpy as np
        out = np.zeros((self.shape[j], self.shape[3]))
        self._call(lib().chasm_reduced_wigner, _ptr(f), j,
                   out.ctypes.data_as(C.POINTER(C.c_double)))
        return out

    def marginal_x12(self, f):
        """P(x1, x2) as a (nx[0], nx[1]) float64 numpy array."""
        import numpy as np
        out = np.zeros((self.shape[0], self.shape[1]))
        self._call(lib().chasm_marginal_x12, _ptr(f), out.ctypes.data_as(C.POINTER(C.c_double)))
        return out

    def expectations(self, f):
        """(<x_1>, <x_2>, <x_3>, <k_1>, <k_2>, <k_3>)."""
        out = (C.c_double * 6)()
        self._call(lib().chasm_expectations, _ptr(f), out)
        return tuple(out)

    def init_gaussians(self, f, packets):
        """chasm_init_gaussians: f = sum of the packets, each a dict w, x0, k0, ax, ak."""
        arr = (Gaussian * len(packets))(*[make_gaussian(p["w"], p["x0"], p["k0"], p["ax"], p["ak"])
                                          for p in packets])
        self._call(lib().chasm_init_gaussians, _ptr(f), arr, len(packets))

    def init_hydrogen_1s(self, f, n_y=128, center=(0.0, 0.0, 0.0)):
        """chasm_init_hydrogen_1s: the 1s Wigner function centred at center, from n_y^3 samples
        of the position-space orbital per k-direction."""
        c = (C.c_double * 3)(*center)
        self._call(lib().chasm_init_hydrogen_1s, _ptr(f), n_y, c)

    def tkm_tensor(self, out_ptr):
        """chasm_tkm_tensor: the FP64 truncated-kernel tensor T into host memory at out_ptr."""
        self._call(lib().chasm_tkm_tensor, C.cast(out_ptr, C.POINTER(C.c_double)))

    def run_host(self, f0_ptr, fout_ptr, dt, nsteps) -> float:
        m = C.c_double()
        self._call(lib().chasm_run_host, f0_ptr, fout_ptr, dt, nsteps, C.byref(m))
        return m.value


def workspace_bytes(nx, nk, nuclei=(), kappa=0.0, precision=FP32_MIXED, n_nb=20,
                    theta_form=THETA_AUTO, integrator=STRANG) -> int:
    """chasm_workspace_bytes: device bytes a handle with these settings allocates besides f."""
    L = lib()
    g = make_grid(nx, nk)
    nuc = (Nucleus * max(1, len(nuclei)))(*[Nucleus((C.c_double * 3)(*p), z) for p, z in nuclei])
    pot = Potential(nuc if nuclei else None, len(nuclei), kappa, (C.c_double * 3)(0, 0, 0))
    opt = Options()
    L.chasm_options_default(C.byref(opt))
    opt.precision = precision
    opt.n_nb = n_nb
    opt.theta_form = theta_form
    opt.integrator = integrator
    return L.chasm_workspace_bytes(C.byref(g), C.byref(pot), C.byref(opt))


class Server:
    """Continuous-batching server (chasm_server_*)."""

    def __init__(self, hbm_budget_bytes, max_slots=8, steps_per_launch=5, queue_capacity=1024):
        s = C.c_void_p()
        _check(lib().chasm_server_create(hbm_budget_bytes, max_slots, steps_per_launch,
                                         queue_capacity, C.byref(s)))
        self.s = s

    def submit(self, req: Request) -> int:
        t = C.c_uint64()
        _check(lib().chasm_submit(self.s, C.byref(req), C.byref(t)))
        return t.value

    def poll(self, ticket):
        r = Result()
        rc = _check(lib().chasm_poll(self.s, ticket, C.byref(r)))
        return None if rc == PENDING else r

    def wait(self, ticket, timeout_s=600.0) -> Result:
        r = Result()
        _check(lib().chasm_wait(self.s, ticket, timeout_s, C.byref(r)))
        return r

    def cancel(self, ticket):
        _check(lib().chasm_cancel(self.s, ticket))

    def stats(self):
        q, r, b = C.c_int32(), C.c_int32(), C.c_size_t()
        _check(lib().chasm_server_stats(self.s, C.byref(q), C.byref(r), C.byref(b)))
        return q.value, r.value, b.value

    def close(self):
        if getattr(self, "s", None):
            lib().chasm_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_request(nx, nk, x_lo, x_hi, lk, dt, nsteps, nuclei=(), kappa=0.0, packets=(),
                 precision=FP32_MIXED, hbar=1.0, m=1.0, n_nb=20, f0_ptr=None, fout_ptr=None) -> Request:
    """chasm_request for the server: the solve's grid, box, potential, dt and steps, its initial
    data (Gaussian packets, or a host buffer f0_ptr) and an optional host output buffer."""
    r = Request()
    r.grid = make_grid(nx, nk)
    r.box = make_box(x_lo, x_hi, lk)
    for i, (p, z) in enumerate(nuclei):
        r.nuclei[i] = Nucleus((C.c_double * 3)(*p), z)
    r.n_nuc = len(nuclei)
    r.harm_kappa = kappa
    r.hbar, r.m = hbar, m
    r.precision = precision
    r.n_nb = n_nb
    r.dt = dt
    r.nsteps = nsteps
    for i, p in enumerate(packets):
        r.packets[i] = make_gaussian(p["w"], p["x0"], p["k0"], p["ax"], p["ak"])
    r.n_packets = len(packets)
    r.f0_host = f0_ptr
    r.f_out_host = fout_ptr
    return r


def fma_peaks():
    """(FP32, FP64) SIMT FMA throughput of the current device in TFLOP/s (chasm_fma_peaks)."""
    a, b = C.c_double(), C.c_double()
    _check(lib().chasm_fma_peaks(C.byref(a), C.byref(b)))
    return a.value, b.value


def fma_peak_f32x2():
    """Packed single-precision FMA throughput in TFLOP/s (chasm_fma_peak_f32x2)."""
    a = C.c_double()
    _check(lib().chasm_fma_peak_f32x2(C.byref(a)))
    return a.value


def fft_pk_rate():
    """Algorithmic TFLOP/s of the P(dt) kernel's register FFT alone (chasm_fft_pk_rate)."""
    a = C.c_double()
    _check(lib().chasm_fft_pk_rate(C.byref(a)))
    return a.value
