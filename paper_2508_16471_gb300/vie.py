"""Thin ctypes binding of libvie.so (names follow include/vie.h).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  There is no fallback: if ``libvie.so`` is missing or
no CUDA device is present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libvie.so")

VIE_OK, VIE_EINVAL, VIE_ENOMEM, VIE_ENOCONV = 0, -1, -2, -3
VIE_ETIMEOUT, VIE_EUNDEF, VIE_EDEVICE, VIE_ESTATE = -4, -5, -6, -7
PREC_MIXED, PREC_FP64, PREC_F32X2 = 0, 1, 2
BASIS_CART, BASIS_SPH, BASIS_CIRC = 0, 1, 2
SOLVER_GMRES, SOLVER_BICGSTAB, SOLVER_COCR = 0, 1, 2
DISC_D1, DISC_D2 = 0, 1

EXPORTS = ["vie_default_opts", "vie_setup", "vie_set_eps", "vie_set_eps_device", "vie_solve",
           "vie_farfield", "vie_farfield_dirs", "vie_farfield_dirs_device", "hom_transfer",
           "vie_hom_map", "vie_get_current", "vie_apply", "vie_apply_device", "vie_fft_lines",
           "vie_get_info", "vie_kernel_launches", "vie_stream", "vie_destroy", "vie_last_error",
           "vie_set_fft_path", "vie_set_farfield_engine", "vie_cgemm", "vie_apply_noalloc", "vie_net_create", "vie_net_destroy", "vie_net_num_params", "vie_net_set_tensor_cores",
           "vie_net_get_params", "vie_net_set_params", "vie_net_forward", "vie_net_gradients",
           "vie_net_train_step", "vie_net_features", "vie_attach_net", "vie_guesses_rejected",
           "vie_net_create_io", "vie_attach_precond", "vie_precond_pairs", "vie_solve_many", "vie_autotune",
           "vie_setup_disc", "vie_farfield_na", "vie_timer_enable", "vie_timer_reset", "vie_timer_read", "vie_timer_name", "vie_timer_count",
           "vie_set_block_precond", "vie_block_apply_device", "vie_block_layout",
           "vie_batch_create", "vie_batch_destroy", "vie_batch_stride", "vie_batch_info", "vie_batch_apply_device",
           "vie_batch_solve", "vie_batch_get_current", "vie_batch_farfield_dirs"]


class VieError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class _Grid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("h", C.c_double), ("origin", C.c_double * 3)]


class _Channel(C.Structure):
    _fields_ = [("khat", C.c_double * 3), ("pol", C.c_double * 6)]


class _Opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("restart", C.c_int), ("max_iter", C.c_int),
                ("precision", C.c_int), ("inner_tol", C.c_double), ("use_x0", C.c_int),
                ("precond", C.c_int), ("solver", C.c_int), ("resid_fp64", C.c_int),
                ("reorth_eta", C.c_double), ("inner_floor", C.c_double), ("arnoldi", C.c_int)]


class _Stats(C.Structure):
    _fields_ = [("n_rhs", C.c_int), ("converged", C.c_int), ("iters_max", C.c_int),
                ("outer_max", C.c_int), ("matvecs32", C.c_longlong), ("matvecs64", C.c_longlong),
                ("relres_max", C.c_double), ("seconds", C.c_double),
                ("iters", C.POINTER(C.c_int)), ("relres", C.POINTER(C.c_double))]


class _Info(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("P", C.c_int * 3), ("n_body", C.c_longlong),
                ("n_rhs", C.c_int), ("device", C.c_int), ("device_bytes", C.c_double)]


_lib = None


def load():
    """Load libvie.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2508_16471_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    P = C.c_void_p
    dp = C.POINTER(C.c_double)
    L.vie_default_opts.argtypes = [C.POINTER(_Opts)]
    L.vie_setup.argtypes = [C.POINTER(_Grid), dp, C.c_double, C.POINTER(P)]
    L.vie_set_eps.argtypes = [P, dp]
    L.vie_set_eps_device.argtypes = [P, P]
    L.vie_solve.argtypes = [P, C.POINTER(_Channel), C.c_int, C.POINTER(_Opts), C.POINTER(_Stats)]
    L.vie_farfield.argtypes = [P, dp, C.c_int, dp, C.c_int, C.c_int, dp]
    L.vie_farfield_dirs.argtypes = [P, dp, C.c_int, C.c_int, dp]
    L.vie_farfield_dirs_device.argtypes = [P, P, C.c_int, C.c_int, P]
    L.hom_transfer.argtypes = [dp, dp, C.c_double, dp, C.c_int, dp, dp, dp]
    L.vie_hom_map.argtypes = [dp, C.c_int, dp, C.c_int, C.c_double, dp, dp, dp]
    L.vie_get_current.argtypes = [P, C.c_int, dp]
    L.vie_apply.argtypes = [P, dp, dp, C.c_int, C.c_int]
    L.vie_apply_device.argtypes = [P, P, P, C.c_int, C.c_int]
    L.vie_fft_lines.argtypes = [dp, dp, C.c_int, C.c_int, C.c_int, C.c_int]
    L.vie_get_info.argtypes = [P, C.POINTER(_Info)]
    L.vie_set_fft_path.argtypes = [P, C.c_int]
    fp = C.POINTER(C.c_float)
    L.vie_net_create.argtypes = [C.POINTER(C.c_int), C.c_ulonglong, C.c_int, C.POINTER(P)]
    L.vie_net_destroy.argtypes = [P]
    L.vie_net_destroy.restype = None
    L.vie_net_num_params.argtypes = [P]
    L.vie_net_num_params.restype = C.c_longlong
    L.vie_net_set_tensor_cores.argtypes = [P, C.c_int]
    L.vie_net_get_params.argtypes = [P, fp]
    L.vie_net_set_params.argtypes = [P, fp]
    L.vie_net_forward.argtypes = [P, P, P, C.c_int, C.c_int]
    L.vie_net_gradients.argtypes = [P, P, P, P, C.c_int, C.c_int, fp, fp]
    L.vie_net_train_step.argtypes = [P, P, P, P, C.c_int, C.c_int, C.c_float, fp]
    L.vie_net_features.argtypes = [P, C.c_int, P, P, P]
    L.vie_attach_net.argtypes = [P, P, C.c_int]
    L.vie_guesses_rejected.argtypes = [P]
    L.vie_guesses_rejected.restype = C.c_int
    L.vie_net_create_io.argtypes = [C.POINTER(C.c_int), C.c_int, C.c_ulonglong, C.c_int, C.POINTER(P)]
    L.vie_attach_precond.argtypes = [P, P, C.c_int]
    L.vie_precond_pairs.argtypes = [P, C.c_int, P, C.c_int, P, P, P]
    L.vie_solve_many.argtypes = [P, P, P, C.c_int, C.POINTER(_Opts), P, C.c_int]
    L.vie_autotune.argtypes = [P, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.vie_setup_disc.argtypes = [C.POINTER(_Grid), dp, C.c_double, C.c_int, C.POINTER(P)]
    L.vie_farfield_na.argtypes = [P, dp, dp, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, dp]
    L.vie_set_farfield_engine.argtypes = [P, C.c_int]
    L.vie_set_block_precond.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int]
    L.vie_block_apply_device.argtypes = [P, P, P]
    L.vie_block_layout.argtypes = [C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_longlong, C.POINTER(C.c_int),
                                   C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.vie_cgemm.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, dp, C.c_int]
    L.vie_kernel_launches.restype = C.c_longlong
    L.vie_stream.argtypes = [P]
    L.vie_stream.restype = P
    L.vie_destroy.argtypes = [P]
    L.vie_destroy.restype = None
    L.vie_batch_create.argtypes = [C.c_int, C.POINTER(_Grid), C.POINTER(dp), C.c_double, C.POINTER(P)]
    L.vie_batch_destroy.argtypes = [P]
    L.vie_batch_destroy.restype = None
    L.vie_batch_stride.argtypes = [P]
    L.vie_batch_stride.restype = C.c_longlong
    L.vie_batch_info.argtypes = [P, C.c_int, C.POINTER(_Info)]
    L.vie_batch_apply_device.argtypes = [P, P, P, C.c_int, C.c_int]
    L.vie_batch_solve.argtypes = [P, C.POINTER(_Channel), C.c_int, C.POINTER(_Opts), C.POINTER(_Stats)]
    L.vie_batch_get_current.argtypes = [P, C.c_int, C.c_int, dp]
    L.vie_batch_farfield_dirs.argtypes = [P, C.c_int, dp, C.c_int, C.c_int, dp]
    L.vie_last_error.restype = C.c_char_p
    L.vie_timer_enable.argtypes = [C.c_int]
    L.vie_timer_enable.restype = None
    L.vie_timer_reset.restype = None
    L.vie_timer_read.argtypes = [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                                 C.POINTER(C.c_double)]
    L.vie_timer_read.restype = C.c_int
    L.vie_timer_name.argtypes = [C.c_int]
    L.vie_timer_name.restype = C.c_char_p
    L.vie_timer_count.restype = C.c_int
    for f in ["vie_setup", "vie_set_eps", "vie_set_eps_device", "vie_solve", "vie_farfield",
              "vie_farfield_dirs", "vie_farfield_dirs_device", "hom_transfer", "vie_hom_map",
              "vie_get_current", "vie_apply", "vie_apply_device", "vie_fft_lines", "vie_get_info",
              "vie_set_fft_path", "vie_set_farfield_engine", "vie_cgemm", "vie_net_create",
              "vie_net_get_params", "vie_net_set_params", "vie_net_forward", "vie_net_gradients",
              "vie_net_train_step", "vie_net_features", "vie_attach_net", "vie_net_create_io",
              "vie_attach_precond", "vie_precond_pairs", "vie_solve_many", "vie_autotune", "vie_setup_disc",
              "vie_farfield_na", "vie_set_block_precond", "vie_block_apply_device", "vie_block_layout"]:
        getattr(L, f).restype = C.c_int
    _lib = L
    return L


def _check(code, allow=()):
    if code != VIE_OK and code not in allow:
        raise VieError(code, load().vie_last_error().decode())
    return code


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def kernel_launches() -> int:
    return int(load().vie_kernel_launches())


def timer_enable(on=True):
    load().vie_timer_enable(int(bool(on)))


def timer_reset():
    load().vie_timer_reset()


def timer_read():
    """{kernel name: (total ms, launches, algorithmic bytes)} since the last reset."""
    L = load()
    out = {}
    for i in range(L.vie_timer_count()):
        ms, n, b = C.c_double(), C.c_longlong(), C.c_double()
        L.vie_timer_read(i, C.byref(ms), C.byref(n), C.byref(b))
        out[L.vie_timer_name(i).decode()] = (ms.value, n.value, b.value)
    return out


def default_opts(**kw):
    o = _Opts()
    load().vie_default_opts(C.byref(o))
    names = {f[0] for f in _Opts._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"unknown solve option {k!r}")
        setattr(o, k, v)
    return o


def _channels(chs):
    arr = (_Channel * len(chs))()
    for i, c in enumerate(chs):
        if hasattr(c, "khat"):
            k, p = c.khat, c.pol
        else:
            k, p = c
        p = np.asarray(p, dtype=np.complex128)
        for q in range(3):
            arr[i].khat[q] = float(k[q])
            arr[i].pol[2 * q] = float(p[q].real)
            arr[i].pol[2 * q + 1] = float(p[q].imag)
    return arr


class Handle:
    """One grid + body on the current CUDA device (vie_setup ... vie_destroy)."""

    def __init__(self, n, h, eps_r, k0=2.0 * np.pi, origin=(0.0, 0.0, 0.0), disc=DISC_D1):
        L = load()
        g = _Grid()
        for a in range(3):
            g.n[a] = int(n[a])
            g.origin[a] = float(origin[a])
        g.h = float(h)
        self.n = tuple(int(v) for v in n)
        eps = np.ascontiguousarray(eps_r, dtype=np.float64).reshape(self.n)
        hp = C.c_void_p()
        _check(L.vie_setup_disc(C.byref(g), _dptr(eps), float(k0), int(disc), C.byref(hp)))
        self._h = hp
        self.n_rhs = 0

    def close(self):
        if getattr(self, "_h", None):
            load().vie_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def ptr(self):
        return self._h

    def info(self):
        i = _Info()
        _check(load().vie_get_info(self._h, C.byref(i)))
        return dict(n=tuple(i.n), P=tuple(i.P), n_body=int(i.n_body), n_rhs=int(i.n_rhs),
                    device=int(i.device), device_bytes=float(i.device_bytes))

    def stream(self):
        return load().vie_stream(self._h)

    def set_fft_path(self, path: int):
        _check(load().vie_set_fft_path(self._h, int(path)))

    def set_farfield_engine(self, engine: int):
        _check(load().vie_set_farfield_engine(self._h, int(engine)))

    def net_features(self, factor, x_ptr, t_ptr=None, m_ptr=None):
        """Coarse-grid network features of the last solve's RHS (device float32
        buffers: x [rhs][10][D^3], optional targets t [rhs][6][D^3], mask m [rhs][D^3])."""
        _check(load().vie_net_features(self._h, int(factor), C.c_void_p(x_ptr),
                                       C.c_void_p(t_ptr) if t_ptr else None,
                                       C.c_void_p(m_ptr) if m_ptr else None))

    def attach_net(self, net, factor):
        _check(load().vie_attach_net(self._h, net.ptr if net is not None else None, int(factor)))
        self._net = net  # keep alive

    def guesses_rejected(self):
        return int(load().vie_guesses_rejected(self._h))

    def farfield_na(self, centers, pols, theta_na, sigma, nt=12, nphi=16):
        """vie_farfield_na: aperture-collected detector amplitudes [n_rhs][D] complex."""
        c = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1, 3)
        p = _c128(np.asarray(pols).reshape(-1, 3))
        D = c.shape[0]
        out = np.zeros((self.n_rhs, D), dtype=np.complex128)
        _check(load().vie_farfield_na(self._h, _dptr(c), _dptr(p.view(np.float64)), D, float(theta_na),
                                      float(sigma), int(nt), int(nphi), _dptr(out.view(np.float64))))
        return out

    def autotune(self, n_rhs=8, reps=3):
        """vie_autotune: time the candidate FFT schedules and keep the fastest;
        returns (padded lengths, ms per FP32 application)."""
        P = (C.c_int * 3)()
        ms = C.c_double()
        _check(load().vie_autotune(self._h, int(n_rhs), int(reps), P, C.byref(ms)))
        return tuple(P), ms.value

    def set_block_precond(self, cuts=((), (), ()), inner=8):
        """Block-Jacobi preconditioner used by solve(..., precond=2): blocks are
        the cells of the tiling with interior cut positions cuts[a] on axis a,
        each solved approximately by `inner` COCR steps."""
        nc = (C.c_int * 3)(*[len(c) for c in cuts])
        flat = [int(v) for c in cuts for v in c]
        arr = (C.c_int * max(1, len(flat)))(*flat) if flat else None
        _check(load().vie_set_block_precond(self._h, arr, nc, int(inner)))

    def block_apply_device(self, w_ptr: int, y_ptr: int):
        """y = A_bd w (block operator) for one complex64 compact vector [3][n_body]."""
        _check(load().vie_block_apply_device(self._h, C.c_void_p(w_ptr), C.c_void_p(y_ptr)))

    def attach_precond(self, net, factor):
        """Network used as the FGMRES right preconditioner by solve(..., precond=1)."""
        _check(load().vie_attach_precond(self._h, net.ptr if net is not None else None, int(factor)))
        self._pnet = net  # keep alive

    def precond_pairs(self, factor, v_ptr, n, x_ptr, t_ptr, m_ptr):
        """Preconditioner training pairs of n complex64 body-layout vectors v
        (device): x [n][7][D^3], t [n][6][D^3], m [n][D^3] (device float32)."""
        _check(load().vie_precond_pairs(self._h, int(factor), C.c_void_p(v_ptr), int(n), C.c_void_p(x_ptr),
                                        C.c_void_p(t_ptr), C.c_void_p(m_ptr)))

    def set_eps(self, eps_r):
        eps = np.ascontiguousarray(eps_r, dtype=np.float64).reshape(self.n)
        _check(load().vie_set_eps(self._h, _dptr(eps)))
        self.n_rhs = 0

    def set_eps_device(self, ptr: int):
        _check(load().vie_set_eps_device(self._h, C.c_void_p(ptr)))
        self.n_rhs = 0

    def solve(self, channels, allow_noconv=False, **opts):
        o = default_opts(**opts)
        R = len(channels)
        iters = np.zeros(R, dtype=np.int32)
        rel = np.zeros(R, dtype=np.float64)
        st = _Stats()
        st.iters = iters.ctypes.data_as(C.POINTER(C.c_int))
        st.relres = rel.ctypes.data_as(C.POINTER(C.c_double))
        code = load().vie_solve(self._h, _channels(channels), R, C.byref(o), C.byref(st))
        _check(code, allow=(VIE_ENOCONV,) if allow_noconv else ())
        self.n_rhs = R
        return dict(code=code, converged=st.converged, iters_max=st.iters_max, outer_max=st.outer_max,
                    matvecs32=st.matvecs32, matvecs64=st.matvecs64, relres_max=st.relres_max,
                    seconds=st.seconds, iters=iters, relres=rel)

    def farfield(self, theta, phi, basis=BASIS_CART):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        ph = np.ascontiguousarray(phi, dtype=np.float64)
        out = np.zeros((self.n_rhs, len(th), len(ph), 3), dtype=np.complex128)
        _check(load().vie_farfield(self._h, _dptr(th), len(th), _dptr(ph), len(ph), int(basis),
                                   out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def farfield_dirs(self, dirs, basis=BASIS_CART):
        d = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
        out = np.zeros((self.n_rhs, len(d), 3), dtype=np.complex128)
        _check(load().vie_farfield_dirs(self._h, _dptr(d), len(d), int(basis),
                                        out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def farfield_dirs_device(self, dirs_ptr: int, D: int, out_ptr: int, basis=BASIS_CART):
        _check(load().vie_farfield_dirs_device(self._h, C.c_void_p(dirs_ptr), int(D), int(basis),
                                               C.c_void_p(out_ptr)))

    def get_current(self, rhs):
        out = np.zeros((3,) + self.n, dtype=np.complex128)
        _check(load().vie_get_current(self._h, int(rhs), out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def apply(self, w, precision=PREC_FP64):
        w = _c128(w)
        if w.ndim != 5 or w.shape[1:] != (3,) + self.n:
            raise ValueError(f"apply takes full-grid fields [n_rhs][3]{list(self.n)}, got {list(w.shape)}")
        R = w.shape[0]
        y = np.zeros_like(w)
        _check(load().vie_apply(self._h, _dptr(w.view(np.float64)), y.ctypes.data_as(C.POINTER(C.c_double)),
                                R, int(precision)))
        return y

    def apply_device(self, w_ptr: int, y_ptr: int, n_rhs: int, precision=PREC_MIXED):
        _check(load().vie_apply_device(self._h, C.c_void_p(w_ptr), C.c_void_p(y_ptr), int(n_rhs),
                                       int(precision)))


class Batch:
    """Many bodies of uneven grids (vie_batch_*): bodies = [(n, h, eps_r), ...]
    with one k0; rows of batch vectors are body-major ([body][rhs][3][stride])."""

    def __init__(self, bodies, k0=2.0 * np.pi):
        L = load()
        nb = len(bodies)
        grids = (_Grid * nb)()
        self._eps = []
        ptrs = (C.POINTER(C.c_double) * nb)()
        self.n = []
        for i, (n, h, eps) in enumerate(bodies):
            for a in range(3):
                grids[i].n[a] = int(n[a])
                grids[i].origin[a] = 0.0
            grids[i].h = float(h)
            e = np.ascontiguousarray(eps, dtype=np.float64).reshape(tuple(int(v) for v in n))
            self._eps.append(e)
            ptrs[i] = _dptr(e)
            self.n.append(tuple(int(v) for v in n))
        hp = C.c_void_p()
        _check(L.vie_batch_create(nb, grids, ptrs, float(k0), C.byref(hp)))
        self._h = hp
        self.n_bodies = nb
        self.n_rhs = 0

    def close(self):
        if getattr(self, "_h", None):
            load().vie_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def stride(self):
        return int(load().vie_batch_stride(self._h))

    def info(self, body):
        i = _Info()
        _check(load().vie_batch_info(self._h, int(body), C.byref(i)))
        return dict(n=tuple(i.n), P=tuple(i.P), n_body=int(i.n_body), n_rhs=int(i.n_rhs),
                    device=int(i.device), device_bytes=float(i.device_bytes))

    def apply_device(self, w_ptr: int, y_ptr: int, n_rhs: int, precision=PREC_MIXED):
        _check(load().vie_batch_apply_device(self._h, C.c_void_p(w_ptr), C.c_void_p(y_ptr), int(n_rhs),
                                             int(precision)))

    def solve(self, channels, allow_noconv=False, **opts):
        o = default_opts(**opts)
        R = len(channels) * self.n_bodies
        iters = np.zeros(R, dtype=np.int32)
        rel = np.zeros(R, dtype=np.float64)
        st = _Stats()
        st.iters = iters.ctypes.data_as(C.POINTER(C.c_int))
        st.relres = rel.ctypes.data_as(C.POINTER(C.c_double))
        code = load().vie_batch_solve(self._h, _channels(channels), len(channels), C.byref(o), C.byref(st))
        _check(code, allow=(VIE_ENOCONV,) if allow_noconv else ())
        self.n_rhs = len(channels)
        return dict(code=code, converged=st.converged, iters_max=st.iters_max, outer_max=st.outer_max,
                    matvecs32=st.matvecs32, matvecs64=st.matvecs64, relres_max=st.relres_max,
                    seconds=st.seconds, iters=iters.reshape(self.n_bodies, -1), relres=rel.reshape(self.n_bodies, -1))

    def get_current(self, body, rhs):
        out = np.zeros((3,) + self.n[body], dtype=np.complex128)
        _check(load().vie_batch_get_current(self._h, int(body), int(rhs),
                                            out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def farfield_dirs(self, body, dirs, basis=BASIS_CART):
        d = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
        out = np.zeros((self.n_rhs, len(d), 3), dtype=np.complex128)
        _check(load().vie_batch_farfield_dirs(self._h, int(body), _dptr(d), len(d), int(basis),
                                              out.ctypes.data_as(C.POINTER(C.c_double))))
        return out


class Net:
    """The learned network (vie_net_*): cin = 10 for the initial guess, 7 for
    the preconditioner; device buffers are passed as raw pointers (e.g.
    torch.Tensor.data_ptr())."""

    def __init__(self, channels=(16, 32, 64, 128), seed=0, bf16=True, cin=10):
        L = load()
        ch = (C.c_int * 4)(*[int(c) for c in channels])
        p = C.c_void_p()
        _check(L.vie_net_create_io(ch, int(cin), C.c_ulonglong(seed), int(bool(bf16)), C.byref(p)))
        self._p = p
        self.channels = tuple(channels)
        self.cin = int(cin)

    @property
    def ptr(self):
        return self._p

    def close(self):
        if getattr(self, "_p", None):
            load().vie_net_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def num_params(self):
        return int(load().vie_net_num_params(self._p))

    def set_tensor_cores(self, on):
        _check(load().vie_net_set_tensor_cores(self._p, 1 if on else 0))

    def get_params(self):
        a = np.zeros(self.num_params(), dtype=np.float32)
        _check(load().vie_net_get_params(self._p, a.ctypes.data_as(C.POINTER(C.c_float))))
        return a

    def set_params(self, a):
        a = np.ascontiguousarray(a, dtype=np.float32)
        assert a.size == self.num_params()
        _check(load().vie_net_set_params(self._p, a.ctypes.data_as(C.POINTER(C.c_float))))

    def forward(self, x_ptr, y_ptr, B, D):
        _check(load().vie_net_forward(self._p, C.c_void_p(x_ptr), C.c_void_p(y_ptr), int(B), int(D)))

    def gradients(self, x_ptr, t_ptr, m_ptr, B, D):
        loss = C.c_float()
        g = np.zeros(self.num_params(), dtype=np.float32)
        _check(load().vie_net_gradients(self._p, C.c_void_p(x_ptr), C.c_void_p(t_ptr), C.c_void_p(m_ptr), int(B),
                                        int(D), C.byref(loss), g.ctypes.data_as(C.POINTER(C.c_float))))
        return float(loss.value), g

    def train_step(self, x_ptr, t_ptr, m_ptr, B, D, lr):
        loss = C.c_float()
        _check(load().vie_net_train_step(self._p, C.c_void_p(x_ptr), C.c_void_p(t_ptr), C.c_void_p(m_ptr), int(B),
                                         int(D), float(lr), C.byref(loss)))
        return float(loss.value)


def hom_transfer(E, omega=None, sigma=1.2, dtau=()):
    """g2, N~c(dtau), visibility for E[2 det][2 ch] complex."""
    e = _c128(np.asarray(E).reshape(2, 2)).view(np.float64).reshape(-1).copy()
    dt = np.ascontiguousarray(dtau, dtype=np.float64)
    nc = np.zeros(len(dt))
    g2 = np.zeros(1)
    vis = np.zeros(1)
    om = None if omega is None else np.ascontiguousarray(omega, dtype=np.float64)
    code = load().hom_transfer(_dptr(e), None if om is None else _dptr(om), float(sigma),
                               _dptr(dt) if len(dt) else None, len(dt), _dptr(g2),
                               _dptr(nc) if len(dt) else None, _dptr(vis))
    _check(code, allow=(VIE_EUNDEF,))
    return float(g2[0]), nc, float(vis[0]), code


def solve_many(handles, channel_lists, allow_noconv=False, max_threads=0, **opts):
    """vie_solve_many: the solves of several handles (bodies) run concurrently;
    returns one stats dict per handle (as Handle.solve)."""
    n = len(handles)
    assert len(channel_lists) == n and n > 0
    o = default_opts(**opts)
    chs = [_channels(c) for c in channel_lists]
    ch_ptrs = (C.POINTER(_Channel) * n)(*[C.cast(c, C.POINTER(_Channel)) for c in chs])
    hs = (C.c_void_p * n)(*[h._h for h in handles])
    nr = (C.c_int * n)(*[len(c) for c in channel_lists])
    stats = (_Stats * n)()
    its = [np.zeros(len(c), dtype=np.int32) for c in channel_lists]
    rels = [np.zeros(len(c), dtype=np.float64) for c in channel_lists]
    for i in range(n):
        stats[i].iters = its[i].ctypes.data_as(C.POINTER(C.c_int))
        stats[i].relres = rels[i].ctypes.data_as(C.POINTER(C.c_double))
    code = load().vie_solve_many(hs, ch_ptrs, nr, n, C.byref(o), stats, int(max_threads))
    _check(code, allow=(VIE_ENOCONV,) if allow_noconv else ())
    out = []
    for i, h in enumerate(handles):
        h.n_rhs = len(channel_lists[i])
        st = stats[i]
        out.append(dict(converged=st.converged, iters_max=st.iters_max, outer_max=st.outer_max,
                        matvecs32=st.matvecs32, matvecs64=st.matvecs64, relres_max=st.relres_max,
                        seconds=st.seconds, iters=its[i], relres=rels[i]))
    return out


def hom_map(Ea, Eb, sigma=1.2):
    """g2, visibility and normalised classical P2 over all pairs (a in A, b in B).
    Ea: [2][nA] complex (channels 1, 2), Eb: [2][nB]."""
    a = _c128(Ea)
    b = _c128(Eb)
    nA, nB = a.shape[1], b.shape[1]
    g2 = np.zeros((nA, nB))
    vis = np.zeros((nA, nB))
    p2 = np.zeros((nA, nB))
    _check(load().vie_hom_map(_dptr(a.view(np.float64)), nA, _dptr(b.view(np.float64)), nB, float(sigma),
                              _dptr(g2), _dptr(vis), _dptr(p2)))
    return g2, vis, p2


def cgemm(A, B, engine=0):
    """C = A B (complex) on the device: engine 0 tensor cores (3xTF32), 1 CUDA cores."""
    a = _c128(A)
    b = _c128(B)
    M, K = a.shape
    K2, N = b.shape
    assert K == K2
    c = np.zeros((M, N), dtype=np.complex128)
    _check(load().vie_cgemm(M, N, K, _dptr(a.view(np.float64)), _dptr(b.view(np.float64)),
                            c.ctypes.data_as(C.POINTER(C.c_double)), int(engine)))
    return c


def block_layout(n, vox, cuts=((), (), ())):
    """Host-side block layout of vie_set_block_precond: (box, blocks, map[blocks][box0][box1][box2])."""
    L = load()
    nn = (C.c_int * 3)(*[int(v) for v in n])
    vx = np.ascontiguousarray(vox, dtype=np.int32)
    nc = (C.c_int * 3)(*[len(c) for c in cuts])
    flat = [int(v) for c in cuts for v in c]
    arr = (C.c_int * max(1, len(flat)))(*flat) if flat else None
    box = (C.c_int * 3)()
    T = C.c_int()
    vp = vx.ctypes.data_as(C.POINTER(C.c_int))
    _check(L.vie_block_layout(nn, vp, len(vx), arr, nc, box, C.byref(T), None))
    m = np.zeros((T.value, box[0], box[1], box[2]), dtype=np.int32)
    _check(L.vie_block_layout(nn, vp, len(vx), arr, nc, box, C.byref(T), m.ctypes.data_as(C.POINTER(C.c_int))))
    return tuple(box), T.value, m


def fft_lines(x, inverse=False, precision=PREC_FP64):
    x = _c128(np.atleast_2d(x))
    out = np.zeros_like(x)
    _check(load().vie_fft_lines(_dptr(x.view(np.float64)), out.ctypes.data_as(C.POINTER(C.c_double)),
                                x.shape[1], x.shape[0], int(bool(inverse)), int(precision)))
    return out
