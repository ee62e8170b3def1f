"""GB300-native three-grid IOFD Helmholtz solver: Python binding of libhz.so.

Thin ctypes marshalling over the C ABI declared in ``include/hz.h``: every
operator, smoother, transfer and Krylov step runs in the library's CUDA
kernels.  PyTorch provides device memory and streams.  There is no CPU
fallback: loading fails loudly when the library or a GPU is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhz.so")
TABLE_PATH = os.path.join(HERE, "tables", "iofd_tables.txt")

HZ_OK, HZ_EINVAL, HZ_ENOMEM, HZ_ECUDA, HZ_ENOCONV, HZ_ETIMEOUT, HZ_ENONFINITE = range(7)
HZ_C64, HZ_C128 = 0, 1
HZ_OP_A, HZ_OP_B, HZ_OP_Q, HZ_OP_A_ADJ, HZ_OP_B_ADJ, HZ_OP_Q_ADJ = range(6)
_STATUS = {0: "HZ_OK", 1: "HZ_EINVAL", 2: "HZ_ENOMEM", 3: "HZ_ECUDA", 4: "HZ_ENOCONV", 5: "HZ_ETIMEOUT",
           6: "HZ_ENONFINITE"}

EXPORTED = ["hz_default_params", "hz_create", "hz_destroy", "hz_last_error", "hz_workspace_bytes",
            "hz_set_params", "iofd_coeffs", "iofd_apply", "threegrid_precond", "helmholtz_solve",
            "helmholtz_adjoint_grad", "hz_kernel_launches", "iofd_residual_static", "hz_layout_check",
            "iofd_jacobi", "iofd_apply_window"]


class HzGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("n_pml", ctypes.c_int),
                ("h", ctypes.c_double), ("omega", ctypes.c_double), ("gamma_max", ctypes.c_double)]


class HzSource(ctypes.Structure):
    _fields_ = [("ix", ctypes.c_int), ("iy", ctypes.c_int), ("iz", ctypes.c_int),
                ("amp_re", ctypes.c_double), ("amp_im", ctypes.c_double)]


class HzParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_pc", ctypes.c_int), ("m_out", ctypes.c_int),
                ("m_h", ctypes.c_int), ("nJ_h", ctypes.c_int), ("c_2h", ctypes.c_int), ("m_2h", ctypes.c_int),
                ("nJ_2h", ctypes.c_int), ("m_4h", ctypes.c_int), ("nJ_4h", ctypes.c_int),
                ("w_h", ctypes.c_double), ("w_2h", ctypes.c_double), ("w_4h", ctypes.c_double),
                ("sigma", ctypes.c_double), ("precision", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("max_refine", ctypes.c_int), ("autotune", ctypes.c_int), ("refine", ctypes.c_int),
                ("block", ctypes.c_int)]


class HzStats(ctypes.Structure):
    _fields_ = [("pc_calls", ctypes.c_int), ("refine_passes", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("t_setup", ctypes.c_double), ("t_solve", ctypes.c_double), ("device_bytes", ctypes.c_size_t),
                ("zblock", ctypes.c_int * 3), ("zblock_frame", ctypes.c_int * 3)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["zblock"] = list(self.zblock)
        d["zblock_frame"] = list(self.zblock_frame)
        return d


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libhz.so (build it with ``paper_2608_22946_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -m paper_2608_22946_gb300.build)")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    lib.hz_default_params.argtypes = [P(HzParams)]
    lib.hz_default_params.restype = None
    lib.hz_create.argtypes = [P(HzGrid), vp, P(HzParams), P(ctypes.c_double), ctypes.c_int, ctypes.c_int, vp,
                              P(vp)]
    lib.hz_destroy.argtypes = [vp]
    lib.hz_last_error.argtypes = [vp]
    lib.hz_last_error.restype = ctypes.c_char_p
    lib.hz_workspace_bytes.argtypes = [P(HzGrid), P(HzParams), ctypes.c_int, P(ctypes.c_size_t)]
    lib.hz_set_params.argtypes = [vp, P(HzParams)]
    lib.hz_kernel_launches.argtypes = []
    lib.hz_kernel_launches.restype = ctypes.c_ulonglong
    lib.iofd_coeffs.argtypes = [vp, ctypes.c_int, vp, vp]
    lib.iofd_apply.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_int, vp]
    lib.iofd_apply_window.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      vp]
    lib.iofd_jacobi.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, vp, vp,
                                ctypes.c_int, vp]
    lib.iofd_residual_static.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp,
                                         ctypes.c_int, vp]
    lib.hz_layout_check.argtypes = [P(HzGrid), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, vp, P(ctypes.c_longlong), P(ctypes.c_longlong)]
    lib.threegrid_precond.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]
    lib.helmholtz_solve.argtypes = [vp, P(HzSource), ctypes.c_int, vp, vp, P(HzStats)]
    lib.helmholtz_adjoint_grad.argtypes = [vp, P(HzSource), ctypes.c_int, P(ctypes.c_int), ctypes.c_int,
                                           P(ctypes.c_double), P(ctypes.c_double), vp, P(HzStats)]
    for name in EXPORTED:
        if name not in ("hz_default_params", "hz_last_error", "hz_kernel_launches"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class HzError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


def default_params(**overrides) -> HzParams:
    p = HzParams()
    load_library().hz_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def load_table(path: str = TABLE_PATH) -> np.ndarray:
    """IOFD Hermite table rows (s, alpha, alpha', beta, beta')."""
    return np.ascontiguousarray(np.loadtxt(path, comments="#"), dtype=np.float64)


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _nrhs(t, n, name):
    """Right-hand sides in a field tensor of level size n (a whole number of fields)."""
    if t.numel() == 0 or t.numel() % n:
        raise ValueError(f"{name}: {t.numel()} elements is not a whole, non-zero number of fields of {n} nodes")
    return t.numel() // n


def _check_field(t, dtype, n, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()
            and t.numel() >= n):
        raise ValueError(f"{name}: need a contiguous CUDA {dtype} tensor with at least {n} elements")


class Solver:
    """One frequency and velocity model (``hz_create``)."""

    def __init__(self, n, n_pml, h, omega, c, params: HzParams | None = None, table=None, max_nrhs=1,
                 gamma_max=1.119058, stream=None):
        import torch
        lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        nx, ny, nz = (n, n, n) if np.isscalar(n) else n
        self.shape = (nz + 1, ny + 1, nx + 1)
        self.grid = HzGrid(nx, ny, nz, n_pml, h, omega, gamma_max)
        self.params = params or default_params()
        tab = load_table() if table is None else np.ascontiguousarray(table, dtype=np.float64)
        c_t = torch.as_tensor(c, dtype=torch.float64).reshape(-1).contiguous().cuda()
        if c_t.numel() != int(np.prod(self.shape)):
            raise ValueError("velocity size does not match the grid")
        self.max_nrhs = max_nrhs
        self._lib = lib
        handle = ctypes.c_void_p()
        st = lib.hz_create(ctypes.byref(self.grid), ctypes.c_void_p(c_t.data_ptr()), ctypes.byref(self.params),
                           tab.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), tab.shape[0], max_nrhs,
                           _stream_ptr(stream), ctypes.byref(handle))
        if st != HZ_OK:
            raise HzError(st, lib.hz_last_error(None).decode())
        self._h = handle
        self.N = [((nx >> L) + 1) * ((ny >> L) + 1) * ((nz >> L) + 1) for L in range(3)]
        self.level_shape = [((nz >> L) + 1, (ny >> L) + 1, (nx >> L) + 1) for L in range(3)]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.hz_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ok(self, st):
        if st not in (HZ_OK,):
            raise HzError(st, self._lib.hz_last_error(self._h).decode())

    def set_params(self, params: HzParams):
        self._ok(self._lib.hz_set_params(self._h, ctypes.byref(params)))
        self.params = params

    # -- iofd_coeffs ---------------------------------------------------------
    def iofd_coeffs(self, level=0, shell=True):
        import torch
        kap = torch.empty(self.N[level], dtype=torch.float64, device="cuda")
        sh = torch.empty(4 * self.N[level], dtype=torch.float64, device="cuda") if shell else None
        self._ok(self._lib.iofd_coeffs(self._h, level, ctypes.c_void_p(kap.data_ptr()),
                                       ctypes.c_void_p(sh.data_ptr()) if shell else None))
        return kap.reshape(self.level_shape[level]), (sh.reshape((4,) + self.level_shape[level]) if shell else None)

    # -- iofd_apply ----------------------------------------------------------
    def iofd_apply(self, x, op=HZ_OP_A, level=0, out=None, stream=None):
        import torch
        prec = HZ_C64 if x.dtype == torch.complex64 else HZ_C128
        n = self.N[level]
        nrhs = _nrhs(x, n, "x")
        _check_field(x, x.dtype, n * nrhs, "x")
        y = torch.empty_like(x) if out is None else out
        _check_field(y, x.dtype, n * nrhs, "out")
        self._ok(self._lib.iofd_apply(self._h, level, op, prec, ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(y.data_ptr()), nrhs, _stream_ptr(stream)))
        return y

    def iofd_apply_window(self, x_win, z0, z1, op=HZ_OP_A, out=None, stream=None):
        """Rows z0 .. z1-1 of Op x on the fine level from a brick with a one-plane
        halo: x_win holds planes z0-1 .. z1 ((z1 - z0 + 2) planes per right-hand
        side), the result (z1 - z0) planes per right-hand side."""
        import torch
        prec = HZ_C64 if x_win.dtype == torch.complex64 else HZ_C128
        nz = self.level_shape[0][0]
        if not (0 <= z0 < z1 <= nz):
            raise ValueError(f"need 0 <= z0 < z1 <= {nz}")
        plane = self.level_shape[0][1] * self.level_shape[0][2]
        nrhs = _nrhs(x_win, (z1 - z0 + 2) * plane, "x_win")
        _check_field(x_win, x_win.dtype, (z1 - z0 + 2) * plane * nrhs, "x_win")
        y = (torch.empty((nrhs, z1 - z0) + self.level_shape[0][1:], dtype=x_win.dtype, device=x_win.device)
             if out is None else out)
        _check_field(y, x_win.dtype, (z1 - z0) * plane * nrhs, "out")
        self._ok(self._lib.iofd_apply_window(self._h, op, prec, ctypes.c_void_p(x_win.data_ptr()),
                                             ctypes.c_void_p(y.data_ptr()), nrhs, z0, z1, _stream_ptr(stream)))
        return y

    # -- iofd_jacobi -----------------------------------------------------------
    def iofd_jacobi(self, g, level=0, nsweeps=2, omega=None, out=None, stream=None):
        """y = J_nsweeps(H, g; omega) with H = A_h on level 0 and B on levels 1, 2
        (the smoothers of Algorithm 1); omega defaults to the handle's weight of
        that level."""
        import torch
        prec = HZ_C64 if g.dtype == torch.complex64 else HZ_C128
        n = self.N[level]
        if g.numel() % n:
            raise ValueError(f"g: {g.numel()} elements is not a whole number of level-{level} fields ({n})")
        nrhs = _nrhs(g, n, "g")
        _check_field(g, g.dtype, n * nrhs, "g")
        y = torch.empty_like(g) if out is None else out
        _check_field(y, g.dtype, n * nrhs, "out")
        if omega is None:
            omega = (self.params.w_h, self.params.w_2h, self.params.w_4h)[level]
        op = HZ_OP_A if level == 0 else HZ_OP_B
        self._ok(self._lib.iofd_jacobi(self._h, level, op, prec, nsweeps, float(omega), ctypes.c_void_p(g.data_ptr()),
                                       ctypes.c_void_p(y.data_ptr()), nrhs, _stream_ptr(stream)))
        return y

    # -- iofd_residual_static --------------------------------------------------
    def residual_static(self, g, x, op=HZ_OP_A, level=0, out=None, norm2_out=None, stream=None):
        """r = g - Op x and ||r||^2 per right-hand side through the entry point
        that allocates no device memory (its reduction scratch is a static
        device array of the library); returns (r, norm2)."""
        import torch
        prec = HZ_C64 if x.dtype == torch.complex64 else HZ_C128
        n = self.N[level]
        nrhs = _nrhs(x, n, "x")
        _check_field(x, x.dtype, n * nrhs, "x")
        _check_field(g, x.dtype, n * nrhs, "g")
        r = torch.empty_like(x) if out is None else out
        _check_field(r, x.dtype, n * nrhs, "out")
        n2 = torch.empty(nrhs, dtype=torch.float64, device=x.device) if norm2_out is None else norm2_out
        if not (isinstance(n2, torch.Tensor) and n2.is_cuda and n2.dtype == torch.float64 and n2.is_contiguous()
                and n2.numel() >= nrhs):
            raise ValueError(f"norm2_out: need a contiguous CUDA float64 tensor with at least {nrhs} elements")
        self._ok(self._lib.iofd_residual_static(self._h, level, op, prec, ctypes.c_void_p(g.data_ptr()),
                                                ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(r.data_ptr()),
                                                ctypes.c_void_p(n2.data_ptr()), nrhs, _stream_ptr(stream)))
        return r, n2

    # -- threegrid_precond ---------------------------------------------------
    def threegrid_precond(self, r, adjoint=False, out=None, stream=None):
        import torch
        prec = HZ_C64 if r.dtype == torch.complex64 else HZ_C128
        n = self.N[0]
        nrhs = _nrhs(r, n, "r")
        _check_field(r, r.dtype, n * nrhs, "r")
        z = torch.empty_like(r) if out is None else out
        self._ok(self._lib.threegrid_precond(self._h, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                             nrhs, 1 if adjoint else 0, prec, _stream_ptr(stream)))
        return z

    # -- helmholtz_solve -----------------------------------------------------
    @staticmethod
    def _sources(sources):
        arr = (HzSource * len(sources))()
        for i, (ix, iy, iz, amp) in enumerate(sources):
            amp = complex(amp)
            arr[i] = HzSource(int(ix), int(iy), int(iz), amp.real, amp.imag)
        return arr

    def helmholtz_solve(self, sources, want_u=True, v_out=None, u_out=None, allow_noconv=False):
        import torch
        ns = len(sources)
        n = self.N[0]
        v = v_out if v_out is not None else torch.empty((ns,) + self.shape, dtype=torch.complex128, device="cuda")
        u = (u_out if u_out is not None else torch.empty_like(v)) if want_u else None
        _check_field(v, torch.complex128, n * ns, "v_out")
        stats = HzStats()
        st = self._lib.helmholtz_solve(self._h, self._sources(sources), ns, ctypes.c_void_p(v.data_ptr()),
                                       ctypes.c_void_p(u.data_ptr()) if want_u else None, ctypes.byref(stats))
        if not (st == HZ_ENOCONV and allow_noconv):
            self._ok(st)
        return v, u, stats.as_dict()

    # -- helmholtz_adjoint_grad ----------------------------------------------
    def helmholtz_adjoint_grad(self, sources, receivers, d_obs, grad_out=None):
        import torch
        rec = np.ascontiguousarray(np.asarray(receivers, dtype=np.int32).reshape(-1, 3))
        d = np.ascontiguousarray(np.asarray(d_obs, dtype=np.complex128).reshape(len(sources), rec.shape[0]))
        dv = d.view(np.float64)
        g = grad_out if grad_out is not None else torch.empty(self.shape, dtype=torch.float64, device="cuda")
        J = ctypes.c_double()
        stats = HzStats()
        self._ok(self._lib.helmholtz_adjoint_grad(
            self._h, self._sources(sources), len(sources), rec.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
            rec.shape[0], dv.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(J),
            ctypes.c_void_p(g.data_ptr()), ctypes.byref(stats)))
        return J.value, g, stats.as_dict()


def kernel_launches() -> int:
    """Kernels launched by libhz.so so far in this process."""
    return int(load_library().hz_kernel_launches())


def workspace_bytes(n, n_pml, h, omega, params=None, max_nrhs=1, gamma_max=1.119058) -> int:
    lib = load_library()
    nx, ny, nz = (n, n, n) if np.isscalar(n) else n
    g = HzGrid(nx, ny, nz, n_pml, h, omega, gamma_max)
    p = params or default_params()
    out = ctypes.c_size_t()
    st = lib.hz_workspace_bytes(ctypes.byref(g), ctypes.byref(p), max_nrhs, ctypes.byref(out))
    if st != HZ_OK:
        raise HzError(st, lib.hz_last_error(None).decode())
    return out.value


def layout_check(n, n_pml, level=0, op=HZ_OP_A, nrhs=1, zblock=0, zblock_f=0, gamma_max=1.119058):
    """hz_layout_check: per-node write counts (right-hand side 0, shape
    (nz+1, ny+1, nx+1) of the level), blocks per right-hand side and the number
    of layout violations of one forward stencil application.  Host only."""
    lib = load_library()
    nx, ny, nz = (n, n, n) if np.isscalar(n) else n
    g = HzGrid(nx, ny, nz, n_pml, 1.0, 1.0, gamma_max)
    f = 1 << level
    counts = np.zeros((nz // f + 1, ny // f + 1, nx // f + 1), dtype=np.uint8)
    blocks, bad = ctypes.c_longlong(), ctypes.c_longlong()
    st = lib.hz_layout_check(ctypes.byref(g), level, op, nrhs, zblock, zblock_f,
                             counts.ctypes.data_as(ctypes.c_void_p), ctypes.byref(blocks), ctypes.byref(bad))
    if st != HZ_OK:
        raise HzError(st, lib.hz_last_error(None).decode())
    return counts, blocks.value, bad.value
