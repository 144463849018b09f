"""Thin Python binding of libvlasov's C ABI (include/vlasov.h).

Argument marshalling only: every step of the hot path runs in the library's CUDA
kernels.  PyTorch provides device memory and streams.  There is no CPU fallback:
if the compiled library is missing, loading raises.

Low level: ``vlasov_init``, ``vlasov_sweep``, ``vlasov_moment``, ``vlasov_poisson``,
``vlasov_step``, ``vlasov_status``, ``vlasov_last_error``, ``vlasov_destroy`` with the
C names and raw pointers.  High level: :class:`Vlasov`, a context bound to one 6D
torch tensor.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

F64, F32, BF16, F16 = 0, 1, 2, 3
AXES = {"x": 0, "y": 1, "z": 2, "ux": 3, "uy": 4, "uz": 5}

OK, EINVAL, ECFL, ECUDA, ENAN, ETIMEOUT, ENOMEM = 0, -1, -2, -3, -4, -5, -6
_NAMES = {EINVAL: "EINVAL", ECFL: "ECFL", ECUDA: "ECUDA", ENAN: "ENAN", ETIMEOUT: "ETIMEOUT",
          ENOMEM: "ENOMEM"}


class VlasovError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (_NAMES.get(code, "E?"), code, msg))
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("nux", ctypes.c_int), ("nuy", ctypes.c_int), ("nuz", ctypes.c_int),
                ("L", ctypes.c_double), ("V", ctypes.c_double), ("dtype", ctypes.c_int)]


_VP = ctypes.c_void_p
_lib = None

SYMBOLS = ("vlasov_init", "vlasov_destroy", "vlasov_set_stream", "vlasov_sweep", "vlasov_moment",
           "vlasov_poisson", "vlasov_step", "vlasov_upload", "vlasov_download",
           "vlasov_enable_timers", "vlasov_read_timers", "vlasov_status", "vlasov_last_error",
           "vlasov_sweep_velocity_static", "vlasov_set_f", "vlasov_sweep_adjoint",
           "vlasov_step_adjoint", "vlasov_step_record", "vlasov_step_adjoint_recorded",
           "vlasov_moment_adjoint", "vlasov_set_fused_kick", "vlasov_moments",
           "vlasov_step_record_sc", "vlasov_step_adjoint_recorded_sc", "vlasov_set_adjoint_arrays",
           "vlasov_set_fused_moment", "vlasov_kick", "vlasov_step_host", "vlasov_encode", "vlasov_decode",
           "vlasov_set_position_tiles", "vlasov_host_wait", "vlasov_selftest_wait")

# spatial cells the allocation-free velocity sweep can hold (its static scratch)
STATIC_MAX_CELLS = 32768

# timer kinds of vlasov_read_timers
T_KINDS = ("sweep_x", "sweep_y", "sweep_z", "sweep_ux", "sweep_uy", "sweep_uz", "moment",
           "poisson", "coef", "mass", "adj_x", "adj_y", "adj_z", "adj_ux", "adj_uy", "adj_uz",
           "grad_adj", "moment_adj", "sweep_uyuz", "moments", "kick")


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libvlasov.so (raises OSError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError("libvlasov.so is not built (run __graft_entry__.build())")
        _build.build()
    L = ctypes.CDLL(path)
    L.vlasov_init.argtypes = [ctypes.POINTER(_VP), ctypes.POINTER(Grid), _VP, _VP, _VP]
    L.vlasov_init.restype = ctypes.c_int
    L.vlasov_destroy.argtypes = [_VP]
    L.vlasov_destroy.restype = None
    L.vlasov_set_stream.argtypes = [_VP, _VP]
    L.vlasov_set_stream.restype = ctypes.c_int
    L.vlasov_sweep.argtypes = [_VP, ctypes.c_int, ctypes.c_double, ctypes.c_double, _VP]
    L.vlasov_sweep.restype = ctypes.c_int
    L.vlasov_moment.argtypes = [_VP, _VP, ctypes.POINTER(ctypes.c_double)]
    L.vlasov_moment.restype = ctypes.c_int
    L.vlasov_poisson.argtypes = [_VP, _VP, _VP, ctypes.c_double, ctypes.c_double, _VP]
    L.vlasov_poisson.restype = ctypes.c_int
    L.vlasov_step.argtypes = [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_double, _VP, _VP,
                              ctypes.c_double, _VP, _VP]
    L.vlasov_step.restype = ctypes.c_int
    L.vlasov_upload.argtypes = [_VP, _VP]
    L.vlasov_upload.restype = ctypes.c_int
    L.vlasov_download.argtypes = [_VP, _VP]
    L.vlasov_download.restype = ctypes.c_int
    L.vlasov_enable_timers.argtypes = [_VP, ctypes.c_int]
    L.vlasov_enable_timers.restype = ctypes.c_int
    L.vlasov_read_timers.argtypes = [_VP, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_longlong), ctypes.c_int]
    L.vlasov_read_timers.restype = ctypes.c_int
    L.vlasov_status.argtypes = [_VP]
    L.vlasov_status.restype = ctypes.c_int
    L.vlasov_sweep_velocity_static.argtypes = [ctypes.POINTER(Grid), _VP, ctypes.c_int,
                                               ctypes.c_double, _VP, _VP, _VP]
    L.vlasov_sweep_velocity_static.restype = ctypes.c_int
    L.vlasov_set_f.argtypes = [_VP, _VP, _VP]
    L.vlasov_set_f.restype = ctypes.c_int
    L.vlasov_sweep_adjoint.argtypes = [_VP, _VP, _VP, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, _VP, _VP]
    L.vlasov_sweep_adjoint.restype = ctypes.c_int
    L.vlasov_step_adjoint.argtypes = [_VP, _VP, _VP, ctypes.c_double, ctypes.c_double, _VP, _VP]
    L.vlasov_step_adjoint.restype = ctypes.c_int
    L.vlasov_step_record.argtypes = [_VP, _VP, _VP, _VP, ctypes.c_double, ctypes.c_double, _VP]
    L.vlasov_step_record.restype = ctypes.c_int
    L.vlasov_step_adjoint_recorded.argtypes = [_VP, _VP, _VP, _VP, ctypes.c_double, ctypes.c_double,
                                               _VP, _VP]
    L.vlasov_step_adjoint_recorded.restype = ctypes.c_int
    L.vlasov_moment_adjoint.argtypes = [_VP, _VP, _VP, ctypes.c_int]
    L.vlasov_moment_adjoint.restype = ctypes.c_int
    L.vlasov_step_record_sc.argtypes = [_VP, _VP, _VP, _VP, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        _VP, _VP, ctypes.c_double, _VP, _VP]
    L.vlasov_step_record_sc.restype = ctypes.c_int
    L.vlasov_step_adjoint_recorded_sc.argtypes = [_VP, _VP, _VP, _VP, ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_double, _VP, _VP, ctypes.c_double, _VP, _VP, _VP]
    L.vlasov_step_adjoint_recorded_sc.restype = ctypes.c_int
    L.vlasov_set_adjoint_arrays.argtypes = [_VP, ctypes.c_int]
    L.vlasov_set_adjoint_arrays.restype = ctypes.c_int
    L.vlasov_moments.argtypes = [_VP, _VP, _VP, _VP]
    L.vlasov_moments.restype = ctypes.c_int
    L.vlasov_set_fused_kick.argtypes = [_VP, ctypes.c_int]
    L.vlasov_set_fused_kick.restype = ctypes.c_int
    L.vlasov_set_position_tiles.argtypes = [_VP, ctypes.c_int]
    L.vlasov_set_position_tiles.restype = ctypes.c_int
    L.vlasov_set_fused_moment.argtypes = [_VP, ctypes.c_int]
    L.vlasov_set_fused_moment.restype = ctypes.c_int
    L.vlasov_kick.argtypes = [_VP, ctypes.c_double, _VP]
    L.vlasov_kick.restype = ctypes.c_int
    L.vlasov_step_host.argtypes = [_VP, _VP, ctypes.c_double, ctypes.c_double, ctypes.c_double, _VP, _VP,
                                   ctypes.c_double, _VP, _VP]
    L.vlasov_step_host.restype = ctypes.c_int
    L.vlasov_host_wait.argtypes = [_VP]
    L.vlasov_host_wait.restype = ctypes.c_int
    L.vlasov_selftest_wait.argtypes = [_VP]
    L.vlasov_selftest_wait.restype = ctypes.c_int
    L.vlasov_encode.argtypes = [ctypes.c_longlong, ctypes.c_int, _VP, ctypes.c_int, _VP, ctypes.c_int, _VP, _VP]
    L.vlasov_encode.restype = ctypes.c_int
    L.vlasov_decode.argtypes = [ctypes.c_longlong, ctypes.c_int, _VP, ctypes.c_int, _VP, _VP, ctypes.c_int, _VP]
    L.vlasov_decode.restype = ctypes.c_int
    L.vlasov_last_error.argtypes = [_VP]
    L.vlasov_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


# ---------------------------------------------------------------------------
# C names, raw pointers (ints or None)
# ---------------------------------------------------------------------------

def vlasov_last_error(ctx) -> str:
    return load().vlasov_last_error(ctx).decode(errors="replace")


def _check(ctx, rc):
    if rc != OK:
        raise VlasovError(rc, vlasov_last_error(ctx))
    return rc


def vlasov_init(grid: Grid, f_ptr: int, scale_ptr, stream: int):
    ctx = _VP()
    rc = load().vlasov_init(ctypes.byref(ctx), ctypes.byref(grid), f_ptr, scale_ptr, stream)
    _check(None, rc)
    return ctx.value


def vlasov_destroy(ctx) -> None:
    load().vlasov_destroy(ctx)


def vlasov_set_stream(ctx, stream: int):
    return _check(ctx, load().vlasov_set_stream(ctx, stream))


def vlasov_set_f(ctx, f_ptr: int, scale_ptr=None):
    return _check(ctx, load().vlasov_set_f(ctx, f_ptr, scale_ptr))


def vlasov_sweep_adjoint(ctx, f_in_ptr: int, lam_ptr: int, axis: int, dt: float, a: float,
                         phi_ptr, dLdg_ptr):
    return _check(ctx, load().vlasov_sweep_adjoint(ctx, f_in_ptr, lam_ptr, axis, dt, a, phi_ptr,
                                                   dLdg_ptr))


def vlasov_step_adjoint(ctx, f_n_ptr: int, lam_ptr: int, dt: float, a_half: float, phi_ptr,
                        dLdphi_ptr):
    return _check(ctx, load().vlasov_step_adjoint(ctx, f_n_ptr, lam_ptr, dt, a_half, phi_ptr,
                                                  dLdphi_ptr))


def _ptr_array(ptrs):
    arr = (_VP * len(ptrs))()
    for i, p in enumerate(ptrs):
        arr[i] = p
    return arr


def vlasov_step_record(ctx, f_n_ptr: int, rec_ptrs, f_next_ptr, dt: float, a_half: float, phi_ptr):
    """rec_ptrs: 8 device pointers (inputs of sweeps 1..8 of the step)."""
    return _check(ctx, load().vlasov_step_record(ctx, f_n_ptr, _ptr_array(rec_ptrs), f_next_ptr, dt,
                                                 a_half, phi_ptr))


def vlasov_step_adjoint_recorded(ctx, f_n_ptr: int, rec_ptrs, lam_ptr: int, dt: float, a_half: float,
                                 phi_ptr, dLdphi_ptr):
    return _check(ctx, load().vlasov_step_adjoint_recorded(ctx, f_n_ptr, _ptr_array(rec_ptrs), lam_ptr,
                                                           dt, a_half, phi_ptr, dLdphi_ptr))


def vlasov_step_record_sc(ctx, f_n_ptr, rec_ptrs, f_next_ptr, dt, a_half, a_full, phi_n_ptr, rho_bg_ptr,
                          four_pi_G, phi_next_ptr, rho_nu_ptr):
    return _check(ctx, load().vlasov_step_record_sc(ctx, f_n_ptr, _ptr_array(rec_ptrs), f_next_ptr, dt, a_half,
                                                    a_full, phi_n_ptr, rho_bg_ptr, four_pi_G, phi_next_ptr,
                                                    rho_nu_ptr))


def vlasov_step_adjoint_recorded_sc(ctx, f_n_ptr, rec_ptrs, lam_ptr, dt, a_half, a_full, phi_n_ptr, phi_next_ptr,
                                    four_pi_G, lam_phi_next_ptr, dLdphi_n_ptr, dLdrho_bg_ptr):
    return _check(ctx, load().vlasov_step_adjoint_recorded_sc(ctx, f_n_ptr, _ptr_array(rec_ptrs), lam_ptr, dt,
                                                              a_half, a_full, phi_n_ptr, phi_next_ptr, four_pi_G,
                                                              lam_phi_next_ptr, dLdphi_n_ptr, dLdrho_bg_ptr))


def vlasov_moment_adjoint(ctx, dLdrho_ptr: int, lam_ptr: int, accumulate: bool = False):
    return _check(ctx, load().vlasov_moment_adjoint(ctx, dLdrho_ptr, lam_ptr, int(bool(accumulate))))


def vlasov_set_fused_kick(ctx, mode: int):
    return _check(ctx, load().vlasov_set_fused_kick(ctx, int(mode)))


def vlasov_set_fused_moment(ctx, on: bool):
    return _check(ctx, load().vlasov_set_fused_moment(ctx, int(bool(on))))


def vlasov_sweep(ctx, axis: int, dt: float, a: float, phi_ptr):
    return _check(ctx, load().vlasov_sweep(ctx, axis, dt, a, phi_ptr))


def vlasov_moment(ctx, rho_ptr: int, want_mass: bool = False):
    m = ctypes.c_double(0.0)
    _check(ctx, load().vlasov_moment(ctx, rho_ptr, ctypes.byref(m) if want_mass else None))
    return m.value if want_mass else None


def vlasov_moments(ctx, rho_ptr, umean_ptr, sigma2_ptr):
    return _check(ctx, load().vlasov_moments(ctx, rho_ptr, umean_ptr, sigma2_ptr))


def vlasov_poisson(ctx, rho_ptr, rho_bg_ptr, a: float, four_pi_G: float, phi_ptr):
    return _check(ctx, load().vlasov_poisson(ctx, rho_ptr, rho_bg_ptr, a, four_pi_G, phi_ptr))


def vlasov_step(ctx, dt, a_half, a_full, phi_n_ptr, rho_bg_ptr, four_pi_G, phi_next_ptr,
                rho_nu_ptr):
    return _check(ctx, load().vlasov_step(ctx, dt, a_half, a_full, phi_n_ptr, rho_bg_ptr,
                                          four_pi_G, phi_next_ptr, rho_nu_ptr))


def vlasov_upload(ctx, f_host_ptr: int):
    return _check(ctx, load().vlasov_upload(ctx, f_host_ptr))


def vlasov_download(ctx, f_host_ptr: int):
    return _check(ctx, load().vlasov_download(ctx, f_host_ptr))


def vlasov_enable_timers(ctx, on: bool):
    return _check(ctx, load().vlasov_enable_timers(ctx, int(bool(on))))


def vlasov_read_timers(ctx):
    """Return ({kind: ms}, {kind: launches}) accumulated since the last read."""
    n = len(T_KINDS)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_longlong * n)()
    _check(ctx, load().vlasov_read_timers(ctx, ms, cnt, n))
    return dict(zip(T_KINDS, list(ms))), dict(zip(T_KINDS, list(cnt)))


def vlasov_status(ctx):
    return _check(ctx, load().vlasov_status(ctx))


def vlasov_sweep_velocity_static(grid: Grid, f_ptr: int, axis: int, dt: float, phi_ptr: int,
                                 status_ptr, stream: int):
    """Velocity sweep that allocates nothing (no context; static device scratch).

    For callers that cannot allocate device memory after start-up.  Calls that may
    overlap on the GPU share the scratch and must be serialised by the caller."""
    rc = load().vlasov_sweep_velocity_static(ctypes.byref(grid), f_ptr, axis, dt, phi_ptr,
                                             status_ptr, stream)
    return _check(None, rc)


# ---------------------------------------------------------------------------
# context bound to a torch tensor
# ---------------------------------------------------------------------------

def _ptr(t):
    return None if t is None else t.data_ptr()


def vlasov_encode(nlines: int, nuz: int, src_ptr, src_dtype: int, codes_ptr, code_dtype: int, scale_ptr,
                  stream: int):
    return _check(None, load().vlasov_encode(nlines, nuz, src_ptr, src_dtype, codes_ptr, code_dtype, scale_ptr,
                                             stream))


def vlasov_decode(nlines: int, nuz: int, codes_ptr, code_dtype: int, scale_ptr, dst_ptr, dst_dtype: int,
                  stream: int):
    return _check(None, load().vlasov_decode(nlines, nuz, codes_ptr, code_dtype, scale_ptr, dst_ptr, dst_dtype,
                                             stream))


def _dtype_codes():
    import torch
    return {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16}


def encode_lines(f, dtype, codes=None, scale=None):
    """16-bit storage of the CUDA tensor f (FP64 or FP32, contiguous, last axis = the u_z
    line) through vlasov_encode: returns (codes of `dtype`, torch.bfloat16 or
    torch.float16, shaped like f; scale, float32, f.shape[:-1]).  codes / scale may be
    given to be filled in place."""
    import torch
    kinds = _dtype_codes()
    if not f.is_cuda or not f.is_contiguous() or kinds.get(f.dtype) not in (F64, F32):
        raise ValueError("f must be a contiguous float64 or float32 CUDA tensor")
    if kinds.get(dtype) not in (BF16, F16):
        raise ValueError("dtype must be torch.bfloat16 or torch.float16")
    if codes is None:
        codes = torch.empty(f.shape, dtype=dtype, device=f.device)
    if scale is None:
        scale = torch.empty(f.shape[:-1], dtype=torch.float32, device=f.device)
    if codes.dtype != dtype or tuple(codes.shape) != tuple(f.shape) or not codes.is_contiguous() or \
            scale.dtype != torch.float32 or tuple(scale.shape) != tuple(f.shape[:-1]) or not scale.is_contiguous():
        raise ValueError("codes / scale do not match f")
    nuz = f.shape[-1]
    with torch.cuda.device(f.device):
        vlasov_encode(f.numel() // nuz, nuz, f.data_ptr(), kinds[f.dtype], codes.data_ptr(), kinds[dtype],
                      scale.data_ptr(), torch.cuda.current_stream(f.device).cuda_stream)
    return codes, scale


def decode_lines(codes, scale, dtype=None):
    """Values held by a 16-bit codec array (code x scale, through vlasov_decode): a CUDA
    tensor of `dtype` (torch.float64, exact, by default; or torch.float32)."""
    import torch
    kinds = _dtype_codes()
    dtype = torch.float64 if dtype is None else dtype
    if not codes.is_cuda or not codes.is_contiguous() or kinds.get(codes.dtype) not in (BF16, F16):
        raise ValueError("codes must be a contiguous bfloat16 or float16 CUDA tensor")
    if scale.dtype != torch.float32 or tuple(scale.shape) != tuple(codes.shape[:-1]) or not scale.is_contiguous():
        raise ValueError("scale must be a contiguous float32 tensor of shape codes.shape[:-1]")
    if kinds.get(dtype) not in (F64, F32):
        raise ValueError("dtype must be torch.float64 or torch.float32")
    out = torch.empty(codes.shape, dtype=dtype, device=codes.device)
    nuz = codes.shape[-1]
    with torch.cuda.device(codes.device):
        vlasov_decode(codes.numel() // nuz, nuz, codes.data_ptr(), kinds[codes.dtype], scale.data_ptr(),
                      out.data_ptr(), kinds[dtype], torch.cuda.current_stream(codes.device).cuda_stream)
    return out


class Vlasov:
    """A libvlasov context over the 6D CUDA tensor ``f`` [nx,ny,nz,nux,nuy,nuz].

    The tensor is updated in place by every sweep; the context keeps a reference.
    Work is queued on the torch stream current at each call.
    """

    def __init__(self, f, L: float = 1.0, V: float = 5.0, scale=None):
        import torch
        if not f.is_cuda or f.dim() != 6 or not f.is_contiguous():
            raise ValueError("f must be a contiguous 6D CUDA tensor")
        dt = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16,
              torch.float16: F16}.get(f.dtype)
        if dt is None:
            raise ValueError("f must be float64, float32, bfloat16 or float16")
        if dt in (BF16, F16):
            if scale is None or scale.dtype != torch.float32 or not scale.is_cuda or \
                    not scale.is_contiguous() or tuple(scale.shape) != tuple(f.shape[:5]):
                raise ValueError("16-bit f needs a contiguous float32 CUDA scale of shape f.shape[:5]")
        elif scale is not None:
            raise ValueError("scale is only used with 16-bit f")
        self.f = f
        self.scale = scale
        self.torch = torch
        g = Grid()
        g.nx, g.ny, g.nz, g.nux, g.nuy, g.nuz = f.shape
        g.L, g.V, g.dtype = L, V, dt
        self.grid = g
        self.shape = tuple(f.shape)
        with torch.cuda.device(f.device):
            self._stream = torch.cuda.current_stream(f.device).cuda_stream
            self.ctx = vlasov_init(g, f.data_ptr(), None if scale is None else scale.data_ptr(),
                                   self._stream)

    # keep the context on the caller's current stream
    def _sync_stream(self):
        s = self.torch.cuda.current_stream(self.f.device).cuda_stream
        if s != self._stream:
            vlasov_set_stream(self.ctx, s)
            self._stream = s

    def _field(self, t, dtype):
        if t is None:
            return None
        if not t.is_cuda or not t.is_contiguous() or t.dtype != dtype or \
                tuple(t.shape) != self.shape[:3]:
            raise ValueError("spatial field must be a contiguous %s CUDA tensor of shape %s"
                             % (dtype, self.shape[:3]))
        return t

    def sweep(self, axis, dt: float, a: float = 1.0, phi=None):
        ax = AXES[axis] if isinstance(axis, str) else int(axis)
        self._sync_stream()
        phi = self._field(phi, self.torch.float32)
        vlasov_sweep(self.ctx, ax, dt, a, _ptr(phi))

    def kick(self, dt: float, phi):
        """D_uz D_uy D_ux (dt) with the acceleration -grad phi (one kick of Eq. 5)."""
        self._sync_stream()
        phi = self._field(phi, self.torch.float32)
        _check(self.ctx, load().vlasov_kick(self.ctx, dt, _ptr(phi)))

    def moment(self, rho=None, mass: bool = False):
        self._sync_stream()
        if rho is None:
            rho = self.torch.empty(self.shape[:3], dtype=self.torch.float64, device=self.f.device)
        self._field(rho, self.torch.float64)
        m = vlasov_moment(self.ctx, rho.data_ptr(), mass)
        return (rho, m) if mass else rho

    def moments(self):
        """(rho [nx,ny,nz], umean [3,nx,ny,nz], sigma2 [6,nx,ny,nz]) in FP64: density, mean
        velocity and velocity dispersion tensor (xx, yy, zz, xy, xz, yz)."""
        self._sync_stream()
        n = self.shape[:3]
        T = self.torch
        rho = T.empty(n, dtype=T.float64, device=self.f.device)
        um = T.empty((3,) + n, dtype=T.float64, device=self.f.device)
        s2 = T.empty((6,) + n, dtype=T.float64, device=self.f.device)
        vlasov_moments(self.ctx, rho.data_ptr(), um.data_ptr(), s2.data_ptr())
        return rho, um, s2

    def poisson(self, rho, a: float, four_pi_G: float = 1.0, rho_bg=None, phi=None):
        self._sync_stream()
        if phi is None:
            phi = self.torch.empty(self.shape[:3], dtype=self.torch.float32, device=self.f.device)
        vlasov_poisson(self.ctx, _ptr(self._field(rho, self.torch.float64)),
                       _ptr(self._field(rho_bg, self.torch.float64)), a, four_pi_G,
                       _ptr(self._field(phi, self.torch.float32)))
        return phi

    def step(self, dt: float, a_half: float, a_full: float, phi_n, rho_bg=None,
             four_pi_G: float = 1.0, phi_next=None, rho_nu=None):
        self._sync_stream()
        vlasov_step(self.ctx, dt, a_half, a_full, _ptr(self._field(phi_n, self.torch.float32)),
                    _ptr(self._field(rho_bg, self.torch.float64)), four_pi_G,
                    _ptr(self._field(phi_next, self.torch.float32)),
                    _ptr(self._field(rho_nu, self.torch.float64)))

    def _like_f(self, t, name):
        if not t.is_cuda or tuple(t.shape) != self.shape or t.dtype != self.f.dtype or \
                not t.is_contiguous() or t.device != self.f.device:
            raise ValueError("%s must be a contiguous CUDA tensor like f" % name)
        return t

    def sweep_adjoint(self, f_in, lam, axis, dt: float, a: float = 1.0, phi=None, dLdg=None):
        """lam <- (dD_axis/df at f_in)^T lam in place; for a velocity axis dL/dg is
        added to dLdg (FP64 spatial field) when given."""
        ax = AXES[axis] if isinstance(axis, str) else int(axis)
        self._sync_stream()
        vlasov_sweep_adjoint(self.ctx, self._like_f(f_in, "f_in").data_ptr(),
                             self._like_f(lam, "lam").data_ptr(), ax, dt, a,
                             _ptr(self._field(phi, self.torch.float32)),
                             _ptr(self._field(dLdg, self.torch.float64)))

    def step_adjoint(self, f_n, lam, dt: float, a_half: float, phi, dLdphi=None):
        """lam <- (d step/df at f_n)^T lam in place (external potential phi for both
        kicks); dL/dphi is added to dLdphi (FP64 spatial field) when given."""
        self._sync_stream()
        vlasov_step_adjoint(self.ctx, self._like_f(f_n, "f_n").data_ptr(),
                            self._like_f(lam, "lam").data_ptr(), dt, a_half,
                            _ptr(self._field(phi, self.torch.float32)),
                            _ptr(self._field(dLdphi, self.torch.float64)))

    def step_record(self, f_n, rec, dt: float, a_half: float, phi, f_next=None):
        """Run one external-potential step from f_n out of place, keeping the input of
        every sweep: rec is a list of 8 tensors like f; f_next (optional) receives
        the result."""
        if len(rec) != 8:
            raise ValueError("rec must hold 8 tensors")
        self._sync_stream()
        vlasov_step_record(self.ctx, self._like_f(f_n, "f_n").data_ptr(),
                           [self._like_f(r, "rec").data_ptr() for r in rec],
                           None if f_next is None else self._like_f(f_next, "f_next").data_ptr(),
                           dt, a_half, _ptr(self._field(phi, self.torch.float32)))

    def step_adjoint_recorded(self, f_n, rec, lam, dt: float, a_half: float, phi, dLdphi=None):
        """lam <- (d step/df at f_n)^T lam from the sweep inputs step_record kept."""
        if len(rec) != 8:
            raise ValueError("rec must hold 8 tensors")
        self._sync_stream()
        vlasov_step_adjoint_recorded(self.ctx, self._like_f(f_n, "f_n").data_ptr(),
                                     [self._like_f(r, "rec").data_ptr() for r in rec],
                                     self._like_f(lam, "lam").data_ptr(), dt, a_half,
                                     _ptr(self._field(phi, self.torch.float32)),
                                     _ptr(self._field(dLdphi, self.torch.float64)))

    def step_record_sc(self, f_n, rec, dt: float, a_half: float, a_full: float, phi_n, phi_next,
                       rho_bg=None, four_pi_G: float = 1.0, f_next=None, rho_nu=None):
        """Self-consistent step from (f_n, phi_n) out of place, keeping every sweep's input
        in rec (8 tensors like f); phi_next (FP32) receives phi^{n+1}."""
        if len(rec) != 8:
            raise ValueError("rec must hold 8 tensors")
        self._sync_stream()
        T = self.torch
        vlasov_step_record_sc(self.ctx, self._like_f(f_n, "f_n").data_ptr(),
                              [self._like_f(r, "rec").data_ptr() for r in rec],
                              None if f_next is None else self._like_f(f_next, "f_next").data_ptr(), dt, a_half,
                              a_full, _ptr(self._field(phi_n, T.float32)), _ptr(self._field(rho_bg, T.float64)),
                              four_pi_G, _ptr(self._field(phi_next, T.float32)), _ptr(self._field(rho_nu, T.float64)))

    def step_adjoint_recorded_sc(self, f_n, rec, lam, dt: float, a_half: float, a_full: float, phi_n, phi_next,
                                 four_pi_G: float = 1.0, lam_phi_next=None, dLdphi_n=None, dLdrho_bg=None):
        """Adjoint of one self-consistent step from step_record_sc's records: lam <- dL/df^n;
        dL/dphi_n and dL/drho_bg are added to dLdphi_n / dLdrho_bg (FP64) when given."""
        if len(rec) != 8:
            raise ValueError("rec must hold 8 tensors")
        self._sync_stream()
        T = self.torch
        vlasov_step_adjoint_recorded_sc(self.ctx, self._like_f(f_n, "f_n").data_ptr(),
                                        [self._like_f(r, "rec").data_ptr() for r in rec],
                                        self._like_f(lam, "lam").data_ptr(), dt, a_half, a_full,
                                        _ptr(self._field(phi_n, T.float32)), _ptr(self._field(phi_next, T.float32)),
                                        four_pi_G, _ptr(self._field(lam_phi_next, T.float64)),
                                        _ptr(self._field(dLdphi_n, T.float64)),
                                        _ptr(self._field(dLdrho_bg, T.float64)))

    def moment_adjoint(self, dLdrho, lam, accumulate: bool = False):
        """lam (+)= du^3 dL/drho(x) broadcast over each velocity cube."""
        self._sync_stream()
        vlasov_moment_adjoint(self.ctx, self._field(dLdrho, self.torch.float64).data_ptr(),
                              self._like_f(lam, "lam").data_ptr(), accumulate)

    def upload(self, f_host):
        """Copy a host tensor (same shape and dtype as f, ideally pinned) into f."""
        if f_host.is_cuda or tuple(f_host.shape) != self.shape or f_host.dtype != self.f.dtype \
                or not f_host.is_contiguous():
            raise ValueError("f_host must be a contiguous host tensor like f")
        self._sync_stream()
        vlasov_upload(self.ctx, f_host.data_ptr())

    def download(self, f_host):
        if f_host.is_cuda or tuple(f_host.shape) != self.shape or f_host.dtype != self.f.dtype \
                or not f_host.is_contiguous():
            raise ValueError("f_host must be a contiguous host tensor like f")
        self._sync_stream()
        vlasov_download(self.ctx, f_host.data_ptr())

    def step_host(self, f_host, dt: float, a_half: float, a_full: float, phi_n, rho_bg=None,
                  four_pi_G: float = 1.0, phi_next=None, rho_nu=None):
        """One Eq. (5) step of the host tensor f_host (like f, ideally pinned), in place:
        its x-slabs are copied in on a second stream and out on a third behind the
        cell-local sweeps.  The downloads may still run when the call returns: the next
        step_host overlaps its uploads with them; host_wait (or status) orders later work."""
        if f_host.is_cuda or tuple(f_host.shape) != self.shape or f_host.dtype != self.f.dtype \
                or not f_host.is_contiguous():
            raise ValueError("f_host must be a contiguous host tensor like f")
        self._sync_stream()
        _check(self.ctx, load().vlasov_step_host(
            self.ctx, f_host.data_ptr(), dt, a_half, a_full, _ptr(self._field(phi_n, self.torch.float32)),
            _ptr(self._field(rho_bg, self.torch.float64)), four_pi_G,
            _ptr(self._field(phi_next, self.torch.float32)), _ptr(self._field(rho_nu, self.torch.float64))))

    def host_wait(self):
        """Queue on the stream the wait for the downloads of the last step_host (they run on
        a stream of their own; the next step_host waits per slab, every other call waits for
        all of them first)."""
        self._sync_stream()
        _check(self.ctx, load().vlasov_host_wait(self.ctx))

    def selftest_wait(self):
        """Queue the failure-path self-test: a kernel whose bounded device wait runs out;
        the next status() raises ETIMEOUT and the context stays usable."""
        self._sync_stream()
        _check(self.ctx, load().vlasov_selftest_wait(self.ctx))

    def set_adjoint_arrays(self, arrays: int):
        """f-sized scratch arrays step_adjoint may hold: 8, 4 or 0 (8 if they fit, else 4)."""
        _check(self.ctx, load().vlasov_set_adjoint_arrays(self.ctx, int(arrays)))

    def set_fused_kick(self, mode=2):
        """How the kicks run: 2 (default) the whole kick in one pass over each velocity cube
        (n_ux = n_uy = n_uz = 16 or 32), 1 (or True) D_ux then D_uy D_uz in one pass, 0 (or
        False) three separate sweeps."""
        vlasov_set_fused_kick(self.ctx, int(mode))

    def set_position_tiles(self, on: bool = True):
        """Run the FP32 position sweeps on whole staged lines (the default) or streamed."""
        _check(self.ctx, load().vlasov_set_position_tiles(self.ctx, int(bool(on))))

    def set_fused_moment(self, on: bool = True):
        """Let the step's x sweep sum the moment of its output (FP32 / FP64 storage)."""
        vlasov_set_fused_moment(self.ctx, on)

    def enable_timers(self, on: bool = True):
        vlasov_enable_timers(self.ctx, on)

    def read_timers(self):
        return vlasov_read_timers(self.ctx)

    def status(self):
        return vlasov_status(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            vlasov_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
