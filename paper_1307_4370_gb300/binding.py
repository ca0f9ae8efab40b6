"""Thin Python binding of the C ABI in include/purify.h (argument marshalling only).

Every function here forwards to the CUDA library of the same name; tensors are
passed as device pointers (``data_ptr()``) together with the current torch CUDA
stream.  There is no fallback: if the library is missing or cannot be loaded,
``load()`` raises.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np
import torch

from . import build as _build

_LIB = None

PURIFY_OK = 0
PURIFY_E_CUDA = -5
STATUS_NAMES = {
    0: "PURIFY_OK", -1: "PURIFY_E_INVALID_ARG", -2: "PURIFY_E_SIZE", -3: "PURIFY_E_NOT_DEVICE_PTR",
    -4: "PURIFY_E_ALLOC", -5: "PURIFY_E_CUDA", -6: "PURIFY_E_TIMEOUT", -7: "PURIFY_E_UNSUPPORTED",
}
SARA_MASK = 0x1FF


class PurifyError(RuntimeError):
    """A negative status from the library."""

    def __init__(self, func: str, status: int):
        self.status = status
        msg = _LIB.purify_status_string(status).decode() if _LIB is not None else str(status)
        if _LIB is not None and status == PURIFY_E_CUDA:
            msg += ": " + _LIB.purify_last_error().decode()
        super().__init__(f"{func} failed: {STATUS_NAMES.get(status, status)} ({msg})")


class Desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("M", ctypes.c_int64), ("J", ctypes.c_int32),
                ("oversample", ctypes.c_int32), ("levels", ctypes.c_int32), ("bases_mask", ctypes.c_uint32),
                ("tile", ctypes.c_int32), ("kernel", ctypes.c_int32)]


KERNELS = {"kb": 0, "gauss": 1}  # purify_kernel: Kaiser-Bessel, the paper's Gaussian


class SdmmParams(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int32), ("cg_iters", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("beta", ctypes.c_double), ("xi", ctypes.c_double),
                ("tau", ctypes.c_double), ("use_graph", ctypes.c_int32)]


class Report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("f1", ctypes.c_double), ("zeta", ctypes.c_double),
                ("nu", ctypes.c_double), ("gamma", ctypes.c_double), ("cg_residual", ctypes.c_double),
                ("nu_min", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_SIGS = {
    "purify_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(Desc), _vp, _vp]),
    "purify_destroy": (None, [_vp]),
    "purify_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "purify_last_error": (ctypes.c_char_p, []),
    "purify_set_beam": (_i32, [_vp, _vp, _vp]),
    "purify_sdmm_set_blocks": (_i32, [_vp, _vp, _i32, _vp, _vp, _vp]),
    "purify_sdmm_set_prior": (_i32, [_vp, _vp, _i32, _i32]),
    "purify_prox_tv": (_i32, [_vp, _vp, _vp, ctypes.c_float, _i32, _vp, _vp]),
    "purify_l2_bound": (ctypes.c_int, [_i64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    "purify_sizes": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i32),
                                    ctypes.POINTER(_i64)]),
    "purify_phi": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "purify_phi_static": (ctypes.c_int, [_i32, _i32, _i64, _vp, _vp, _vp, _vp]),
    "purify_phi_adj": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "purify_sara_analysis": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "purify_sara_synthesis": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "purify_prox_l1_reweighted": (ctypes.c_int, [_vp, _i64, _vp, _vp, ctypes.c_float, _vp, _vp]),
    "purify_proj_l2ball": (ctypes.c_int, [_vp, _i64, _vp, _vp, ctypes.c_double, _vp, _vp, _vp]),
    "purify_proj_positive": (ctypes.c_int, [_vp, _i64, _vp, _vp, _vp]),
    "purify_cg_solve": (ctypes.c_int, [_vp, _vp, _vp, _i32, _vp, _vp]),
    "purify_sdmm_default_params": (None, [ctypes.POINTER(SdmmParams)]),
    "purify_sdmm_state_create": (ctypes.c_int, [_vp, ctypes.POINTER(_vp)]),
    "purify_sdmm_state_destroy": (None, [_vp]),
    "purify_sdmm_init": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.POINTER(SdmmParams), _vp]),
    "purify_sdmm_set_data": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "purify_sdmm_set_data_bf16": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "purify_sdmm_step": (ctypes.c_int, [_vp, _vp, _vp]),
    "purify_sdmm_reweight": (ctypes.c_int, [_vp, _vp, _i32, _vp]),
    "purify_sdmm_set_weights": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "purify_sdmm_get_image": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "purify_sdmm_get_report": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(Report), _vp]),
    "purify_sdmm_solve": (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.POINTER(SdmmParams), _vp,
                                         ctypes.POINTER(Report), _vp]),
    "purify_sdmm_state_bytes": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "purify_sdmm_export": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_size_t, _vp]),
    "purify_sdmm_import": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_size_t, _vp]),
    "purify_diff_penalty": (_i32, [_vp, _vp, _vp, ctypes.c_double, ctypes.POINTER(ctypes.c_double), _vp]),
    "purify_diff_tape_bytes": (_i32, [_vp, _i32, ctypes.POINTER(ctypes.c_size_t)]),
    "purify_diff_iteration": (_i32, [_vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_double, _i32,
                                     ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp, _vp]),
    "purify_diff_iteration_vjp": (_i32, [_vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_double, _i32,
                                         ctypes.POINTER(_vp), _vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                         _vp, _vp, _vp]),
    "purify_vjp_soft_threshold": (_i32, [_i64, _vp, _vp, ctypes.c_float, _vp, _vp, _vp, _vp]),
    "purify_vjp_l2ball": (_i32, [_vp, _i64, _vp, _vp, ctypes.c_double, _vp, _vp, _vp, _vp]),
    "purify_vjp_positive": (_i32, [_i64, _vp, _vp, _vp, _vp]),
    "purify_profile_enable": (ctypes.c_int, [_vp, ctypes.c_int]),
    "purify_profile_collect": (ctypes.c_int, [_vp, _i32, _vp, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(_i32)]),
    "purify_launch_count": (ctypes.c_uint64, []),
    "purify_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i32]),
    "purify_batch_step": (ctypes.c_int, [_vp, _i32, _vp]),
    "purify_batch_size": (ctypes.c_int, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "purify_batch_destroy": (None, [_vp]),
}


def library_path() -> str:
    return _build.LIB_PATH


def load(path: str | None = None) -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or library_path()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def declared_symbols() -> list[str]:
    return list(_SIGS)


def _check(func: str, status: int) -> None:
    if status != PURIFY_OK:
        raise PurifyError(func, status)


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return t.ctypes.data
    return int(t)


def _c64(t: torch.Tensor, n: int, what: str) -> torch.Tensor:
    if t.dtype != torch.complex64 or not t.is_cuda or t.numel() != n:
        raise ValueError(f"{what}: expected {n} complex64 values on a CUDA device, got "
                         f"{t.dtype} {tuple(t.shape)} on {t.device}")
    return t.contiguous()


def _f32(t: torch.Tensor, n: int, what: str) -> torch.Tensor:
    if t.dtype != torch.float32 or not t.is_cuda or t.numel() != n or not t.is_contiguous():
        raise ValueError(f"{what}: expected {n} contiguous float32 values on a CUDA device, got "
                         f"{t.dtype} {tuple(t.shape)} on {t.device}")
    return t


def _ptr_array(ts, sizes):
    """A C array of the device pointers of complex64 tensors of the given sizes."""
    if len(ts) != len(sizes):
        raise ValueError(f"expected {len(sizes)} arrays")
    arr = (ctypes.c_void_p * len(ts))()
    for i, (t, n) in enumerate(zip(ts, sizes)):
        if t.dtype != torch.complex64 or not t.is_cuda or t.numel() != n or not t.is_contiguous():
            raise ValueError(f"state array {i}: expected {n} contiguous complex64 values on a CUDA device")
        arr[i] = t.data_ptr()
    return arr


# ---------------------------------------------------------------------------
# Raw functions with the C names (pointer-level)
# ---------------------------------------------------------------------------
def purify_create(desc: Desc, uv_ptr: int, stream=None) -> int:
    lib = load()
    out = _vp()
    _check("purify_create", lib.purify_create(ctypes.byref(out), ctypes.byref(desc), uv_ptr, _stream(stream)))
    return out.value


def purify_destroy(ctx: int) -> None:
    load().purify_destroy(ctx)


class Context:
    """A measurement set-up (u-v coverage, image side, kernel, dictionary).

    Methods are named after the C entry points without the ``purify_`` prefix
    and take / return torch complex64 tensors on the context's device.
    """

    def __init__(self, n: int, uv, J: int = 6, levels: int = 4, bases_mask: int = SARA_MASK,
                 device=None, tile: int = 0, kernel: str = "kb"):
        self.lib = load()
        if device is not None:
            torch.cuda.set_device(device)
        self.device = torch.device("cuda", torch.cuda.current_device())
        uv_t = torch.as_tensor(uv, dtype=torch.float32)
        if uv_t.dim() != 2 or uv_t.shape[1] != 2:
            raise ValueError("uv must be (M, 2)")
        uv_t = uv_t.contiguous()
        self.M = int(uv_t.shape[0])
        self.n = int(n)
        self.J = int(J)
        self.levels = int(levels)
        self.bases_mask = int(bases_mask)
        self.q = bin(self.bases_mask & 0x1FF).count("1")
        self.N = self.n * self.n
        self.D = self.q * self.N
        self.tile = int(tile)
        if kernel not in KERNELS:
            raise ValueError(f"kernel must be one of {sorted(KERNELS)}")
        self.kernel = kernel
        desc = Desc(self.n, self.M, self.J, 2, self.levels, self.bases_mask, self.tile, KERNELS[kernel])
        uv_keep = uv_t if uv_t.is_cuda else uv_t.numpy()
        self.ctx = purify_create(desc, _ptr(uv_keep))

    def set_beam(self, beam=None, stream=None) -> None:
        """Primary beam B of Phi = G F D Z B: a real n x n map, or None for B = I."""
        if beam is None:
            _check("purify_set_beam", self.lib.purify_set_beam(self.ctx, None, _stream(stream)))
            return
        b = torch.as_tensor(beam, dtype=torch.float32)
        if tuple(b.shape) not in ((self.n, self.n), (self.N,)):
            raise ValueError("beam must be n x n")
        b = b.to(self.device).contiguous()
        _check("purify_set_beam", self.lib.purify_set_beam(self.ctx, _ptr(b), _stream(stream)))

    def close(self) -> None:
        if getattr(self, "ctx", None):
            purify_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _img(self, shape=None):
        return torch.empty(self.N if shape is None else shape, dtype=torch.complex64, device=self.device)

    # operators -----------------------------------------------------------
    def phi(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        x = _c64(x, self.N, "x")
        y = out if out is not None else torch.empty(self.M, dtype=torch.complex64, device=self.device)
        _check("purify_phi", self.lib.purify_phi(self.ctx, _ptr(x), _ptr(y), _stream(stream)))
        return y

    def phi_adj(self, y: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        y = _c64(y, self.M, "y")
        x = out if out is not None else self._img((self.n, self.n))
        _check("purify_phi_adj", self.lib.purify_phi_adj(self.ctx, _ptr(y), _ptr(x), _stream(stream)))
        return x

    def sara_analysis(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        x = _c64(x, self.N, "x")
        a = out if out is not None else self._img((self.q, self.n, self.n))
        _check("purify_sara_analysis", self.lib.purify_sara_analysis(self.ctx, _ptr(x), _ptr(a), _stream(stream)))
        return a

    def sara_synthesis(self, alpha: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        alpha = _c64(alpha, self.D, "alpha")
        x = out if out is not None else self._img((self.n, self.n))
        _check("purify_sara_synthesis",
               self.lib.purify_sara_synthesis(self.ctx, _ptr(alpha), _ptr(x), _stream(stream)))
        return x

    def prox_l1_reweighted(self, a: torch.Tensor, w: torch.Tensor | None, gamma: float,
                           out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        out = out if out is not None else torch.empty_like(a)
        if w is not None and (w.dtype != torch.float32 or w.numel() != a.numel()):
            raise ValueError("w: float32, one weight per entry")
        _check("purify_prox_l1_reweighted",
               self.lib.purify_prox_l1_reweighted(self.ctx, a.numel(), _ptr(a.contiguous()), _ptr(w),
                                                  float(gamma), _ptr(out), _stream(stream)))
        return out

    def prox_tv(self, x: torch.Tensor, w: torch.Tensor | None, lam: float, iters: int = 20,
                out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """prox of lam ||W grad .||_1 by `iters` FGP iterations (x: n x n complex64)."""
        x = x.contiguous()
        out = out if out is not None else torch.empty_like(x)
        if w is not None and (w.dtype != torch.float32 or w.numel() != self.N):
            raise ValueError("w: float32, one weight per pixel")
        _check("purify_prox_tv", self.lib.purify_prox_tv(self.ctx, _ptr(x), _ptr(w), float(lam), int(iters),
                                                         _ptr(out), _stream(stream)))
        return out

    def proj_l2ball(self, r: torch.Tensor, y: torch.Tensor, eps: float, out: torch.Tensor | None = None,
                    norm_out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        out = out if out is not None else torch.empty_like(r)
        _check("purify_proj_l2ball",
               self.lib.purify_proj_l2ball(self.ctx, r.numel(), _ptr(r.contiguous()), _ptr(y.contiguous()),
                                           float(eps), _ptr(out), _ptr(norm_out), _stream(stream)))
        return out

    def proj_positive(self, a: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        out = out if out is not None else torch.empty_like(a)
        _check("purify_proj_positive",
               self.lib.purify_proj_positive(self.ctx, a.numel(), _ptr(a.contiguous()), _ptr(out),
                                             _stream(stream)))
        return out

    def cg_solve(self, b: torch.Tensor, x0: torch.Tensor, iters: int, stream=None):
        """Returns (x, residual) after ``iters`` CG steps on (Phi^H Phi + 2I) x = b."""
        b = _c64(b, self.N, "b")
        x = _c64(x0, self.N, "x0").clone()
        res = torch.zeros(1, dtype=torch.float64, device=self.device)
        _check("purify_cg_solve",
               self.lib.purify_cg_solve(self.ctx, _ptr(b), _ptr(x), int(iters), _ptr(res), _stream(stream)))
        return x, res

    # kernel timing -------------------------------------------------------
    def profile_enable(self, on: bool = True) -> None:
        _check("purify_profile_enable", self.lib.purify_profile_enable(self.ctx, int(bool(on))))

    def profile_collect(self, max_entries: int = 64) -> list[tuple[str, int, float]]:
        """[(kernel, launches, total ms)] since the last collect (synchronises)."""
        names = ctypes.create_string_buffer(32 * max_entries)
        launches = (_i64 * max_entries)()
        ms = (ctypes.c_double * max_entries)()
        n = _i32()
        _check("purify_profile_collect",
               self.lib.purify_profile_collect(self.ctx, max_entries, names, launches, ms, ctypes.byref(n)))
        out = []
        for k in range(n.value):
            nm = names.raw[32 * k: 32 * (k + 1)].split(b"\0", 1)[0].decode()
            out.append((nm, int(launches[k]), float(ms[k])))
        return out

    # differentiation (reverse mode of one SDMM iteration) -----------------
    def diff_penalty(self, y: torch.Tensor, wvis: torch.Tensor, beta: float = 1e-3, stream=None) -> float:
        """purify_diff_penalty: gamma = beta ||Psi^H Phi_w^H y_w||_inf."""
        out = ctypes.c_double()
        _check("purify_diff_penalty", self.lib.purify_diff_penalty(
            self.ctx, _ptr(_c64(y, self.M, "y")), _ptr(_f32(wvis, self.M, "w")), float(beta), ctypes.byref(out),
            _stream(stream)))
        return out.value

    def diff_tape(self, cg_iters: int) -> torch.Tensor:
        """Device buffer for the tape of one differentiable iteration."""
        nb = ctypes.c_size_t()
        _check("purify_diff_tape_bytes", self.lib.purify_diff_tape_bytes(self.ctx, int(cg_iters), ctypes.byref(nb)))
        return torch.empty(nb.value, dtype=torch.uint8, device=self.device)

    def diff_state_shapes(self) -> list:
        """Sizes of the seven state arrays (x_hat, z1, z2, z3, x1, x2, x3)."""
        return [self.N, self.D, self.M, self.N, self.N, self.N, self.N]

    def diff_iteration(self, y, wvis, omega, gamma: float, eps: float, cg_iters: int, state_in, state_out, tape,
                       stream=None) -> None:
        """purify_diff_iteration: state_out = one SDMM iteration of state_in, tape filled."""
        sin = _ptr_array(state_in, self.diff_state_shapes())
        sout = _ptr_array(state_out, self.diff_state_shapes())
        _check("purify_diff_iteration", self.lib.purify_diff_iteration(
            self.ctx, _ptr(_c64(y, self.M, "y")), _ptr(_f32(wvis, self.M, "w")), _ptr(_f32(omega, self.D, "omega")),
            float(gamma), float(eps), int(cg_iters), sin, sout, _ptr(tape), _stream(stream)))

    def diff_iteration_vjp(self, y, wvis, omega, gamma: float, eps: float, cg_iters: int, state_in, tape,
                           bar_out, bar_in, wvis_bar, omega_bar, stream=None) -> None:
        """purify_diff_iteration_vjp: adjoints of the inputs from those of the outputs;
        adds to wvis_bar and omega_bar."""
        shapes = self.diff_state_shapes()
        _check("purify_diff_iteration_vjp", self.lib.purify_diff_iteration_vjp(
            self.ctx, _ptr(_c64(y, self.M, "y")), _ptr(_f32(wvis, self.M, "w")), _ptr(_f32(omega, self.D, "omega")),
            float(gamma), float(eps), int(cg_iters), _ptr_array(state_in, shapes), _ptr(tape),
            _ptr_array(bar_out, shapes), _ptr_array(bar_in, shapes), _ptr(_f32(wvis_bar, self.M, "w_bar")),
            _ptr(_f32(omega_bar, self.D, "omega_bar")), _stream(stream)))

    def vjp_l2ball(self, a: torch.Tensor, y: torch.Tensor, eps: float, rbar: torch.Tensor, stream=None):
        """purify_vjp_l2ball: (abar, ybar)."""
        n = a.numel()
        abar = torch.empty_like(a)
        ybar = torch.empty_like(a)
        _check("purify_vjp_l2ball", self.lib.purify_vjp_l2ball(
            self.ctx, n, _ptr(_c64(a, n, "a")), _ptr(_c64(y, n, "y")), float(eps), _ptr(_c64(rbar, n, "rbar")),
            _ptr(abar), _ptr(ybar), _stream(stream)))
        return abar, ybar

    # SDMM ----------------------------------------------------------------
    def sdmm_state(self) -> "SdmmState":
        return SdmmState(self)

    def sdmm_solve(self, y, eps: float, max_iters: int = 300, cg_iters: int = 10, rounds: int = 1,
                   check_every: int = 0, beta: float = 1e-3, xi: float = 1e-3, tau: float = 0.1,
                   out=None, stream=None):
        """Whole solve; y and out may be host (numpy / CPU tensor) or device tensors."""
        p = default_params()
        p.max_iters, p.cg_iters, p.rounds, p.check_every = max_iters, cg_iters, rounds, check_every
        p.beta, p.xi, p.tau = beta, xi, tau
        if out is None:
            out = self._img((self.n, self.n))
        rep = Report()
        _check("purify_sdmm_solve",
               self.lib.purify_sdmm_solve(self.ctx, _ptr(y), float(eps), ctypes.byref(p), _ptr(out),
                                          ctypes.byref(rep), _stream(stream)))
        return out, rep.as_dict()


def vjp_soft_threshold(a: torch.Tensor, w, gamma: float, rbar: torch.Tensor, wbar=None, stream=None):
    """purify_vjp_soft_threshold: abar (and wbar += gamma dL/dlam when given)."""
    lib = load()
    n = a.numel()
    abar = torch.empty_like(a)
    _check("purify_vjp_soft_threshold", lib.purify_vjp_soft_threshold(
        n, _ptr(_c64(a, n, "a")), _ptr(_f32(w, n, "w")) if w is not None else None, float(gamma),
        _ptr(_c64(rbar, n, "rbar")), _ptr(abar), _ptr(_f32(wbar, n, "wbar")) if wbar is not None else None,
        _stream(stream)))
    return abar


def vjp_positive(a: torch.Tensor, rbar: torch.Tensor, stream=None):
    """purify_vjp_positive: abar."""
    lib = load()
    n = a.numel()
    abar = torch.empty_like(a)
    _check("purify_vjp_positive", lib.purify_vjp_positive(n, _ptr(_c64(a, n, "a")), _ptr(_c64(rbar, n, "rbar")),
                                                          _ptr(abar), _stream(stream)))
    return abar


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().purify_launch_count())


def phi_static(n: int, J: int, uv: torch.Tensor, x: torch.Tensor, out: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
    """y = Phi x through purify_phi_static (no context, no allocation in the library)."""
    lib = load()
    M = int(uv.shape[0])
    if uv.dtype != torch.float32 or not uv.is_cuda or uv.dim() != 2 or uv.shape[1] != 2:
        raise ValueError("uv: (M, 2) float32 on a CUDA device")
    x = _c64(x, n * n, "x")
    y = out if out is not None else torch.empty(M, dtype=torch.complex64, device=x.device)
    _check("purify_phi_static", lib.purify_phi_static(int(n), int(J), M, _ptr(uv.contiguous()), _ptr(x), _ptr(y),
                                                      _stream(stream)))
    return y


def default_params() -> SdmmParams:
    p = SdmmParams()
    load().purify_sdmm_default_params(ctypes.byref(p))
    return p


class SdmmState:
    """Iteration variables of Algorithm 1 on a context."""

    def __init__(self, ctx: Context):
        self.c = ctx
        self.lib = ctx.lib
        out = _vp()
        _check("purify_sdmm_state_create", self.lib.purify_sdmm_state_create(ctx.ctx, ctypes.byref(out)))
        self.st = out.value

    def close(self) -> None:
        if getattr(self, "st", None):
            self.lib.purify_sdmm_state_destroy(self.st)
            self.st = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, y, eps: float, cg_iters: int = 10, beta: float = 1e-3, max_iters: int = 300,
             rounds: int = 1, use_graph: bool = True, stream=None) -> None:
        p = default_params()
        p.cg_iters, p.beta, p.max_iters, p.rounds = cg_iters, beta, max_iters, rounds
        p.use_graph = int(bool(use_graph))
        _check("purify_sdmm_init", self.lib.purify_sdmm_init(self.c.ctx, self.st, _ptr(y), float(eps),
                                                             ctypes.byref(p), _stream(stream)))

    def set_prior(self, prior: str = "sara", fgp_iters: int = 20) -> None:
        """"sara" (eq. delta) or "tv" (eq. tvproblem with positivity); before init()."""
        code = {"sara": 0, "tv": 1}[prior]
        _check("purify_sdmm_set_prior", self.lib.purify_sdmm_set_prior(self.c.ctx, self.st, code, int(fgp_iters)))

    def set_blocks(self, offsets=None, eps=None, stream=None) -> None:
        """Distributed-block form: blocks y[offsets[i]:offsets[i+1]] (caller order),
        one l2 ball of radius eps[i] each; None returns to the single ball."""
        if offsets is None:
            _check("purify_sdmm_set_blocks",
                   self.lib.purify_sdmm_set_blocks(self.c.ctx, self.st, 0, None, None, _stream(stream)))
            return
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        e = np.ascontiguousarray(eps, dtype=np.float64)
        R = len(e)
        if off.shape != (R + 1,):
            raise ValueError("offsets must have len(eps) + 1 entries")
        _check("purify_sdmm_set_blocks",
               self.lib.purify_sdmm_set_blocks(self.c.ctx, self.st, R, off.ctypes.data, e.ctypes.data,
                                               _stream(stream)))

    def set_data(self, y, stream=None) -> None:
        _check("purify_sdmm_set_data", self.lib.purify_sdmm_set_data(self.c.ctx, self.st, _ptr(y),
                                                                     _stream(stream)))

    def set_data_bf16(self, y, stream=None) -> None:
        _check("purify_sdmm_set_data_bf16",
               self.lib.purify_sdmm_set_data_bf16(self.c.ctx, self.st, _ptr(y), _stream(stream)))

    def step(self, stream=None) -> None:
        _check("purify_sdmm_step", self.lib.purify_sdmm_step(self.c.ctx, self.st, _stream(stream)))

    def reweight(self, round_index: int, stream=None) -> None:
        _check("purify_sdmm_reweight",
               self.lib.purify_sdmm_reweight(self.c.ctx, self.st, int(round_index), _stream(stream)))

    def set_weights(self, w: torch.Tensor, stream=None) -> None:
        if w.dtype != torch.float32 or w.numel() != self.c.D or not w.is_cuda:
            raise ValueError("w: D float32 values on the device")
        _check("purify_sdmm_set_weights",
               self.lib.purify_sdmm_set_weights(self.c.ctx, self.st, _ptr(w.contiguous()), _stream(stream)))

    def get_image(self, out=None, stream=None):
        if out is None:
            out = self.c._img((self.c.n, self.c.n))
        _check("purify_sdmm_get_image", self.lib.purify_sdmm_get_image(self.c.ctx, self.st, _ptr(out),
                                                                       _stream(stream)))
        return out

    def report(self, stream=None) -> dict:
        rep = Report()
        _check("purify_sdmm_get_report",
               self.lib.purify_sdmm_get_report(self.c.ctx, self.st, ctypes.byref(rep), _stream(stream)))
        return rep.as_dict()

    def export(self, stream=None) -> bytes:
        nb = ctypes.c_size_t()
        _check("purify_sdmm_state_bytes", self.lib.purify_sdmm_state_bytes(self.c.ctx, ctypes.byref(nb)))
        buf = ctypes.create_string_buffer(nb.value)
        _check("purify_sdmm_export",
               self.lib.purify_sdmm_export(self.c.ctx, self.st, buf, nb.value, _stream(stream)))
        return buf.raw

    def import_(self, blob: bytes, stream=None) -> None:
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check("purify_sdmm_import",
               self.lib.purify_sdmm_import(self.c.ctx, self.st, buf, len(blob), _stream(stream)))


def l2_bound(M: int, sigma: float) -> float:
    """purify_l2_bound: the chi^2 bound eps of §6 for M visibilities with noise level sigma."""
    out = ctypes.c_double()
    _check("purify_l2_bound", load().purify_l2_bound(int(M), float(sigma), ctypes.byref(out)))
    return out.value


class Batch:
    """Independent SDMM problems advanced together (one CUDA graph per iteration)."""

    def __init__(self, states: list[SdmmState]):
        self.lib = load()
        self.states = list(states)  # keep the contexts and states alive
        n = len(self.states)
        ctxs = (_vp * n)(*[st.c.ctx for st in self.states])
        sts = (_vp * n)(*[st.st for st in self.states])
        out = _vp()
        _check("purify_batch_create", self.lib.purify_batch_create(ctypes.byref(out), ctxs, sts, n))
        self.b = out.value

    def step(self, iters: int = 1, stream=None) -> None:
        _check("purify_batch_step", self.lib.purify_batch_step(self.b, int(iters), _stream(stream)))

    def kernels_per_iteration(self) -> int:
        cnt, k = _i32(), _i32()
        _check("purify_batch_size", self.lib.purify_batch_size(self.b, ctypes.byref(cnt), ctypes.byref(k)))
        return int(k.value)

    def close(self) -> None:
        if getattr(self, "b", None):
            self.lib.purify_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
