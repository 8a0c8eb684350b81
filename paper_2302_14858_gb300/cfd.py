"""Thin ctypes binding of the C ABI in include/cfd.h (argument marshalling only).

Every function keeps the C name and forwards to libcfd.so; all arithmetic
runs in the library's CUDA kernels.  Device buffers are passed as torch
tensors (or raw integer addresses); streams as torch.cuda.Stream, an integer
cudaStream_t, or None for the current torch stream.  A failed call raises
``CfdError`` carrying the status and the library's message.  Importing this
module fails loudly when libcfd.so has not been built.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_size_t, c_uint, c_void_p
from typing import Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcfd.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -m paper_2302_14858_gb300.build` "
        "(the CFD operators have no other implementation)")

_lib = ctypes.CDLL(LIB_PATH)

# status codes
CFD_OK, CFD_ERR_ARG, CFD_ERR_CUDA, CFD_ERR_UNSUPPORTED, CFD_ERR_NOT_CONVERGED, CFD_ERR_TIMEOUT, \
    CFD_ERR_DEVICE_ASSERT, CFD_ERR_ALLOC = range(8)
# precisions
CFD_FP64_BANDED, CFD_TC_BF16X3, CFD_TC_BF16_EXACT, CFD_TC_TF32 = range(4)
# dtypes
CFD_F64, CFD_F32 = 0, 1
# ops
OPS = ("dx", "dy", "dz", "dxx", "dyy", "dzz", "dxy", "dxz", "dyz")
OP_BITS = {name: 1 << i for i, name in enumerate(OPS)}
CFD_OP_DX, CFD_OP_DY, CFD_OP_DZ, CFD_OP_DXX, CFD_OP_DYY, CFD_OP_DZZ, CFD_OP_DXY, CFD_OP_DXZ, CFD_OP_DYZ = \
    (1 << i for i in range(9))
CFD_OP_ALL = 0x1FF

EXPORTS = ("cfd_scheme_create", "cfd_scheme_closure", "cfd_scheme_destroy", "cfd_blocks_bind",
           "cfd_blocks_destroy", "cfd_exchange_ghosts", "cfd_apply_workspace", "cfd_apply",
           "cfd_wave_workspace", "cfd_wave_rk_step", "cfd_wave_lsrk_workspace", "cfd_wave_lsrk_step",
           "cfd_sync_status", "cfd_last_error",
           "cfd_kernel_launches", "cfd_profile_enable", "cfd_profile_read", "cfd_apply_static",
           "cfd_debug_set_wait_limit", "cfd_blocks_set_mixed_order", "cfd_autotune", "cfd_autotune_report",
           "cfd_scheme_set_biased", "cfd_biased_workspace", "cfd_apply_biased", "cfd_advect",
           "cfd_shifted_wave_workspace", "cfd_shifted_wave_lsrk_step", "cfd_advect_lsrk_workspace",
           "cfd_advect_lsrk_step", "cfd_halo_plan_create", "cfd_halo_plan_bytes", "cfd_halo_pack",
           "cfd_halo_unpack", "cfd_halo_plan_destroy")
KERNEL_FAMILIES = {"exchange": 0, "line": 1, "rk_combine": 2, "dense": 3, "dense_halo": 4, "biased": 5}


class CfdError(RuntimeError):
    """A call that returned a status other than CFD_OK (status and the library's message)."""
    def __init__(self, status: int, msg: str):
        super().__init__(f"cfd status {status}: {msg}")
        self.status = status


class SchemeDesc(ctypes.Structure):
    """cfd_scheme_desc: one centred tridiagonal scheme of one derivative degree."""
    _fields_ = [("deriv", c_int), ("order", c_int), ("M", c_int), ("lhs_offdiag", c_double),
                ("rhs", POINTER(c_double)), ("closure_halfwidth", c_int), ("closure", POINTER(c_double))]


_lib.cfd_scheme_create.argtypes = [POINTER(SchemeDesc), POINTER(SchemeDesc), POINTER(c_void_p)]
_lib.cfd_scheme_create.restype = c_int
_lib.cfd_scheme_closure.argtypes = [c_void_p, c_int, POINTER(c_double), POINTER(c_int)]
_lib.cfd_scheme_closure.restype = c_int
_lib.cfd_scheme_destroy.argtypes = [c_void_p]
_lib.cfd_scheme_destroy.restype = None
_lib.cfd_blocks_bind.argtypes = [c_void_p, c_int, POINTER(c_int), POINTER(c_double), POINTER(c_int), c_int, c_int,
                                 POINTER(c_void_p)]
_lib.cfd_blocks_bind.restype = c_int
_lib.cfd_blocks_destroy.argtypes = [c_void_p]
_lib.cfd_blocks_destroy.restype = None
_lib.cfd_exchange_ghosts.argtypes = [c_void_p, c_void_p, c_int, c_void_p]
_lib.cfd_exchange_ghosts.restype = c_int
_lib.cfd_apply_workspace.argtypes = [c_void_p, c_int, c_uint, c_int, c_int, POINTER(c_size_t)]
_lib.cfd_apply_workspace.restype = c_int
_lib.cfd_apply.argtypes = [c_void_p, c_void_p, c_int, c_uint, c_int, c_int, c_void_p, c_void_p, c_size_t, c_void_p]
_lib.cfd_apply.restype = c_int
_lib.cfd_apply_static.argtypes = [c_void_p, c_void_p, c_int, c_uint, c_void_p, c_void_p]
_lib.cfd_apply_static.restype = c_int
_lib.cfd_wave_workspace.argtypes = [c_void_p, c_int, c_int, POINTER(c_size_t)]
_lib.cfd_wave_workspace.restype = c_int
_lib.cfd_wave_rk_step.argtypes = [c_void_p, c_void_p, c_void_p, c_double, c_int, c_int, c_void_p, c_size_t, c_void_p]
_lib.cfd_wave_rk_step.restype = c_int


class LsrkDesc(ctypes.Structure):
    """cfd_lsrk_desc: the coefficients of a two-register (2S) low-storage RK method."""
    _fields_ = [("stages", c_int), ("gamma1", POINTER(c_double)), ("gamma2", POINTER(c_double)),
                ("beta", POINTER(c_double)), ("delta", POINTER(c_double))]


_lib.cfd_wave_lsrk_workspace.argtypes = [c_void_p, c_int, c_int, POINTER(c_size_t)]
_lib.cfd_wave_lsrk_workspace.restype = c_int
_lib.cfd_wave_lsrk_step.argtypes = [c_void_p, c_void_p, c_void_p, c_double, POINTER(LsrkDesc), c_double, c_int,
                                    c_int, c_int, c_void_p, c_size_t, c_void_p]
_lib.cfd_wave_lsrk_step.restype = c_int


class BiasedDesc(ctypes.Structure):
    """cfd_biased_desc: a left-biased first-degree scheme with its closure."""
    _fields_ = [("order", c_int), ("a", c_double), ("rhs_lo", c_int), ("rhs_n", c_int), ("rhs", POINTER(c_double)),
                ("closure_sup", c_double), ("closure_lo", c_int), ("closure_n", c_int),
                ("closure", POINTER(c_double)), ("kc", c_int)]


_lib.cfd_scheme_set_biased.argtypes = [c_void_p, POINTER(BiasedDesc)]
_lib.cfd_scheme_set_biased.restype = c_int
_lib.cfd_biased_workspace.argtypes = [c_void_p, c_int, c_int, c_int, POINTER(c_size_t)]
_lib.cfd_biased_workspace.restype = c_int
_lib.cfd_apply_biased.argtypes = [c_void_p, c_void_p, c_int, c_uint, c_int, c_int, c_int, c_void_p, c_void_p,
                                  c_size_t, c_void_p]
_lib.cfd_apply_biased.restype = c_int
_lib.cfd_advect.argtypes = [c_void_p, c_void_p, c_int, c_void_p, c_int, c_int, c_void_p, c_void_p, c_size_t,
                            c_void_p]
_lib.cfd_advect.restype = c_int
_lib.cfd_shifted_wave_workspace.argtypes = [c_void_p, c_int, c_int, POINTER(c_size_t)]
_lib.cfd_shifted_wave_workspace.restype = c_int
_lib.cfd_shifted_wave_lsrk_step.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_double, POINTER(LsrkDesc),
                                            c_double, c_int, c_int, c_int, c_void_p, c_size_t, c_void_p]
_lib.cfd_shifted_wave_lsrk_step.restype = c_int
_lib.cfd_advect_lsrk_workspace.argtypes = [c_void_p, c_int, c_int, c_int, POINTER(c_size_t)]
_lib.cfd_advect_lsrk_workspace.restype = c_int
_lib.cfd_advect_lsrk_step.argtypes = [c_void_p, c_void_p, c_int, c_void_p, c_double, POINTER(LsrkDesc), c_double,
                                      c_int, c_int, c_int, c_void_p, c_size_t, c_void_p]
_lib.cfd_advect_lsrk_step.restype = c_int
_lib.cfd_halo_plan_create.argtypes = [c_void_p, POINTER(c_int), c_int, POINTER(c_void_p)]
_lib.cfd_halo_plan_create.restype = c_int
_lib.cfd_halo_plan_bytes.argtypes = [c_void_p, c_int, POINTER(c_size_t)]
_lib.cfd_halo_plan_bytes.restype = c_int
_lib.cfd_halo_pack.argtypes = [c_void_p, c_void_p, c_int, c_void_p, c_void_p]
_lib.cfd_halo_pack.restype = c_int
_lib.cfd_halo_unpack.argtypes = [c_void_p, c_void_p, c_int, c_void_p, c_void_p]
_lib.cfd_halo_unpack.restype = c_int
_lib.cfd_halo_plan_destroy.argtypes = [c_void_p]
_lib.cfd_halo_plan_destroy.restype = None
_lib.cfd_sync_status.argtypes = [c_void_p, c_void_p]
_lib.cfd_sync_status.restype = c_int
_lib.cfd_kernel_launches.argtypes = []
_lib.cfd_kernel_launches.restype = ctypes.c_ulonglong
_lib.cfd_profile_enable.argtypes = [c_int]
_lib.cfd_profile_enable.restype = c_int
_lib.cfd_profile_read.argtypes = [c_int, POINTER(ctypes.c_ulonglong), POINTER(c_double)]
_lib.cfd_profile_read.restype = c_int
_lib.cfd_autotune.argtypes = [c_void_p, c_void_p, c_int, ctypes.c_uint, c_int, c_int, c_void_p, c_void_p, ctypes.c_size_t,
                              c_void_p]
_lib.cfd_autotune.restype = c_int
_lib.cfd_autotune_report.argtypes = [c_void_p, ctypes.c_char_p, ctypes.c_size_t, POINTER(ctypes.c_size_t)]
_lib.cfd_autotune_report.restype = c_int
_lib.cfd_blocks_set_mixed_order.argtypes = [c_void_p, c_int]
_lib.cfd_blocks_set_mixed_order.restype = c_int
_lib.cfd_debug_set_wait_limit.argtypes = [ctypes.c_longlong]
_lib.cfd_debug_set_wait_limit.restype = c_int
_lib.cfd_last_error.argtypes = []
_lib.cfd_last_error.restype = ctypes.c_char_p


def cfd_last_error() -> str:
    """Message of the last failed call on this thread."""
    return _lib.cfd_last_error().decode()


def _check(status: int):
    if status != CFD_OK:
        raise CfdError(status, cfd_last_error())


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _nbytes(work, work_bytes=None) -> int:
    """Size of a workspace: a tensor's own size, or `work_bytes` for a raw device address."""
    if work is None:
        return 0
    if work_bytes is not None:
        return int(work_bytes)
    if isinstance(work, int):
        raise ValueError("a workspace given as a raw device address needs work_bytes")
    return work.numel() * work.element_size()


def _stream(s) -> Optional[int]:
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


class Scheme:
    """Owning wrapper of cfd_scheme_t."""

    def __init__(self, handle: int, keep):
        self.handle = handle
        self._keep = keep

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.cfd_scheme_destroy(self.handle)
            self.handle = None


class Blocks:
    """Owning wrapper of cfd_blocks_t."""

    def __init__(self, handle: int, nblocks: int, block_n, ng: int, dtype: int):
        self.handle = handle
        self.nblocks = nblocks
        self.block_n = list(block_n)
        self.ng = ng
        self.dtype = dtype

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.cfd_blocks_destroy(self.handle)
            self.handle = None


def _desc(d) -> Optional[SchemeDesc]:
    if d is None:
        return None
    rhs = (c_double * len(d["rhs"]))(*d["rhs"])
    clo = None
    if d.get("closure") is not None:
        clo = (c_double * len(d["closure"]))(*d["closure"])
    M = (len(d["rhs"]) - 1) // 2
    h = (len(d["closure"]) - 1) // 2 if clo is not None else 0
    s = SchemeDesc(d["deriv"], d["order"], M, float(d["a"]), ctypes.cast(rhs, POINTER(c_double)), h,
                   ctypes.cast(clo, POINTER(c_double)) if clo is not None else None)
    s._keep = (rhs, clo)
    return s


def cfd_scheme_create(first: Optional[dict], second: Optional[dict]) -> Scheme:
    """Scheme pair from dicts {deriv, order, a, rhs, closure (optional)}."""
    d1, d2 = _desc(first), _desc(second)
    h = c_void_p()
    _check(_lib.cfd_scheme_create(ctypes.byref(d1) if d1 else None, ctypes.byref(d2) if d2 else None,
                                  ctypes.byref(h)))
    return Scheme(h.value, (d1, d2))


def cfd_scheme_closure(scheme: Scheme, deriv: int):
    """The closure coefficients the scheme uses for degree `deriv` (given or C_0-matched)."""
    buf = (c_double * 13)()
    hw = c_int()
    _check(_lib.cfd_scheme_closure(scheme.handle, deriv, buf, ctypes.byref(hw)))
    return [buf[i] for i in range(2 * hw.value + 1)]


def cfd_blocks_bind(scheme: Scheme, block_n: Sequence[int], dx, neighbors, ng: int, dtype: int) -> Blocks:
    """Bind a scheme to a MeshBlock layout: per-block sizes, spacings and 26 neighbours (-1: none)."""
    import numpy as np
    nb = len(block_n)
    n_arr = (c_int * nb)(*[int(v) for v in block_n])
    dx = np.ascontiguousarray(dx, dtype=np.float64).reshape(nb, 3)
    nbr = np.ascontiguousarray(neighbors, dtype=np.int32).reshape(nb, 26)
    h = c_void_p()
    _check(_lib.cfd_blocks_bind(scheme.handle, nb, n_arr, dx.ctypes.data_as(POINTER(c_double)),
                                nbr.ctypes.data_as(POINTER(c_int)), ng, dtype, ctypes.byref(h)))
    return Blocks(h.value, nb, block_n, ng, dtype)


def cfd_exchange_ghosts(blocks: Blocks, fields, nfields: int, stream=None):
    """Ghost fill of every block from its neighbours (matrix G, Eq. example_G)."""
    _check(_lib.cfd_exchange_ghosts(blocks.handle, _ptr(fields), nfields, _stream(stream)))


def cfd_apply_workspace(blocks: Blocks, nfields: int, op_mask: int, prec: int, n_iter: int) -> int:
    """Device workspace bytes cfd_apply needs for this request."""
    n = c_size_t()
    _check(_lib.cfd_apply_workspace(blocks.handle, nfields, op_mask, prec, n_iter, ctypes.byref(n)))
    return n.value


def cfd_apply(blocks: Blocks, fields, nfields: int, op_mask: int, prec: int, n_iter: int, out, work,
              stream=None, work_bytes=None):
    """The requested derivatives of every field (Eq. sch_cent_om closed, Eq. iter_center_P iterated)."""
    _check(_lib.cfd_apply(blocks.handle, _ptr(fields), nfields, op_mask, prec, n_iter, _ptr(out), _ptr(work),
                          _nbytes(work, work_bytes), _stream(stream)))


def cfd_apply_static(blocks: Blocks, fields, nfields: int, op_mask: int, out, stream=None):
    """cfd_apply (FP64 banded, closures only) with its scratch in the library's static device array.

    For callers that cannot allocate device memory at the call site; see
    include/cfd.h for the 64 MiB limit and the first-call set-up.
    """
    _check(_lib.cfd_apply_static(blocks.handle, _ptr(fields), nfields, op_mask, _ptr(out), _stream(stream)))


def cfd_wave_workspace(blocks: Blocks, prec: int, n_iter: int) -> int:
    """Device workspace bytes of cfd_wave_rk_step."""
    n = c_size_t()
    _check(_lib.cfd_wave_workspace(blocks.handle, prec, n_iter, ctypes.byref(n)))
    return n.value


def cfd_wave_rk_step(blocks: Blocks, phi, K, dt: float, prec: int, n_iter: int, work, stream=None,
                     work_bytes=None):
    """One classical RK4 step of Phi_t = K, K_t = sum_i D2_i Phi, in place."""
    _check(_lib.cfd_wave_rk_step(blocks.handle, _ptr(phi), _ptr(K), float(dt), prec, n_iter, _ptr(work),
                                 _nbytes(work, work_bytes), _stream(stream)))


def cfd_wave_lsrk_workspace(blocks: Blocks, prec: int, n_iter: int) -> int:
    """Device workspace bytes of cfd_wave_lsrk_step."""
    n = c_size_t()
    _check(_lib.cfd_wave_lsrk_workspace(blocks.handle, prec, n_iter, ctypes.byref(n)))
    return n.value


def _lsrk_desc(coef):
    """cfd_lsrk_desc of coef = (gamma1, gamma2, beta, delta), sequences of equal length; the
    arrays it points to are returned beside it and must stay alive for the call."""
    g1, g2, be, de = (list(map(float, c)) for c in coef)
    m = len(be)
    if not (len(g1) == len(g2) == len(de) == m):
        raise ValueError("the four coefficient sequences need the same length")
    arrs = [(c_double * m)(*v) for v in (g1, g2, be, de)]
    return LsrkDesc(m, *[ctypes.cast(a, POINTER(c_double)) for a in arrs]), arrs


def cfd_wave_lsrk_step(blocks: Blocks, phi, K, dt: float, coef, sigma: float, ko_r: int, prec: int, n_iter: int,
                       work, stream=None, work_bytes=None):
    """coef = (gamma1, gamma2, beta, delta), sequences of equal length (the 2S coefficients)."""
    desc, _keep = _lsrk_desc(coef)
    _check(_lib.cfd_wave_lsrk_step(blocks.handle, _ptr(phi), _ptr(K), float(dt), ctypes.byref(desc), float(sigma),
                                   int(ko_r), prec, n_iter, _ptr(work), _nbytes(work, work_bytes), _stream(stream)))


def cfd_scheme_set_biased(scheme: Scheme, d: dict):
    """Attach a left-biased scheme: dict {order, a, lo, rhs, c_sup, c_lo, closure, kc}
    (a = alpha^{(1)}_{-1}, rhs over offsets lo.., closure over offsets c_lo.. with
    alpha-bar^{(1)}_{+1} = c_sup)."""
    rhs = (c_double * len(d["rhs"]))(*map(float, d["rhs"]))
    clo = (c_double * len(d["closure"]))(*map(float, d["closure"]))
    desc = BiasedDesc(int(d["order"]), float(d["a"]), int(d["lo"]), len(d["rhs"]), ctypes.cast(rhs, POINTER(c_double)),
                      float(d["c_sup"]), int(d["c_lo"]), len(d["closure"]), ctypes.cast(clo, POINTER(c_double)),
                      int(d["kc"]))
    _check(_lib.cfd_scheme_set_biased(scheme.handle, ctypes.byref(desc)))


def cfd_biased_workspace(blocks: Blocks, nfields: int, prec: int, n_iter: int) -> int:
    """Device workspace bytes of cfd_apply_biased / cfd_advect."""
    n = c_size_t()
    _check(_lib.cfd_biased_workspace(blocks.handle, nfields, prec, n_iter, ctypes.byref(n)))
    return n.value


def cfd_apply_biased(blocks: Blocks, fields, nfields: int, axis_mask: int, side: int, prec: int, n_iter: int, out,
                     work=None, stream=None, work_bytes=None):
    """Biased first derivatives along the masked axes: side +1 left-biased S+, -1 right-biased S-
    (Eqs. closure_left_X, iter_left_X and their mirrors)."""
    _check(_lib.cfd_apply_biased(blocks.handle, _ptr(fields), nfields, axis_mask, side, prec, n_iter, _ptr(out),
                                 _ptr(work), _nbytes(work, work_bytes), _stream(stream)))


def cfd_advect(blocks: Blocks, fields, nfields: int, beta, prec: int, n_iter: int, out, work=None, stream=None,
               work_bytes=None):
    """The upwinded shift-advection term sum_i beta^i d_i f of every field (Eq. biasderapproxadv)."""
    _check(_lib.cfd_advect(blocks.handle, _ptr(fields), nfields, _ptr(beta), prec, n_iter, _ptr(out), _ptr(work),
                           _nbytes(work, work_bytes), _stream(stream)))


def cfd_shifted_wave_workspace(blocks: Blocks, prec: int, n_iter: int) -> int:
    """Device workspace bytes of cfd_shifted_wave_lsrk_step."""
    n = c_size_t()
    _check(_lib.cfd_shifted_wave_workspace(blocks.handle, prec, n_iter, ctypes.byref(n)))
    return n.value


def cfd_shifted_wave_lsrk_step(blocks: Blocks, phi, K, beta, dt: float, coef, sigma: float, ko_r: int, prec: int,
                               n_iter: int, work, stream=None, work_bytes=None):
    """As cfd_wave_lsrk_step with the upwinded shift terms; beta = three fields in the field layout."""
    desc, _keep = _lsrk_desc(coef)
    _check(_lib.cfd_shifted_wave_lsrk_step(blocks.handle, _ptr(phi), _ptr(K), _ptr(beta), float(dt),
                                           ctypes.byref(desc), float(sigma), int(ko_r), prec, n_iter, _ptr(work),
                                           _nbytes(work, work_bytes), _stream(stream)))


def cfd_advect_lsrk_workspace(blocks: Blocks, nfields: int, prec: int, n_iter: int) -> int:
    """Device workspace bytes of cfd_advect_lsrk_step."""
    n = c_size_t()
    _check(_lib.cfd_advect_lsrk_workspace(blocks.handle, nfields, prec, n_iter, ctypes.byref(n)))
    return n.value


def cfd_advect_lsrk_step(blocks: Blocks, u, nfields: int, beta, dt: float, coef, sigma: float, ko_r: int, prec: int,
                         n_iter: int, work, stream=None, work_bytes=None):
    """2S step of u_t = beta . grad u (+ Kreiss-Oliger) for nfields fields; coef = (gamma1, gamma2, beta, delta)."""
    desc, _keep = _lsrk_desc(coef)
    _check(_lib.cfd_advect_lsrk_step(blocks.handle, _ptr(u), nfields, _ptr(beta), float(dt), ctypes.byref(desc),
                                     float(sigma), int(ko_r), prec, n_iter, _ptr(work), _nbytes(work, work_bytes),
                                     _stream(stream)))


class HaloPlan:
    """Owning wrapper of cfd_halo_plan_t (keeps its Blocks alive)."""

    def __init__(self, handle: int, blocks: Blocks, n: int):
        self.handle = handle
        self.blocks = blocks
        self.n = n

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.cfd_halo_plan_destroy(self.handle)
            self.handle = None


def cfd_halo_plan_create(blocks: Blocks, items) -> HaloPlan:
    """items: sequence of (local block, direction) pairs (see include/cfd.h)."""
    import numpy as np
    arr = np.ascontiguousarray(np.asarray(items, dtype=np.int32).reshape(-1, 2))
    h = c_void_p()
    _check(_lib.cfd_halo_plan_create(blocks.handle, arr.ctypes.data_as(POINTER(c_int)), len(arr), ctypes.byref(h)))
    return HaloPlan(h.value, blocks, len(arr))


def cfd_halo_plan_bytes(plan: HaloPlan, nfields: int) -> int:
    """Bytes of the contiguous buffer that holds the plan's slabs for nfields fields."""
    n = c_size_t()
    _check(_lib.cfd_halo_plan_bytes(plan.handle, nfields, ctypes.byref(n)))
    return n.value


def cfd_halo_pack(plan: HaloPlan, fields, nfields: int, buf, stream=None):
    """Copy the plan's interior slabs of every field into `buf` (plan order)."""
    _check(_lib.cfd_halo_pack(plan.handle, _ptr(fields), nfields, _ptr(buf), _stream(stream)))


def cfd_halo_unpack(plan: HaloPlan, fields, nfields: int, buf, stream=None):
    """Write `buf` (plan order) into the plan's ghost regions of every field."""
    _check(_lib.cfd_halo_unpack(plan.handle, _ptr(fields), nfields, _ptr(buf), _stream(stream)))


def cfd_autotune(blocks: Blocks, fields, nfields: int, op_mask: int, prec: int, n_iter: int, out, work,
                 stream=None, work_bytes=None):
    """cfd_apply once with every kernel launched under each candidate configuration; the fastest
    per kernel is kept for later calls of the same request (synchronises the stream)."""
    _check(_lib.cfd_autotune(blocks.handle, _ptr(fields), nfields, op_mask, prec, n_iter, _ptr(out), _ptr(work),
                             _nbytes(work, work_bytes), _stream(stream)))


def cfd_autotune_report(blocks: Blocks) -> dict:
    """The autotuner's choices and times: {request: [{stage, staging, order, ms}, ...]}."""
    import json
    need = ctypes.c_size_t(0)
    _check(_lib.cfd_autotune_report(blocks.handle, None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(need.value)
    _check(_lib.cfd_autotune_report(blocks.handle, buf, need.value, ctypes.byref(need)))
    return json.loads(buf.value.decode())


def cfd_blocks_set_mixed_order(blocks: Blocks, one_order: bool):
    """FP64 banded mixed derivatives as D_i D_j only (True) or the symmetrised average (False)."""
    _check(_lib.cfd_blocks_set_mixed_order(blocks.handle, 1 if one_order else 0))


def cfd_sync_status(blocks: Blocks, stream=None):
    """Synchronise the stream and raise a status latched on the device (e.g. a bounded wait that ran out)."""
    _check(_lib.cfd_sync_status(blocks.handle, _stream(stream)))


def cfd_kernel_launches() -> int:
    """Kernels this library has launched in the process so far."""
    return int(_lib.cfd_kernel_launches())


def cfd_profile_enable(on: bool):
    """Turn per-launch CUDA-event timing of the kernel families on or off."""
    _check(_lib.cfd_profile_enable(1 if on else 0))


def cfd_profile_read(family: int):
    """(launches, summed device ms) of one kernel family since profiling was enabled."""
    n = ctypes.c_ulonglong()
    ms = c_double()
    _check(_lib.cfd_profile_read(family, ctypes.byref(n), ctypes.byref(ms)))
    return int(n.value), float(ms.value)


def op_mask(ops: Sequence[str]) -> int:
    """Bit mask of the named ops (dx ... dyz)."""
    m = 0
    for o in ops:
        m |= OP_BITS[o]
    return m


def ops_in_mask(mask: int):
    """Names of the ops in a bit mask, in output order."""
    return [o for o in OPS if mask & OP_BITS[o]]


def cfd_debug_set_wait_limit(cycles: int):
    """Main-loop wait limit of the tensor-core kernel in clock cycles (<= 0: the default, ~2 s)."""
    _check(_lib.cfd_debug_set_wait_limit(int(cycles)))
