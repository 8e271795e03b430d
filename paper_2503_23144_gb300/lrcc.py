"""Thin ctypes binding of the C ABI in ``include/lrcc.h`` (argument marshalling only).

Every function keeps the C name.  Host arrays are numpy; the ``*_dev`` calls
take CUDA tensors from PyTorch (device memory and the current stream) and
pass their raw pointers.  No arithmetic of the method happens here: the CUDA
library does every step, and importing this module fails loudly when the
library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lrcc.so")

LRCC_OK, LRCC_EINVAL, LRCC_ENOMEM, LRCC_ENOCONV, LRCC_ETIMEOUT, LRCC_ECUDA, LRCC_ESTATE = range(7)
LRCC_FP64, LRCC_MIXED_TF32, LRCC_MIXED_BF16X3, LRCC_FP64_EMULATED = 0, 1, 2, 3
LRCC_RES_T, LRCC_RES_SIGMA, LRCC_RES_VJP, LRCC_RES_XI, LRCC_RES_ENERGY, LRCC_RES_VJP_FULL = range(6)

STATUS_NAMES = {0: "LRCC_OK", 1: "LRCC_EINVAL", 2: "LRCC_ENOMEM", 3: "LRCC_ENOCONV", 4: "LRCC_ETIMEOUT",
                5: "LRCC_ECUDA", 6: "LRCC_ESTATE"}


class lrcc_options(ctypes.Structure):
    _fields_ = [("r_tol", ctypes.c_double), ("x_tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("diis_size", ctypes.c_int), ("rhs_chunk", ctypes.c_int), ("prec", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("plus_omega", ctypes.c_int), ("slab_rows", ctypes.c_int),
                ("pm_omega", ctypes.c_int), ("fp64_products", ctypes.c_int), ("fns_density", ctypes.c_int),
                ("solver", ctypes.c_int), ("subspace_max", ctypes.c_int), ("ladder_hermitian", ctypes.c_int),
                ("embed_budget_mb", ctypes.c_int)]


class LrccError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p
_i64p = ctypes.POINTER(ctypes.c_int64)

# (name, restype, argtypes) of every exported symbol
SIGNATURES = [
    ("lrcc_default_options", None, [ctypes.POINTER(lrcc_options)]),
    ("lrcc_setup", ctypes.c_int, [_dp, _dp, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.POINTER(lrcc_options), ctypes.POINTER(_vp)]),
    ("lrcc_destroy", None, [_vp]),
    ("lrcc_last_error", ctypes.c_char_p, [_vp]),
    ("lrcc_ccsd_ground", ctypes.c_int, [_vp, _dp, _ip, _ip]),
    ("lrcc_fns_truncate", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, _ip, _dp]),
    ("lrcc_solve", ctypes.c_int, [_vp, _dp, ctypes.c_int, _ip, ctypes.c_int, _dp, _dp]),
    ("lrcc_residual", ctypes.c_int, [_vp, ctypes.c_int, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]),
    ("lrcc_residual_dev", ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         _vp, _vp]),
    ("lrcc_ladder_dev", ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp]),
    ("lrcc_ladder_packed_dev", ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _vp]),
    ("lrcc_phase_times", ctypes.c_int, [_vp, _dp]),
    ("lrcc_kernel_launches", ctypes.c_int64, [_vp]),
    ("lrcc_memory_stats", ctypes.c_int, [_vp, _i64p, _i64p, _i64p]),
    ("lrcc_profile", ctypes.c_int, [_vp, ctypes.c_int]),
    ("lrcc_profile_dump", ctypes.c_int, [_vp, ctypes.c_char_p]),
    ("lrcc_get_amplitudes", ctypes.c_int, [_vp, ctypes.c_int, _dp]),
    ("lrcc_mp2_correction", ctypes.c_int, [_vp, _dp, _dp, _dp]),
    ("lrcc_mp2_alpha", ctypes.c_int, [_vp, _dp, ctypes.c_int, _ip, ctypes.c_int, _dp]),
    ("lrcc_embed_layout", ctypes.c_int, [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    ("lrcc_plan_slabs", ctypes.c_int64, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_int64), ctypes.c_int64]),
    ("lrcc_ladder_noalloc", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp,
                                           ctypes.c_int, _vp]),
    ("lrcc_solve_counts", ctypes.c_int, [_vp, _ip, _ip]),
    ("lrcc_linearize", ctypes.c_int, [_vp, _dp, ctypes.c_int]),
    ("lrcc_kernel_stats", ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                         ctypes.POINTER(ctypes.c_int64), _dp, _dp, _dp]),
]


def library():
    """Load ``_lrcc.so`` (raises ImportError if it is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"CUDA library not built: {_LIB_PATH} (run paper_2503_23144_gb300.build.build())")
        lib = ctypes.CDLL(_LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _cd(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def lrcc_default_options() -> lrcc_options:
    o = lrcc_options()
    library().lrcc_default_options(ctypes.byref(o))
    return o


class Context:
    """Owns one ``lrcc_ctx*``; sizes are kept for marshalling."""

    def __init__(self, handle, O, V, L, ncomp):
        self.h = handle
        self.O, self.V, self.L, self.ncomp = O, V, L, ncomp

    def check(self, st):
        if st != LRCC_OK:
            raise LrccError(st, library().lrcc_last_error(self.h).decode())

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.lrcc_destroy(self.h)
            self.h = None

    @property
    def n_amp(self):
        return self.O * self.V + self.O * self.O * self.V * self.V


def lrcc_setup(eps, B, mu, O: int, V: int, opt: lrcc_options | None = None) -> Context:
    lib = library()
    eps = np.ascontiguousarray(np.asarray(eps, dtype=np.float64))
    B = _c128(B)
    mu = _c128(mu)
    if mu.ndim == 2:
        mu = mu[None]
    L, ncomp = B.shape[0], mu.shape[0]
    h = _vp()
    st = lib.lrcc_setup(_cd(eps), _cd(B.view(np.float64)), L, _cd(mu.view(np.float64)), ncomp, O, V,
                        ctypes.byref(opt) if opt is not None else None, ctypes.byref(h))
    if st != LRCC_OK:
        raise LrccError(st, lib.lrcc_last_error(None).decode())
    return Context(h, O, V, L, ncomp)


def lrcc_ccsd_ground(ctx: Context):
    e = np.zeros(2)
    it_t, it_l = ctypes.c_int(0), ctypes.c_int(0)
    ctx.check(library().lrcc_ccsd_ground(ctx.h, _cd(e), ctypes.byref(it_t), ctypes.byref(it_l)))
    return complex(e[0], e[1]), it_t.value, it_l.value


def lrcc_solve(ctx: Context, omegas, comps):
    om = np.ascontiguousarray(np.asarray(omegas, dtype=np.float64).reshape(-1))
    cp = np.ascontiguousarray(np.asarray(comps, dtype=np.int32).reshape(-1))
    alpha = np.zeros((om.size, cp.size, cp.size), dtype=np.complex128)
    err = np.zeros((om.size, cp.size))
    ctx.check(library().lrcc_solve(ctx.h, _cd(om), om.size, cp.ctypes.data_as(_ip), cp.size,
                                   _cd(alpha.view(np.float64)), _cd(err)))
    return alpha, err


def lrcc_fns_truncate(ctx: Context, by_count: bool, value: float, omega: float = 0.0):
    vk = ctypes.c_int(0)
    occ = np.zeros(ctx.V)
    ctx.check(library().lrcc_fns_truncate(ctx.h, int(by_count), float(value), float(omega), ctypes.byref(vk),
                                          _cd(occ)))
    ctx.V = vk.value
    return vk.value, occ


def lrcc_mp2_correction(ctx: Context):
    """(E_MP2 full, E_MP2 truncated, Delta = full - truncated), complex (Eq. 51)."""
    a, b, d = np.zeros(2), np.zeros(2), np.zeros(2)
    ctx.check(library().lrcc_mp2_correction(ctx.h, _cd(a), _cd(b), _cd(d)))
    return complex(*a), complex(*b), complex(*d)


def lrcc_mp2_alpha(ctx: Context, omegas, comps) -> np.ndarray:
    """MP2-level alpha [n_w, n_c, n_c] in the context's current basis (Eq. 53-54 ingredient)."""
    om = np.ascontiguousarray(np.asarray(omegas, dtype=np.float64).reshape(-1))
    cp = np.ascontiguousarray(np.asarray(comps, dtype=np.int32).reshape(-1))
    alpha = np.zeros((om.size, cp.size, cp.size), dtype=np.complex128)
    ctx.check(library().lrcc_mp2_alpha(ctx.h, _cd(om), om.size, cp.ctypes.data_as(_ip), cp.size,
                                       _cd(alpha.view(np.float64))))
    return alpha


def lrcc_embed_layout(prec: int, K: int, rows: int, batch: int = 1):
    """(panels, panel width in elements) of an embedded tensor-core operand (host only)."""
    n, w = ctypes.c_int64(0), ctypes.c_int64(0)
    st = library().lrcc_embed_layout(int(prec), int(K), int(rows), int(batch), ctypes.byref(n), ctypes.byref(w))
    if st != LRCC_OK:
        raise LrccError(st, "lrcc_embed_layout: bad arguments")
    return n.value, w.value


def lrcc_plan_slabs(V: int, budget_el: int, row_cap: int, cap_rows: int) -> np.ndarray:
    """Assembly chunks of the uncached ladder, [n, 7] int64 rows
    (a0, a1, b0, b1, prow0, nrows, group) (host only)."""
    lib = library()
    n = lib.lrcc_plan_slabs(int(V), int(budget_el), int(row_cap), int(cap_rows), None, 0)
    if n < 0:
        raise LrccError(LRCC_EINVAL, "lrcc_plan_slabs: bad arguments")
    out = np.zeros((max(n, 1), 7), dtype=np.int64)
    lib.lrcc_plan_slabs(int(V), int(budget_el), int(row_cap), int(cap_rows),
                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n)
    return out[:n]


def pack_amplitudes(t1, t2) -> np.ndarray:
    """[R, O, V] and [R, O, O, V, V] -> the flat [R, O*V + O*O*V*V] layout of the ABI."""
    t1 = np.asarray(t1, dtype=np.complex128)
    t2 = np.asarray(t2, dtype=np.complex128)
    R = t1.shape[0]
    return np.ascontiguousarray(np.concatenate([t1.reshape(R, -1), t2.reshape(R, -1)], axis=1))


def unpack_amplitudes(flat, O, V):
    flat = np.asarray(flat)
    R = flat.shape[0]
    n1 = O * V
    return flat[:, :n1].reshape(R, O, V), flat[:, n1:].reshape(R, O, O, V, V)


def lrcc_residual(ctx: Context, kind: int, t, x, comp: int = 0, prec: int = LRCC_FP64) -> np.ndarray:
    """t: flat [n_amp] (or None), x: flat [R, n_amp]; returns [R, n_amp] (ENERGY: [R])."""
    x = _c128(x)
    if x.ndim == 1:
        x = x[None]
    R = x.shape[0]
    tp = _cd(_c128(t).view(np.float64)) if t is not None else None
    if kind == LRCC_RES_ENERGY:
        out = np.zeros(R, dtype=np.complex128)
    else:
        out = np.zeros((R, ctx.n_amp), dtype=np.complex128)
    tt = _c128(t) if t is not None else None
    ctx.check(library().lrcc_residual(ctx.h, kind, _cd(tt.view(np.float64)) if tt is not None else None,
                                      _cd(x.view(np.float64)), R, comp, prec, _cd(out.view(np.float64))))
    del tp
    return out


def lrcc_linearize(ctx: Context, t, prec: int = LRCC_FP64) -> None:
    """Fix the amplitudes t (flat [n_amp], host) at which later residual maps
    with t=None are applied (the program is evaluated once at t)."""
    tt = _c128(t).reshape(-1)
    ctx.check(library().lrcc_linearize(ctx.h, _cd(tt.view(np.float64)), prec))


def _stream_ptr():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def lrcc_residual_dev(ctx: Context, kind: int, t, x, comp: int = 0, prec: int = LRCC_FP64):
    """torch.complex128 CUDA tensors: t [n_amp] (or None), x [R, n_amp] -> new tensor."""
    import torch
    x = x.resolve_conj().contiguous()      # pass materialised values, never a lazy conj view
    if t is not None:
        t = t.resolve_conj().contiguous()
    assert x.is_cuda and x.dtype == torch.complex128
    R = x.shape[0]
    if kind == LRCC_RES_ENERGY:
        out = torch.empty(R, dtype=torch.complex128, device=x.device)
    else:
        out = torch.empty((R, ctx.n_amp), dtype=torch.complex128, device=x.device)
    tp = ctypes.c_void_p(t.data_ptr()) if t is not None else None
    ctx.check(library().lrcc_residual_dev(ctx.h, kind, tp, ctypes.c_void_p(x.data_ptr()), R, comp, prec,
                                          ctypes.c_void_p(out.data_ptr()), _stream_ptr()))
    return out


def lrcc_ladder_dev(ctx: Context, x, transpose: bool = False, prec: int = LRCC_FP64):
    """x: torch.complex128 CUDA [R, O, O, V, V] -> Z = 1/2 sum_ef <ab||ef> X_ij^ef."""
    import torch
    x = x.resolve_conj().contiguous()
    assert x.is_cuda and x.dtype == torch.complex128
    z = torch.empty_like(x)
    ctx.check(library().lrcc_ladder_dev(ctx.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                        x.shape[0], int(transpose), prec, _stream_ptr()))
    return z


def lrcc_ladder_packed_dev(ctx: Context, xt, transpose: bool = False, prec: int = LRCC_FP64, out=None):
    """xt: torch.complex128 CUDA [ncol, P_V] (pairs e<f) -> Zt [ncol, P_V],
    Zt[n][ab] = sum_{e<f} <ab||ef> Xt[n][ef]."""
    import torch
    xt = xt.resolve_conj().contiguous()
    assert xt.is_cuda and xt.dtype == torch.complex128 and xt.dim() == 2
    zt = torch.empty_like(xt) if out is None else out
    ctx.check(library().lrcc_ladder_packed_dev(ctx.h, ctypes.c_void_p(xt.data_ptr()),
                                               ctypes.c_void_p(zt.data_ptr()), xt.shape[0], int(transpose), prec,
                                               _stream_ptr()))
    return zt


def lrcc_ladder_noalloc(bvv, x, transpose: bool = False, out=None):
    """Ladder through the entry point that allocates nothing.  bvv: CUDA
    complex128 [L, V, V]; x: [R, O, O, V, V]; out (optional, preallocated by
    the caller) receives Z."""
    import torch
    bvv = bvv.resolve_conj().contiguous()
    x = x.resolve_conj().contiguous()
    z = torch.empty_like(x) if out is None else out
    R, O, _, V, _ = x.shape
    st = library().lrcc_ladder_noalloc(ctypes.c_void_p(bvv.data_ptr()), bvv.shape[0], O, V, R,
                                       ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                       int(transpose), _stream_ptr())
    if st != LRCC_OK:
        raise LrccError(st, library().lrcc_last_error(None).decode())
    return z


def lrcc_phase_times(ctx: Context) -> np.ndarray:
    ms = np.zeros(7)
    ctx.check(library().lrcc_phase_times(ctx.h, _cd(ms)))
    return ms


def lrcc_kernel_launches(ctx: Context) -> int:
    return int(library().lrcc_kernel_launches(ctx.h))


def lrcc_memory_stats(ctx: Context) -> tuple:
    """(live, peak, largest) bytes of ctx's device allocator."""
    v = [ctypes.c_int64(0) for _ in range(3)]
    ctx.check(library().lrcc_memory_stats(ctx.h, *[ctypes.byref(x) for x in v]))
    return tuple(int(x.value) for x in v)


def lrcc_get_amplitudes(ctx: Context, which: int = 0) -> np.ndarray:
    """which 0: T, 1: Lambda -> flat [O*V + O*O*V*V] complex."""
    out = np.zeros(ctx.n_amp, dtype=np.complex128)
    ctx.check(library().lrcc_get_amplitudes(ctx.h, which, _cd(out.view(np.float64))))
    return out


def lrcc_solve_counts(ctx: Context):
    a, b = ctypes.c_int(0), ctypes.c_int(0)
    ctx.check(library().lrcc_solve_counts(ctx.h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def lrcc_profile(ctx: Context, enable: bool) -> None:
    ctx.check(library().lrcc_profile(ctx.h, int(enable)))


def lrcc_profile_dump(ctx: Context, path: str) -> None:
    ctx.check(library().lrcc_profile_dump(ctx.h, path.encode()))


def lrcc_kernel_stats(ctx: Context) -> dict:
    """{name: dict(count, ms, flops, bytes)} aggregated over recorded launches."""
    out = {}
    i = 0
    while True:
        nm = ctypes.c_char_p()
        cnt = ctypes.c_int64()
        ms, fl, by = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        st = library().lrcc_kernel_stats(ctx.h, i, ctypes.byref(nm), ctypes.byref(cnt), ctypes.byref(ms),
                                         ctypes.byref(fl), ctypes.byref(by))
        if st != LRCC_OK:
            break
        out[nm.value.decode()] = dict(count=cnt.value, ms=ms.value, flops=fl.value, bytes=by.value)
        i += 1
    return out


def _make_residual_fn():
    import torch

    class ResidualFn(torch.autograd.Function):
        """R(T) of the CCSD equations on full amplitude arrays (device), with a
        backward that calls the library's transpose-Jacobian product.  For the
        holomorphic R, PyTorch's complex convention wants conj(J^T conj(g))."""

        @staticmethod
        def forward(ctx_, cc: Context, t):
            ctx_.cc = cc
            ctx_.save_for_backward(t)
            return lrcc_residual_dev(cc, LRCC_RES_T, None, t.reshape(1, -1).contiguous()).reshape(t.shape)

        @staticmethod
        def backward(ctx_, g):
            (t,) = ctx_.saved_tensors
            cc = ctx_.cc
            gt = lrcc_residual_dev(cc, LRCC_RES_VJP_FULL, t.reshape(-1).contiguous(),
                                   g.conj().reshape(1, -1).contiguous())
            return None, gt.conj().reshape(t.shape)

    return ResidualFn


_residual_fn = None


def ResidualFn():
    global _residual_fn
    if _residual_fn is None:
        _residual_fn = _make_residual_fn()
    return _residual_fn
