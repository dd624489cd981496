"""Python binding of libeo (include/eo.h): block orthogonalization on one GPU.

Argument marshalling only: every step runs in the library's CUDA kernels.
Matrices are torch tensors on the GPU in column-major layout, i.e. an n-by-k
matrix is a tensor of shape (n, k) with stride (1, ld), ld >= n (for example
``t.t()`` of a contiguous (k, n) tensor, or :func:`colmajor`).  Small k-by-k
results are returned as FP64 tensors (hi, lo) on the same device.

The library must have been built (``__graft_entry__.build()`` or
``python -m paper_1806_01036_gb300.build``); importing this module on a
machine without it raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

FP64, DD, F32, DD_EFT = 0, 1, 2, 3
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = range(6)
KMAX = 64

_lib = None
_p, _i64, _int, _dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double


class Block(C.Structure):
    """eo_block: one block of a batch (include/eo.h)."""
    _fields_ = [("n", _i64), ("k", _int), ("X", _p), ("ldx", _i64), ("Z_hi", _p), ("Z_lo", _p), ("ldz", _int)]


BATCH_SVQB, BATCH_CHOLQR = 0, 1
BATCH_NO_TUNE, BATCH_CHAINS = 1, 2


class EoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"eo status {status}: {msg}")
        self.status = status


def lib_path() -> str:
    return _build.LIB


def lib():
    """The loaded libeo.so (ctypes.CDLL) with argument types declared."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise ImportError(f"libeo.so is not built ({path}); run __graft_entry__.build()")
        L = C.CDLL(path)
        L.eo_version.restype = _int
        L.eo_kernel_launches.argtypes = [_p]
        L.eo_kernel_launches.restype = C.c_uint64
        L.eo_device_status.argtypes = [_p]
        L.eo_device_status.restype = _int
        L.eo_selftest_wait_timeout.argtypes = [_p, _dbl]
        L.eo_selftest_wait_timeout.restype = _int
        L.eo_create.argtypes = [C.POINTER(_p), _int]
        L.eo_destroy.argtypes = [_p]
        L.eo_set_stream.argtypes = [_p, _p]
        L.eo_last_error.argtypes = [_p]
        L.eo_last_error.restype = C.c_char_p
        L.eo_gram.argtypes = [_p, _i64, _int, _p, _i64, _int, _p, _i64, _p, _p, _int, _int]
        L.eo_project.argtypes = [_p, _i64, _int, _p, _i64, _int, _p, _i64, _p, _i64, _p, _p, _int, _p, _p, _int, _int]
        L.eo_project_apply.argtypes = [_p, _i64, _int, _p, _i64, _int, _p, _i64, _p, _i64, _p, _p, _int, _p, _p, _int,
                                       _int]
        L.eo_orthogonalize.argtypes = [_p, _i64, _int, _p, _i64, _int, _p, _i64, _dbl, _int, _dbl, _int, _p, _p]
        L.eo_cholqr.argtypes = [_p, _i64, _int, _p, _i64, _p, _p, _int, _p, _p, _int, _int, _int, _p]
        L.eo_svqb.argtypes = [_p, _i64, _int, _p, _i64, _p, _p, _int, _p, _p, _int, _dbl, _int, _int, _p]
        L.eo_svqb_rotated.argtypes = [_p, _i64, _int, _p, _i64, _p, _p, _int, _p, _p, _int, _dbl, _int, _p]
        L.eo_cholqr_piv.argtypes = [_p, _i64, _int, _p, _i64, _p, _p, _int, _dbl, _int, _int, _p, _p, _p]
        L.eo_gram_dd_noalloc.argtypes = [_i64, _int, _p, _i64, _int, _p, _i64, _p, _p, _int, _p]
        L.eo_cholqr_b.argtypes = [_p, _i64, _int, _p, _i64, _p, _i64, _p, _p, _int, _int, _int, _p]
        L.eo_svqb_b.argtypes = [_p, _i64, _int, _p, _i64, _p, _i64, _p, _p, _int, _dbl, _int, _int, _p]
        L.eo_project_b.argtypes = [_p, _i64, _int, _p, _i64, _p, _i64, _int, _p, _i64, _p, _i64, _p, _p, _int, _p,
                                   _p, _int, _int]
        L.eo_tune_cache.argtypes = [_p, C.c_char_p]
        L.eo_batch_create.argtypes = [_p, _int, C.POINTER(Block), _int, _dbl, _int, _int, _p, _int, _int,
                                      C.POINTER(_p)]
        L.eo_batch_run.argtypes = [_p]
        L.eo_batch_destroy.argtypes = [_p]
        L.eo_batch_tile.argtypes = [_p, _int, C.POINTER(_int), C.POINTER(_int)]
        L.eo_batch_passes.argtypes = [_p, _p]
        L.eo_batch_sweeps.argtypes = [_p, _p]
        _sz = C.c_size_t
        L.eo_server_create.argtypes = [_p, _sz, _int, C.POINTER(_p)]
        L.eo_server_destroy.argtypes = [_p]
        L.eo_server_add_basis.argtypes = [_p, _i64, _int, _p, _i64, C.POINTER(_int)]
        L.eo_server_submit.argtypes = [_p, _int, _int, _p, _i64, _p, _i64, _p, _p, _int, _p, C.POINTER(_i64)]
        L.eo_server_wait.argtypes = [_p, _i64, _dbl, C.POINTER(_int), C.POINTER(_dbl)]
        L.eo_server_poll.argtypes = [_p, _int, _p, _p, _p, _p, C.POINTER(_int)]
        L.eo_server_stats.argtypes = [_p, C.POINTER(_sz), C.POINTER(_sz), C.POINTER(_int), C.POINTER(_int),
                                      C.POINTER(_int), C.POINTER(C.c_uint64)]
        L.eo_admission_simulate.argtypes = [_sz, _int, _sz, _int, _p, _p, _p, _p, _p]
        L.eo_admission_simulate.restype = _int
        L.eo_batch_kernels.argtypes = [_p]
        L.eo_batch_kernels.restype = C.c_int64
        L.eo_batch_branches.argtypes = [_p]
        L.eo_batch_branches.restype = _int
        for f in ("eo_create", "eo_destroy", "eo_set_stream", "eo_gram", "eo_project", "eo_project_apply",
                  "eo_cholqr", "eo_svqb", "eo_svqb_rotated", "eo_cholqr_piv", "eo_orthogonalize", "eo_gram_dd_noalloc", "eo_tune_cache",
                  "eo_cholqr_b", "eo_svqb_b", "eo_project_b",
                  "eo_batch_create", "eo_batch_run", "eo_batch_destroy", "eo_batch_tile", "eo_batch_passes", "eo_batch_sweeps",
                  "eo_server_create", "eo_server_destroy", "eo_server_add_basis", "eo_server_submit",
                  "eo_server_wait", "eo_server_poll", "eo_server_stats"):
            getattr(L, f).restype = _int
        _lib = L
    return _lib


def colmajor(t):
    """Column-major copy (shape unchanged) of a 2-D tensor."""
    return t.t().contiguous().t()


def _mat(t, name, dtype=None):
    import torch
    if t.dim() == 1:
        t = t.reshape(-1, 1)
    if t.dim() != 2 or not t.is_cuda:
        raise ValueError(f"{name} must be a 2-D CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}")
    if t.shape[0] > 1 and t.stride(0) != 1:
        raise ValueError(f"{name} must be column-major (stride(0) == 1); use colmajor()")
    ld = t.stride(1) if t.shape[1] > 1 else max(1, t.shape[0])
    return t, int(t.shape[0]), int(t.shape[1]), int(max(ld, t.shape[0], 1))


def _ld(t):
    """Leading dimension of a column-major 2-D tensor (torch normalises the
    stride of a one-column tensor, so that one is taken from its rows)."""
    ld = t.stride(1) if t.shape[1] > 1 else max(1, t.shape[0])
    return int(max(ld, t.shape[0], 1))


def _dd_pair(pair, rows, cols, name, copy_ok):
    """(hi, lo, ld) of a double-double pair of rows x cols column-major FP64
    CUDA tensors (lo may be None) laid out with one leading dimension; an
    input pair with different layouts is copied to one (copy_ok), an output
    pair must already share one."""
    import torch
    hi, lo = pair
    hi, r, c, _ = _mat(hi, name + "_hi", torch.float64)
    if (r, c) != (rows, cols):
        raise ValueError(f"{name}_hi must be {rows} x {cols}")
    if lo is not None:
        lo, r2, c2, _ = _mat(lo, name + "_lo", torch.float64)
        if (r2, c2) != (rows, cols):
            raise ValueError(f"{name}_lo must be {rows} x {cols}")
        if _ld(lo) != _ld(hi):
            if not copy_ok:
                raise ValueError(f"{name}_hi and {name}_lo must share one leading dimension")
            hi, lo = colmajor(hi.clone()), colmajor(lo.clone())
    return hi, lo, _ld(hi)


def _small(k1, k2, device):
    import torch
    hi = torch.zeros((k2, k1), dtype=torch.float64, device=device).t()
    lo = torch.zeros((k2, k1), dtype=torch.float64, device=device).t()
    return hi, lo


class Context:
    """An eo_ctx bound to one device; calls run on torch's current stream."""

    def __init__(self, device: int = 0):
        h = _p()
        st = lib().eo_create(C.byref(h), int(device))
        if st != OK:
            raise EoError(st, "eo_create failed")
        self.h = h
        self.device = int(device)

    def close(self):
        if getattr(self, "h", None):
            lib().eo_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream=None):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        lib().eo_set_stream(self.h, C.c_void_p(s.cuda_stream))

    def device_status(self) -> int:
        """EO_OK, or EO_ETIMEOUT if a bounded device-side wait ran out since the
        last call (waits for the context's stream; clears the record)."""
        return int(lib().eo_device_status(self.h))

    def selftest_wait_timeout(self, seconds: float = 0.05):
        """Launch the one-thread kernel whose bounded wait runs out after `seconds`."""
        self.check(lib().eo_selftest_wait_timeout(self.h, float(seconds)))

    def launches(self) -> int:
        """Kernels this context has launched (eo_kernel_launches)."""
        return int(lib().eo_kernel_launches(self.h))

    def check(self, st: int):
        if st != OK:
            raise EoError(st, lib().eo_last_error(self.h).decode())

    def tune_cache(self, path=None):
        """Load (and later save) tuned launch shapes from a text file (eo_tune_cache)."""
        self.check(lib().eo_tune_cache(self.h, None if path is None else os.fsencode(path)))


def _dtype(prec):
    import torch
    return torch.float32 if prec == F32 else torch.float64


def gram(ctx: Context, X, Y=None, prec: int = DD, out=None):
    """(G_hi, G_lo) with G = X^T Y (Y = X when None)."""
    X, n, kx, ldx = _mat(X, "X", _dtype(prec))
    if Y is not None:
        Y, ny, ky, ldy = _mat(Y, "Y", _dtype(prec))
        if ny != n:
            raise ValueError("X and Y must have the same number of rows")
    else:
        ky, ldy = kx, ldx
    hi, lo, ldg = _dd_pair(out if out is not None else _small(kx, ky, X.device), kx, ky, "G", False)
    ctx.set_stream()
    ctx.check(lib().eo_gram(ctx.h, n, kx, X.data_ptr(), ldx, ky, None if Y is None else Y.data_ptr(), ldy,
                            hi.data_ptr(), None if lo is None else lo.data_ptr(), ldg, prec))
    return hi, lo


def project(ctx: Context, V, Y, Yout=None, prec: int = DD, want_m: bool = True):
    """(Yout, (C_hi, C_lo), (M_hi, M_lo) or None): Yout = Y - V (V^T Y), M = Yout^T Yout."""
    import torch
    V, n, kv, ldv = _mat(V, "V", torch.float64)
    Y, ny, k, ldy = _mat(Y, "Y", torch.float64)
    if ny != n:
        raise ValueError("V and Y must have the same number of rows")
    if Yout is None:
        Yout = colmajor(torch.empty((n, k), dtype=torch.float64, device=Y.device))
    Yout, _, _, ldyo = _mat(Yout, "Yout", torch.float64)
    ch, cl = _small(kv, k, V.device)
    mh, ml = _small(k, k, V.device) if want_m else (None, None)
    ctx.set_stream()
    ctx.check(lib().eo_project(ctx.h, n, kv, V.data_ptr(), ldv, k, Y.data_ptr(), ldy, Yout.data_ptr(), ldyo,
                               ch.data_ptr(), cl.data_ptr(), _ld(ch), None if mh is None else mh.data_ptr(),
                               None if ml is None else ml.data_ptr(), k, prec))
    return Yout, (ch, cl), ((mh, ml) if want_m else None)


def project_apply(ctx: Context, V, Y, C, Yout=None, prec: int = DD, want_m: bool = True):
    """(Yout, (M_hi, M_lo) or None): Yout = Y - V C for C = (C_hi, C_lo), M = Yout^T Yout."""
    import torch
    V, n, kv, ldv = _mat(V, "V", torch.float64)
    Y, ny, k, ldy = _mat(Y, "Y", torch.float64)
    if ny != n:
        raise ValueError("V and Y must have the same number of rows")
    ch, cl, ldc = _dd_pair(C, kv, k, "C", True)
    if Yout is None:
        Yout = colmajor(torch.empty((n, k), dtype=torch.float64, device=Y.device))
    Yout, _, _, ldyo = _mat(Yout, "Yout", torch.float64)
    mh, ml = _small(k, k, V.device) if want_m else (None, None)
    ctx.set_stream()
    ctx.check(lib().eo_project_apply(ctx.h, n, kv, V.data_ptr(), ldv, k, Y.data_ptr(), ldy, Yout.data_ptr(), ldyo,
                                     ch.data_ptr(), None if cl is None else cl.data_ptr(), ldc,
                                     None if mh is None else mh.data_ptr(), None if ml is None else ml.data_ptr(),
                                     k, prec))
    return Yout, ((mh, ml) if want_m else None)


def cholqr(ctx: Context, X, passes: int = 1, prec: int = DD, M=None, info=None):
    """In place X <- Q.  Returns (R_hi, R_lo, info) with info a device int32 tensor."""
    import torch
    X, n, k, ldx = _mat(X, "X", _dtype(prec))
    rh, rl = _small(k, k, X.device)
    if info is None:
        info = torch.zeros(1, dtype=torch.int32, device=X.device)
    mh, ml, ldm = None, None, k
    if M is not None:
        mh, ml, ldm = _dd_pair(M, k, k, "M", True)
    ctx.set_stream()
    ctx.check(lib().eo_cholqr(ctx.h, n, k, X.data_ptr(), ldx, None if mh is None else mh.data_ptr(),
                              None if ml is None else ml.data_ptr(), ldm, rh.data_ptr(), rl.data_ptr(), _ld(rh),
                              int(passes), prec, info.data_ptr()))
    return rh, rl, info


def svqb(ctx: Context, X, passes: int = 1, prec: int = DD, tol: float = -1.0, M=None, rank=None):
    """In place X <- X Z.  Returns (Z_hi, Z_lo, rank) with rank a device int32 tensor."""
    import torch
    X, n, k, ldx = _mat(X, "X", _dtype(prec))
    zh, zl = _small(k, k, X.device)
    if rank is None:
        rank = torch.zeros(1, dtype=torch.int32, device=X.device)
    mh, ml, ldm = None, None, k
    if M is not None:
        mh, ml, ldm = _dd_pair(M, k, k, "M", True)
    ctx.set_stream()
    ctx.check(lib().eo_svqb(ctx.h, n, k, X.data_ptr(), ldx, None if mh is None else mh.data_ptr(),
                            None if ml is None else ml.data_ptr(), ldm, zh.data_ptr(), zl.data_ptr(), _ld(zh),
                            float(tol), int(passes), prec, rank.data_ptr()))
    return zh, zl, rank


def svqb_rotated(ctx: Context, X, prec: int = DD, tol: float = -1.0, M=None, rank=None):
    """One pass of X <- X Z with Z = D U Lambda^{-1/2} (D = diag(M)^{-1/2},
    eigenvalues ascending, each eigenvector's largest entry positive).
    Returns (Z_hi, Z_lo, rank) with rank a device int32 tensor."""
    import torch
    X, n, k, ldx = _mat(X, "X", _dtype(prec))
    zh, zl = _small(k, k, X.device)
    if rank is None:
        rank = torch.zeros(1, dtype=torch.int32, device=X.device)
    mh, ml, ldm = None, None, k
    if M is not None:
        mh, ml, ldm = _dd_pair(M, k, k, "M", True)
    ctx.set_stream()
    ctx.check(lib().eo_svqb_rotated(ctx.h, n, k, X.data_ptr(), ldx, None if mh is None else mh.data_ptr(),
                                    None if ml is None else ml.data_ptr(), ldm, zh.data_ptr(), zl.data_ptr(),
                                    _ld(zh), float(tol), prec, rank.data_ptr()))
    return zh, zl, rank


def cholqr_piv(ctx: Context, X, passes: int = 1, prec: int = DD, tol: float = -1.0):
    """Pivoted, partial CholQR of X (in place): X <- Q with its first `rank`
    columns orthonormal and the rest zero, X_in[:, perm] ~ Q R.  Returns
    (R_hi, R_lo, perm, rank, info) as device tensors."""
    import torch
    X, n, k, ldx = _mat(X, "X", torch.float64)
    rh, rl = _small(k, k, X.device)
    perm = torch.zeros(k, dtype=torch.int32, device=X.device)
    rank = torch.zeros(1, dtype=torch.int32, device=X.device)
    info = torch.zeros(1, dtype=torch.int32, device=X.device)
    ctx.set_stream()
    ctx.check(lib().eo_cholqr_piv(ctx.h, n, k, X.data_ptr(), ldx, rh.data_ptr(), rl.data_ptr(), _ld(rh),
                                  float(tol), int(passes), prec, perm.data_ptr(), rank.data_ptr(), info.data_ptr()))
    return rh, rl, perm, rank, info


def cholqr_b(ctx: Context, X, BX, passes: int = 1, prec: int = DD, info=None):
    """CholQR in the B-inner product, given BX = B X: in place X <- Q,
    BX <- B Q.  Returns (R_hi, R_lo, info)."""
    import torch
    X, n, k, ldx = _mat(X, "X", _dtype(prec))
    BX, nb, kb, ldbx = _mat(BX, "BX", _dtype(prec))
    if (nb, kb) != (n, k):
        raise ValueError("X and BX must have the same shape")
    rh, rl = _small(k, k, X.device)
    if info is None:
        info = torch.zeros(1, dtype=torch.int32, device=X.device)
    ctx.set_stream()
    ctx.check(lib().eo_cholqr_b(ctx.h, n, k, X.data_ptr(), ldx, BX.data_ptr(), ldbx, rh.data_ptr(), rl.data_ptr(),
                                _ld(rh), int(passes), prec, info.data_ptr()))
    return rh, rl, info


def svqb_b(ctx: Context, X, BX, passes: int = 1, prec: int = DD, tol: float = -1.0, rank=None):
    """SVQB in the B-inner product, given BX = B X: in place X <- X Z,
    BX <- BX Z.  Returns (Z_hi, Z_lo, rank)."""
    import torch
    X, n, k, ldx = _mat(X, "X", _dtype(prec))
    BX, nb, kb, ldbx = _mat(BX, "BX", _dtype(prec))
    if (nb, kb) != (n, k):
        raise ValueError("X and BX must have the same shape")
    zh, zl = _small(k, k, X.device)
    if rank is None:
        rank = torch.zeros(1, dtype=torch.int32, device=X.device)
    ctx.set_stream()
    ctx.check(lib().eo_svqb_b(ctx.h, n, k, X.data_ptr(), ldx, BX.data_ptr(), ldbx, zh.data_ptr(), zl.data_ptr(),
                              _ld(zh), float(tol), int(passes), prec, rank.data_ptr()))
    return zh, zl, rank


def project_b(ctx: Context, W, BW, Y, BY, prec: int = DD, want_m: bool = True):
    """B-projection in place: C = BW^T Y, Y <- Y - W C, BY <- BY - BW C.
    Returns ((C_hi, C_lo), (M_hi, M_lo) or None) with M = sym(Y^T BY)."""
    import torch
    W, n, kv, ldw = _mat(W, "W", torch.float64)
    BW, n2, kv2, ldbw = _mat(BW, "BW", torch.float64)
    Y, n3, k, ldy = _mat(Y, "Y", torch.float64)
    BY, n4, k2, ldby = _mat(BY, "BY", torch.float64)
    if not (n == n2 == n3 == n4 and kv == kv2 and k == k2):
        raise ValueError("W, BW and Y, BY must match in shape")
    ch, cl = _small(kv, k, W.device)
    mh, ml = _small(k, k, W.device) if want_m else (None, None)
    ctx.set_stream()
    ctx.check(lib().eo_project_b(ctx.h, n, kv, W.data_ptr(), ldw, BW.data_ptr(), ldbw, k, Y.data_ptr(), ldy,
                                 BY.data_ptr(), ldby, ch.data_ptr(), cl.data_ptr(), _ld(ch),
                                 None if mh is None else mh.data_ptr(), None if ml is None else ml.data_ptr(), k,
                                 prec))
    return (ch, cl), ((mh, ml) if want_m else None)


def orthogonalize(ctx: Context, V, Y, eps: float = 1e-10, max_iter: int = 8, prec: int = DD, tol: float = -1.0):
    """Iterated two-phase orthogonalization of Y (in place) against V and
    among its columns.  Returns (iters, rank) as device int32 tensors."""
    import torch
    V, n, kv, ldv = _mat(V, "V", torch.float64)
    Y, ny, k, ldy = _mat(Y, "Y", torch.float64)
    if ny != n:
        raise ValueError("V and Y must have the same number of rows")
    iters = torch.zeros(1, dtype=torch.int32, device=Y.device)
    rank = torch.zeros(1, dtype=torch.int32, device=Y.device)
    ctx.set_stream()
    ctx.check(lib().eo_orthogonalize(ctx.h, n, kv, V.data_ptr(), ldv, k, Y.data_ptr(), ldy, float(eps),
                                     int(max_iter), float(tol), prec, iters.data_ptr(), rank.data_ptr()))
    return iters, rank


NOALLOC_KMAX = 16
NOALLOC_NMAX = 152 << 22  # rows: 152 row chunks of at most 2^22 rows


def gram_dd_noalloc(X, Y=None, out=None):
    """(G_hi, G_lo) = X^T Y in EO_DD through eo_gram_dd_noalloc (no context,
    no device allocation inside the library; kx, ky <= 16).  Runs on torch's
    current stream and device."""
    import torch
    X, n, kx, ldx = _mat(X, "X", torch.float64)
    if Y is not None:
        Y, ny, ky, ldy = _mat(Y, "Y", torch.float64)
        if ny != n:
            raise ValueError("X and Y must have the same number of rows")
    else:
        ky, ldy = kx, ldx
    hi, lo, ldg = _dd_pair(out if out is not None else _small(kx, ky, X.device), kx, ky, "G", False)
    st = lib().eo_gram_dd_noalloc(n, kx, X.data_ptr(), ldx, ky, None if Y is None else Y.data_ptr(), ldy,
                                  hi.data_ptr(), None if lo is None else lo.data_ptr(), ldg,
                                  C.c_void_p(torch.cuda.current_stream(X.device).cuda_stream))
    if st != OK:
        raise EoError(st, "eo_gram_dd_noalloc failed")
    return hi, lo


class Batch:
    """Many blocks orthogonalized by one CUDA graph launch (eo_batch_create).

    blocks: list of column-major CUDA tensors X_b (n_b x k_b; FP64, or FP32
    with prec F32), orthogonalized in place by each run().  method:
    BATCH_SVQB or BATCH_CHOLQR.  want_z: also return each block's Z (SVQB)
    or R (CholQR) as a (hi, lo) pair.  chains: each block's whole sequence on
    its branch instead of the phase order.  out: device int32 tensor with one
    rank (SVQB) or info (CholQR) per block.  The tensors must outlive the
    batch (the graph holds their addresses)."""

    def __init__(self, ctx: Context, blocks, method: int = BATCH_SVQB, passes: int = 0, prec: int = DD,
                 tol: float = -1.0, branches: int = 0, tune: bool = True, want_z: bool = False,
                 chains: bool = False):
        import torch
        if not blocks:
            raise ValueError("a batch needs at least one block")
        self.ctx = ctx
        self.blocks = []
        self.z = []
        desc = (Block * len(blocks))()
        for i, X in enumerate(blocks):
            X, n, k, ldx = _mat(X, f"blocks[{i}]", _dtype(prec))
            self.blocks.append(X)
            zh = zl = None
            if want_z:
                zh, zl = _small(k, k, X.device)
                self.z.append((zh, zl))
            desc[i] = Block(n, k, X.data_ptr(), ldx, None if zh is None else zh.data_ptr(),
                            None if zl is None else zl.data_ptr(), k)
        self.out = torch.zeros(len(blocks), dtype=torch.int32, device=self.blocks[0].device)
        h = _p()
        ctx.check(lib().eo_batch_create(ctx.h, len(blocks), desc, int(method), float(tol), int(passes), int(prec),
                                        self.out.data_ptr(), int(branches),
                                        (0 if tune else BATCH_NO_TUNE) | (BATCH_CHAINS if chains else 0),
                                        C.byref(h)))
        self.h = h

    def run(self):
        """Enqueue one graph launch on torch's current stream."""
        self.ctx.set_stream()
        self.ctx.check(lib().eo_batch_run(self.h))

    def tile(self, i: int):
        """(gram_ctas, row_ctas) caps chosen for block i (0 = default)."""
        g, r = _int(), _int()
        self.ctx.check(lib().eo_batch_tile(self.h, int(i), C.byref(g), C.byref(r)))
        return g.value, r.value

    def passes(self):
        """Passes each block took in the last run (list of 1 or 2); waits for the stream."""
        out = (_int * len(self.blocks))()
        self.ctx.set_stream()
        self.ctx.check(lib().eo_batch_passes(self.h, C.cast(out, _p)))
        return list(out)

    def sweeps(self):
        """Jacobi sweeps of each block's last SVQB eigensolve (0 for CholQR)."""
        out = (_int * len(self.blocks))()
        self.ctx.set_stream()
        self.ctx.check(lib().eo_batch_sweeps(self.h, C.cast(out, _p)))
        return list(out)

    def kernels(self) -> int:
        return int(lib().eo_batch_kernels(self.h))

    def branches(self) -> int:
        return int(lib().eo_batch_branches(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.ctx.set_stream()
            lib().eo_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request server (eo_server_*): resident bases, blocks orthogonalized
    against them (projection + compensated CholQR) on `slots` concurrent
    streams under a device-memory budget (bytes)."""

    def __init__(self, ctx: Context, budget: int, slots: int = 16):
        h = _p()
        ctx.check(lib().eo_server_create(ctx.h, int(budget), int(slots), C.byref(h)))
        self.ctx = ctx
        self.h = h
        self.bases = []

    def add_basis(self, V) -> int:
        """Register a resident column-major FP64 basis; returns its id."""
        import torch
        V, n, kv, ldv = _mat(V, "V", torch.float64)
        bid = _int()
        self.ctx.check(lib().eo_server_add_basis(self.h, n, kv, V.data_ptr(), ldv, C.byref(bid)))
        self.bases.append(V)
        return bid.value

    def submit(self, basis: int, Y, Yout=None, R=None, info=None) -> int:
        """Queue Yout = CholQR(Y - V V^T Y); returns the request id.  R: optional
        (hi, lo) k-by-k pair; info: optional device int32 tensor."""
        import torch
        Y, n, k, ldy = _mat(Y, "Y", torch.float64)
        Yout = Y if Yout is None else Yout
        Yout, _, _, ldyo = _mat(Yout, "Yout", torch.float64)
        rh = rl = None
        ldr = k
        if R is not None:
            rh, rl, ldr = _dd_pair(R, k, k, "R", False)
        rid = _i64()
        self.ctx.check(lib().eo_server_submit(self.h, int(basis), k, Y.data_ptr(), ldy, Yout.data_ptr(), ldyo,
                                              None if rh is None else rh.data_ptr(),
                                              None if rl is None else rl.data_ptr(), ldr,
                                              None if info is None else info.data_ptr(), C.byref(rid)))
        return rid.value

    def wait(self, rid: int, timeout: float = 60.0):
        """(status, latency_ms) of a request, waiting for it."""
        st, lat = _int(), _dbl()
        self.ctx.check(lib().eo_server_wait(self.h, int(rid), float(timeout), C.byref(st), C.byref(lat)))
        return st.value, lat.value

    def poll(self, max_out: int = 4096):
        """Completed requests not yet reported: list of (id, latency_ms, queue_ms, status)."""
        ids = (_i64 * max_out)()
        lat = (_dbl * max_out)()
        qms = (_dbl * max_out)()
        sts = (_int * max_out)()
        n = _int()
        self.ctx.check(lib().eo_server_poll(self.h, max_out, C.cast(ids, _p), C.cast(lat, _p), C.cast(qms, _p),
                                            C.cast(sts, _p), C.byref(n)))
        return [(ids[i], lat[i], qms[i], sts[i]) for i in range(n.value)]

    def stats(self):
        r, p = C.c_size_t(), C.c_size_t()
        pr, q, ru = _int(), _int(), _int()
        kn = C.c_uint64()
        self.ctx.check(lib().eo_server_stats(self.h, C.byref(r), C.byref(p), C.byref(pr), C.byref(q), C.byref(ru),
                                             C.byref(kn)))
        return {"resident": r.value, "peak_inflight": p.value, "peak_running": pr.value, "queued": q.value,
                "running": ru.value, "kernels": kn.value}

    def close(self):
        if getattr(self, "h", None):
            lib().eo_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def admission_simulate(budget, slots, resident, basis, nbytes, arrival, duration):
    """The server's admission policy on the host (eo_admission_simulate):
    returns (start times, peak running).  No GPU needed."""
    import numpy as np
    n = len(basis)
    b = np.ascontiguousarray(basis, dtype=np.int32)
    by = np.ascontiguousarray(nbytes, dtype=np.int64)
    a = np.ascontiguousarray(arrival, dtype=np.float64)
    d = np.ascontiguousarray(duration, dtype=np.float64)
    start = np.zeros(n, dtype=np.float64)
    peak = lib().eo_admission_simulate(int(budget), int(slots), int(resident), n, b.ctypes.data, by.ctypes.data,
                                       a.ctypes.data, d.ctypes.data, start.ctypes.data)
    if peak < 0:
        raise ValueError("bad arguments to eo_admission_simulate")
    return start, peak
