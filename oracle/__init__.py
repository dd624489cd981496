"""CPU oracle for block orthogonalization (arXiv:1806.01036, Sec. 4.2).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
CPU-baseline leg of the benchmark, never by the product path.  It shares no
code with the CUDA library.

The reference arithmetic lives in ``eo_oracle.c`` (IEEE binary128): every
result from its plain definition.  ``eo_oracle_fp64.c`` holds the paper's own
CPU arithmetic, plain FP64 and the double-double (Dot2) form, used to pin the
kappa^2 u versus kappa^2 u^2 behaviour on the CPU and as the timed CPU
baseline (functions ``fp64_*``).  This module compiles both on first use (gcc,
``-O2 -ffp-contract=off``, OpenMP when available) and wraps them for numpy
column-major FP64 arrays.  Results that the oracle keeps in binary128 come
back as (hi, lo) pairs of FP64 arrays with hi + lo equal to the binary128
value to about 2^-107 relative.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "eo_oracle.c"), os.path.join(_HERE, "eo_oracle_fp64.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_p = C.c_void_p
_i64 = C.c_int64
_int = C.c_int
_dbl = C.c_double


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (returns its path)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(s) for s in _SRCS + [__file__])):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=gnu11"]
    try:
        subprocess.run(base + ["-fopenmp"] + _SRCS + ["-o", tmp, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + _SRCS + ["-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.eoq_threads.restype = _int
            L.eoq_gram.argtypes = [_i64, _int, _p, _i64, _int, _p, _i64, _p, _p, _int]
            L.eoq_gram_f32.argtypes = [_i64, _int, _p, _i64, _int, _p, _i64, _p, _p, _int]
            L.eoq_project.argtypes = [_i64, _int, _p, _i64, _int, _p, _i64, _p, _i64, _p, _p, _int, _p, _p, _int]
            L.eoq_project_apply.argtypes = [_i64, _int, _p, _i64, _int, _p, _i64, _p, _p, _int, _p, _i64]
            L.eoq_cholesky.argtypes = [_int, _p, _p, _int, _p, _p, _int]
            L.eoq_cholesky.restype = _int
            L.eoq_triinv.argtypes = [_int, _p, _p, _int, _p, _p, _int]
            L.eoq_jacobi.argtypes = [_int, _p, _p, _int, _p, _int, _p, _p]
            L.eoq_svqb_z.argtypes = [_int, _p, _p, _int, _dbl, _p, _p, _int]
            L.eoq_svqb_z.restype = _int
            L.eoq_cholqr.argtypes = [_i64, _int, _p, _i64, _p, _p, _int, _int, _p, _p, _int]
            L.eoq_cholqr.restype = _int
            L.eoq_svqb.argtypes = [_i64, _int, _p, _i64, _p, _p, _int, _dbl, _int, _p, _p, _int]
            L.eoq_svqb.restype = _int
            L.eoq_svqb_rot.argtypes = [_i64, _int, _p, _i64, _p, _p, _int, _dbl, _p, _p, _int]
            L.eoq_svqb_rot.restype = _int
            L.eoq_orth_err.argtypes = [_i64, _int, _p, _i64, _p]
            L.eoq_orth_err_diag.argtypes = [_i64, _int, _p, _i64, _p, _p]
            L.eoq_cholqr_b.argtypes = [_i64, _int, _p, _i64, _p, _i64, _int, _p, _p, _int]
            L.eoq_cholqr_b.restype = _int
            L.eoq_svqb_b.argtypes = [_i64, _int, _p, _i64, _p, _i64, _dbl, _int, _p, _p, _int]
            L.eoq_svqb_b.restype = _int
            L.eoq_project_b.argtypes = [_i64, _int, _p, _i64, _p, _i64, _int, _p, _i64, _p, _i64, _p, _p, _int,
                                        _p, _p, _int]
            L.eoq_cross_err.argtypes = [_i64, _int, _p, _i64, _int, _p, _i64]
            L.eoq_cross_err.restype = _dbl
            L.eoq_fact_err.argtypes = [_i64, _int, _p, _i64, _p, _i64, _p, _p, _int]
            L.eoq_fact_err.restype = _dbl
            L.eoq_orthogonalize.argtypes = [_i64, _int, _p, _i64, _int, _p, _i64, _dbl, _int, _dbl, _p]
            L.eoq_orthogonalize.restype = _int
            L.eoq_set_threads.argtypes = [_int]
            L.eoq_cholqr_piv.argtypes = [_i64, _int, _p, _i64, _dbl, _int, _p, _p, _p, _p, _int]
            L.eoq_cholqr_piv.restype = _int
            L.eo64_gram.argtypes = [_int, _i64, _int, _p, _i64, _int, _p, _i64, _p, _p, _int]
            L.eo64_project.argtypes = [_int, _i64, _int, _p, _i64, _int, _p, _i64, _p, _i64, _p, _p, _int, _p, _p,
                                       _int]
            L.eo64_cholqr.argtypes = [_int, _i64, _int, _p, _i64, _p, _p, _int, _int, _p, _p, _int]
            L.eo64_cholqr.restype = _int
            _lib = L
    return _lib


def threads() -> int:
    return int(lib().eoq_threads())


def set_threads(t: int) -> None:
    """Threads of the oracle's later parallel loops (OpenMP)."""
    lib().eoq_set_threads(int(t))


def _f64(a) -> np.ndarray:
    a = np.asarray(a)
    if a.ndim == 1:
        a = a.reshape(-1, 1)
    return np.asfortranarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data


def _sq(k):
    return np.zeros((k, k), dtype=np.float64, order="F"), np.zeros((k, k), dtype=np.float64, order="F")


def gram(x, y=None):
    """(G_hi, G_lo) with G = X^T Y (Y = X when None) in binary128."""
    x = _f64(x)
    n, kx = x.shape
    if y is None:
        ky, yp, ldy = kx, None, 0
    else:
        y = _f64(y)
        assert y.shape[0] == n
        ky, yp, ldy = y.shape[1], y, n
    hi = np.zeros((kx, ky), order="F")
    lo = np.zeros((kx, ky), order="F")
    lib().eoq_gram(n, kx, _ptr(x), n, ky, _ptr(yp), ldy, _ptr(hi), _ptr(lo), kx)
    return hi, lo


def gram_f32(x, y=None):
    """Gram of FP32 inputs (widened exactly), binary128, returned as (hi, lo)."""
    x = np.asfortranarray(x, dtype=np.float32)
    n, kx = x.shape
    if y is None:
        ky, yp, ldy = kx, None, 0
    else:
        y = np.asfortranarray(y, dtype=np.float32)
        ky, yp, ldy = y.shape[1], y, n
    hi = np.zeros((kx, ky), order="F")
    lo = np.zeros((kx, ky), order="F")
    lib().eoq_gram_f32(n, kx, _ptr(x), n, ky, _ptr(yp), ldy, _ptr(hi), _ptr(lo), kx)
    return hi, lo


def project(v, y, with_gram=True):
    """Phase I projection.  Returns (Yt, (C_hi, C_lo), (M_hi, M_lo) or None).

    C = V^T Y and Yt = Y - V C in binary128 (Yt rounded once to FP64);
    M = Yt^T Yt of the rounded Yt."""
    v = _f64(v)
    y = _f64(y)
    n, kv = v.shape
    k = y.shape[1]
    yt = np.zeros((n, k), order="F")
    chi = np.zeros((kv, k), order="F")
    clo = np.zeros((kv, k), order="F")
    mhi, mlo = _sq(k) if with_gram else (None, None)
    lib().eoq_project(n, kv, _ptr(v), n, k, _ptr(y), n, _ptr(yt), n, _ptr(chi), _ptr(clo), kv,
                      _ptr(mhi), _ptr(mlo), k)
    return yt, (chi, clo), ((mhi, mlo) if with_gram else None)


def project_apply(v, y, c_hi, c_lo=None):
    """Yt = Y - V (C_hi + C_lo) in binary128, rounded once to FP64 (phase I with C given)."""
    v = _f64(v)
    y = _f64(y)
    n, kv = v.shape
    k = y.shape[1]
    c_hi = _f64(c_hi)
    c_lo = None if c_lo is None else _f64(c_lo)
    assert c_hi.shape == (kv, k)
    yt = np.zeros((n, k), order="F")
    lib().eoq_project_apply(n, kv, _ptr(v), n, k, _ptr(y), n, _ptr(c_hi), _ptr(c_lo), kv, _ptr(yt), n)
    return yt


def cholesky(m_hi, m_lo=None):
    """(R_hi, R_lo, info): M = R^T R in binary128; info = first failing pivot (1-based) or 0."""
    m_hi = _f64(m_hi)
    k = m_hi.shape[0]
    m_lo = None if m_lo is None else _f64(m_lo)
    r_hi, r_lo = _sq(k)
    info = lib().eoq_cholesky(k, _ptr(m_hi), _ptr(m_lo), k, _ptr(r_hi), _ptr(r_lo), k)
    return r_hi, r_lo, int(info)


def triinv(r_hi, r_lo=None):
    r_hi = _f64(r_hi)
    k = r_hi.shape[0]
    r_lo = None if r_lo is None else _f64(r_lo)
    z_hi, z_lo = _sq(k)
    lib().eoq_triinv(k, _ptr(r_hi), _ptr(r_lo), k, _ptr(z_hi), _ptr(z_lo), k)
    return z_hi, z_lo


def jacobi(m_hi, m_lo=None):
    """(lam (hi, lo), U): eigenpairs of the symmetric M by cyclic Jacobi in binary128."""
    m_hi = _f64(m_hi)
    k = m_hi.shape[0]
    m_lo = None if m_lo is None else _f64(m_lo)
    u = np.zeros((k, k), order="F")
    lh = np.zeros(k)
    ll = np.zeros(k)
    lib().eoq_jacobi(k, _ptr(m_hi), _ptr(m_lo), k, _ptr(u), k, _ptr(lh), _ptr(ll))
    return (lh, ll), u


def svqb_z(m_hi, m_lo=None, tol=0.0):
    """(Z_hi, Z_lo, rank): Z = M^{-1/2} (pseudo-inverse square root with cut tol)."""
    m_hi = _f64(m_hi)
    k = m_hi.shape[0]
    m_lo = None if m_lo is None else _f64(m_lo)
    z_hi, z_lo = _sq(k)
    rank = lib().eoq_svqb_z(k, _ptr(m_hi), _ptr(m_lo), k, float(tol), _ptr(z_hi), _ptr(z_lo), k)
    return z_hi, z_lo, int(rank)


def cholqr(x, passes=1, m=None):
    """(Q, (R_hi, R_lo), info): CholQR with `passes` passes in binary128, Q rounded per pass."""
    q = _f64(x).copy(order="F")
    n, k = q.shape
    r_hi, r_lo = _sq(k)
    mh, ml = (None, None) if m is None else (_f64(m[0]), None if m[1] is None else _f64(m[1]))
    info = lib().eoq_cholqr(n, k, _ptr(q), n, _ptr(mh), _ptr(ml), k, int(passes), _ptr(r_hi), _ptr(r_lo), k)
    return q, (r_hi, r_lo), int(info)


def svqb(x, passes=1, tol=0.0, m=None):
    """(Q, (Z_hi, Z_lo), rank): SVQB with Z = M^{-1/2} per pass, binary128."""
    q = _f64(x).copy(order="F")
    n, k = q.shape
    z_hi, z_lo = _sq(k)
    mh, ml = (None, None) if m is None else (_f64(m[0]), None if m[1] is None else _f64(m[1]))
    rank = lib().eoq_svqb(n, k, _ptr(q), n, _ptr(mh), _ptr(ml), k, float(tol), int(passes),
                          _ptr(z_hi), _ptr(z_lo), k)
    return q, (z_hi, z_lo), int(rank)


def svqb_rotated(x, tol=0.0, m=None):
    """(Q, (Z_hi, Z_lo), rank): one SVQB pass with Z = D U Lambda^{-1/2}
    (D = diag(M)^{-1/2}, D M D = U Lambda U^T, eigenvalues ascending, each
    eigenvector's largest entry positive), binary128."""
    q = _f64(x).copy(order="F")
    n, k = q.shape
    z_hi, z_lo = _sq(k)
    mh, ml = (None, None) if m is None else (_f64(m[0]), None if m[1] is None else _f64(m[1]))
    rank = lib().eoq_svqb_rot(n, k, _ptr(q), n, _ptr(mh), _ptr(ml), k, float(tol), _ptr(z_hi), _ptr(z_lo), k)
    return q, (z_hi, z_lo), int(rank)


def cholqr_b(x, p, passes=1):
    """(Q, BQ, (R_hi, R_lo), info): CholQR in the inner product <x, y>_B given
    P = B X (M = sym(X^T P); X and P both updated by Z = R^{-1}), binary128."""
    q = _f64(x).copy(order="F")
    bq = _f64(p).copy(order="F")
    n, k = q.shape
    r_hi, r_lo = _sq(k)
    info = lib().eoq_cholqr_b(n, k, _ptr(q), n, _ptr(bq), n, int(passes), _ptr(r_hi), _ptr(r_lo), k)
    return q, bq, (r_hi, r_lo), int(info)


def svqb_b(x, p, passes=1, tol=0.0):
    """(Q, BQ, (Z_hi, Z_lo), rank): SVQB in the inner product <x, y>_B given P = B X, binary128."""
    q = _f64(x).copy(order="F")
    bq = _f64(p).copy(order="F")
    n, k = q.shape
    z_hi, z_lo = _sq(k)
    rank = lib().eoq_svqb_b(n, k, _ptr(q), n, _ptr(bq), n, float(tol), int(passes), _ptr(z_hi), _ptr(z_lo), k)
    return q, bq, (z_hi, z_lo), int(rank)


def project_b(w, bw, x, p, with_gram=True):
    """(Xt, Pt, (C_hi, C_lo), (M_hi, M_lo) or None): B-projection against a
    B-orthonormal W with BW = B W: C = BW^T X, Xt = X - W C, Pt = P - BW C
    (rounded once), M = sym(Xt^T Pt), binary128."""
    w = _f64(w)
    bw = _f64(bw)
    xt = _f64(x).copy(order="F")
    pt = _f64(p).copy(order="F")
    n, kv = w.shape
    k = xt.shape[1]
    chi = np.zeros((kv, k), order="F")
    clo = np.zeros((kv, k), order="F")
    mhi, mlo = _sq(k) if with_gram else (None, None)
    lib().eoq_project_b(n, kv, _ptr(w), n, _ptr(bw), n, k, _ptr(xt), n, _ptr(pt), n, _ptr(chi), _ptr(clo), kv,
                        _ptr(mhi), _ptr(mlo), k)
    return xt, pt, (chi, clo), ((mhi, mlo) if with_gram else None)


def orth_err_diag(q, d):
    """(2-norm, Frobenius, max-abs) of Q^T diag(d) Q - I, binary128."""
    q = _f64(q)
    d = np.ascontiguousarray(d, dtype=np.float64)
    n, k = q.shape
    out = np.zeros(3)
    lib().eoq_orth_err_diag(n, k, _ptr(q), n, _ptr(d), _ptr(out))
    return tuple(float(v) for v in out)


def orth_err(q):
    """(2-norm, Frobenius, max-abs) of Q^T Q - I, computed in binary128."""
    q = _f64(q)
    n, k = q.shape
    out = np.zeros(3)
    lib().eoq_orth_err(n, k, _ptr(q), n, _ptr(out))
    return tuple(float(v) for v in out)


def cross_err(w, q):
    """||W^T Q||_2 in binary128."""
    w = _f64(w)
    q = _f64(q)
    n, kv = w.shape
    return float(lib().eoq_cross_err(n, kv, _ptr(w), n, q.shape[1], _ptr(q), n))


def fact_err(x, q, r_hi, r_lo=None):
    """||X - Q R||_F / ||X||_F in binary128 (R upper triangular, hi + lo)."""
    x = _f64(x)
    q = _f64(q)
    r_hi = _f64(r_hi)
    r_lo = None if r_lo is None else _f64(r_lo)
    n, k = x.shape
    return float(lib().eoq_fact_err(n, k, _ptr(x), n, _ptr(q), n, _ptr(r_hi), _ptr(r_lo), k))


def cholqr_piv(x, tol=0.0, passes=1):
    """(Q, perm, rank, (R_hi, R_lo), info): CholQR with a diagonally pivoted
    Cholesky stopped at the numerical rank (pivots whose remaining diagonal
    is not above tol * max_i M_ii are dropped), Q's columns beyond the rank
    zero, X[:, perm] ~ Q R; an unpivoted second pass on the kept columns when
    passes = 2.  binary128."""
    q = _f64(x).copy(order="F")
    n, k = q.shape
    perm = np.zeros(k, dtype=np.int32)
    rank = C.c_int(0)
    r_hi, r_lo = _sq(k)
    info = lib().eoq_cholqr_piv(n, k, _ptr(q), n, float(tol), int(passes), perm.ctypes.data, C.byref(rank),
                                _ptr(r_hi), _ptr(r_lo), k)
    return q, perm, int(rank.value), (r_hi, r_lo), int(info)


def orthogonalize(w, x, eps=1e-10, max_iter=8, tol=0.0):
    """(Q, iters, rank): the iterated two-phase algorithm in binary128 --
    phase I, then stop if max(||W^T Y||_F, ||Y^T Y - I||_F) <= eps, else SVQB
    (cut tol) -- repeated at most max_iter times; iters = SVQB updates applied
    before convergence, or -max_iter."""
    w = _f64(w)
    q = _f64(x).copy(order="F")
    n, kv = w.shape
    k = q.shape[1]
    rank = C.c_int(0)
    iters = lib().eoq_orthogonalize(n, kv, _ptr(w), n, k, _ptr(q), n, float(eps), int(max_iter), float(tol),
                                    C.byref(rank))
    return q, int(iters), int(rank.value)


# ------------------------------------------- the paper's CPU arithmetic

FP64, DD = 0, 1  # modes of the fp64_* functions: plain FP64, double-double (Dot2)


def fp64_gram(x, y=None, mode=DD):
    """(G_hi, G_lo): X^T Y in plain FP64 (row-ordered sums, G_lo = 0) or by Dot2."""
    x = _f64(x)
    n, kx = x.shape
    if y is None:
        ky, yp, ldy = kx, None, 0
    else:
        y = _f64(y)
        ky, yp, ldy = y.shape[1], y, n
    hi = np.zeros((kx, ky), order="F")
    lo = np.zeros((kx, ky), order="F")
    lib().eo64_gram(int(mode), n, kx, _ptr(x), n, ky, _ptr(yp), ldy, _ptr(hi), _ptr(lo), kx)
    return hi, lo


def fp64_project(v, y, mode=DD, with_gram=True):
    """(Yt, (C_hi, C_lo), (M_hi, M_lo) or None): phase I in plain FP64 or DD."""
    v = _f64(v)
    y = _f64(y)
    n, kv = v.shape
    k = y.shape[1]
    yt = np.zeros((n, k), order="F")
    chi = np.zeros((kv, k), order="F")
    clo = np.zeros((kv, k), order="F")
    mhi, mlo = _sq(k) if with_gram else (None, None)
    lib().eo64_project(int(mode), n, kv, _ptr(v), n, k, _ptr(y), n, _ptr(yt), n, _ptr(chi), _ptr(clo), kv,
                       _ptr(mhi), _ptr(mlo), k)
    return yt, (chi, clo), ((mhi, mlo) if with_gram else None)


def fp64_cholqr(x, passes=1, mode=DD, m=None):
    """(Q, (R_hi, R_lo), info): CholQR in plain FP64 or DD, Q rounded per pass."""
    q = _f64(x).copy(order="F")
    n, k = q.shape
    r_hi, r_lo = _sq(k)
    mh, ml = (None, None) if m is None else (_f64(m[0]), None if m[1] is None else _f64(m[1]))
    info = lib().eo64_cholqr(int(mode), n, k, _ptr(q), n, _ptr(mh), _ptr(ml), k, int(passes), _ptr(r_hi),
                             _ptr(r_lo), k)
    return q, (r_hi, r_lo), int(info)
