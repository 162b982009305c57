"""Oracle: plain sequential FP64 CPU solvers for the structured systems of
Amodio & Brugnano, "Parallel Factorizations in Numerical Analysis".

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library under ``paper_0912_3678_gb300``) never imports it, and the
two share no code: no kernels, headers, helpers or constants.

What the partition method computes is the unique solution x = A^{-1} f of the
nonsingular structured system A x = f (Sec. 2, Eq. (syst)); the factorization
A = F T G of Eq. (parfact) is exact, so the method reaches that solution up to
rounding.  The oracle writes the definition out with textbook sequential
algorithms in plain C (``oracle.c``, FP64, -ffp-contract=off, no BLAS):

* ``tri_solve``    scalar tridiagonal, Thomas algorithm (LU, no pivoting);
* ``btri_solve``   block tridiagonal, block Thomas with m x m GEPP pivots;
* ``babd_solve``   lower block bidiagonal + upper-right corner (BABD,
                   Sec. 2, Eq. (parpart1) with c = 0), GEPP restricted to the
                   rows that are nonzero in each pivot column;
* ``dense_solve``  dense GEPP (brute force for tiny cases);
* ``*_residual``   r = f - A x.

``oracle.partition`` adds the quantities of the partition method itself
(reduced matrix, F/T/G factors) by their plain definitions, for small cases.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with gcc into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(ctypes.c_double)
            i64, i32 = ctypes.c_int64, ctypes.c_int
            sigs = {
                "oracle_dense_solve": [i32, P, P, P, i32],
                "oracle_tri_solve": [i64, P, P, P, P, P, i32],
                "oracle_tri_residual": [i64, P, P, P, P, P, P, i32],
                "oracle_btri_solve": [i64, i32, P, P, P, P, P, i32],
                "oracle_btri_residual": [i64, i32, P, P, P, P, P, P, i32],
                "oracle_babd_solve": [i64, i32, P, P, P, P, P, P, i32],
                "oracle_babd_residual": [i64, i32, P, P, P, P, P, P, P, i32],
            }
            for name, args in sigs.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            _lib = lib
    return _lib


class SingularError(ArithmeticError):
    """A zero pivot was met: the input is singular for this algorithm."""


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _rhs2d(f, rows):
    f = _f64(f)
    vec = f.ndim == 1
    f2 = f.reshape(rows, -1)
    return f2, vec


def _check(rc, what):
    if rc == -1:
        raise SingularError(f"{what}: zero pivot")
    if rc != 0:
        raise ValueError(f"{what}: invalid sizes (rc={rc})")


def dense_solve(A, f):
    """x = A^{-1} f by dense Gaussian elimination with partial pivoting."""
    A = _f64(A)
    n = A.shape[0]
    f2, vec = _rhs2d(f, n)
    x = np.empty_like(f2)
    _check(_load().oracle_dense_solve(n, _ptr(A), _ptr(f2), _ptr(x), f2.shape[1]), "dense_solve")
    return x.reshape(-1) if vec else x


def tri_solve(dl, d, du, f):
    """Thomas algorithm for dl[i] x[i-1] + d[i] x[i] + du[i] x[i+1] = f[i]."""
    dl, d, du = _f64(dl), _f64(d), _f64(du)
    n = d.shape[0]
    f2, vec = _rhs2d(f, n)
    x = np.empty_like(f2)
    _check(_load().oracle_tri_solve(n, _ptr(dl), _ptr(d), _ptr(du), _ptr(f2), _ptr(x), f2.shape[1]),
           "tri_solve")
    return x.reshape(-1) if vec else x


def tri_residual(dl, d, du, x, f):
    dl, d, du = _f64(dl), _f64(d), _f64(du)
    n = d.shape[0]
    f2, vec = _rhs2d(f, n)
    x2, _ = _rhs2d(x, n)
    r = np.empty_like(f2)
    _check(_load().oracle_tri_residual(n, _ptr(dl), _ptr(d), _ptr(du), _ptr(x2), _ptr(f2), _ptr(r),
                                       f2.shape[1]), "tri_residual")
    return r.reshape(-1) if vec else r


def btri_solve(B, D, C, F):
    """Block Thomas for B_j x_{j-1} + D_j x_j + C_j x_{j+1} = f_j.

    B, D, C: [N, m, m]; F: [N*m] or [N*m, nrhs] (or [N, m, nrhs]).
    Returns X shaped like F (2-D [N*m, nrhs] unless F was 1-D)."""
    B, D, C = _f64(B), _f64(D), _f64(C)
    N, m = D.shape[0], D.shape[1]
    F = _f64(F)
    vec = F.ndim == 1
    F2 = F.reshape(N * m, -1)
    X = np.empty_like(F2)
    _check(_load().oracle_btri_solve(N, m, _ptr(B), _ptr(D), _ptr(C), _ptr(F2), _ptr(X), F2.shape[1]),
           "btri_solve")
    return X.reshape(-1) if vec else X


def btri_residual(B, D, C, X, F):
    B, D, C = _f64(B), _f64(D), _f64(C)
    N, m = D.shape[0], D.shape[1]
    F = _f64(F)
    vec = F.ndim == 1
    F2 = F.reshape(N * m, -1)
    X2 = _f64(X).reshape(N * m, -1)
    R = np.empty_like(F2)
    _check(_load().oracle_btri_residual(N, m, _ptr(B), _ptr(D), _ptr(C), _ptr(X2), _ptr(F2), _ptr(R),
                                        F2.shape[1]), "btri_residual")
    return R.reshape(-1) if vec else R


def babd_solve(S, R, B0, B1, RHS):
    """Solve B0 y_0 + B1 y_N = beta;  S_j y_j + R_j y_{j+1} = r_j (j < N).

    S, R: [N, m, m]; B0, B1: [m, m]; RHS: [(N+1)*m] or [(N+1)*m, nrhs] with
    beta first.  Returns Y shaped like RHS."""
    S, R, B0, B1 = _f64(S), _f64(R), _f64(B0), _f64(B1)
    N, m = S.shape[0], S.shape[1]
    RHS = _f64(RHS)
    vec = RHS.ndim == 1
    F2 = RHS.reshape((N + 1) * m, -1)
    Y = np.empty_like(F2)
    _check(_load().oracle_babd_solve(N, m, _ptr(S), _ptr(R), _ptr(B0), _ptr(B1), _ptr(F2), _ptr(Y),
                                     F2.shape[1]), "babd_solve")
    return Y.reshape(-1) if vec else Y


def babd_residual(S, R, B0, B1, Y, RHS):
    S, R, B0, B1 = _f64(S), _f64(R), _f64(B0), _f64(B1)
    N, m = S.shape[0], S.shape[1]
    RHS = _f64(RHS)
    vec = RHS.ndim == 1
    F2 = RHS.reshape((N + 1) * m, -1)
    Y2 = _f64(Y).reshape((N + 1) * m, -1)
    Rout = np.empty_like(F2)
    _check(_load().oracle_babd_residual(N, m, _ptr(S), _ptr(R), _ptr(B0), _ptr(B1), _ptr(Y2), _ptr(F2),
                                        _ptr(Rout), F2.shape[1]), "babd_residual")
    return Rout.reshape(-1) if vec else Rout


def rel_err(X, Xref):
    """Normwise relative error ||X - Xref||_F / ||Xref||_F over all entries."""
    X = np.asarray(X, dtype=np.float64)
    Xref = np.asarray(Xref, dtype=np.float64)
    den = np.linalg.norm(Xref.ravel())
    return float(np.linalg.norm((X - Xref).ravel()) / (den if den > 0 else 1.0))
