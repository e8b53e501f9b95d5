"""ctypes wrapper of the sparse C oracle ``csrc/oracle_unfold.c`` (test infrastructure only).

``build()`` compiles it with gcc into ``oracle/_build/``; ``unfold()`` returns the
matrix of one Lindbladian term in the generator basis as a scipy CSR matrix
(Eq. 1, Eq. 6, Eq. 8: G_sm = Tr(F_s L(F_m)), K_s = Tr(F_s L(1/N))).
"""
import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "oracle_unfold.c")
_LIB = os.path.join(_HERE, "_build", "liboracle_unfold.so")
_lib = None


def build(force=False):
    """Compile the C oracle with gcc (portable flags: runs on x86-64 and aarch64)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", _LIB, "-lm"])
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        lib.oracle_unfold.restype = ctypes.c_longlong
        lib.oracle_unfold.argtypes = [ctypes.c_int, P, P, P, P, P, P, P, P, ctypes.c_double,
                                      P, ctypes.c_longlong, P, P, P, P, P]
        _lib = lib
    return _lib


def _csr_parts(X):
    if X is None:
        return None
    X = sp.csr_matrix(X, dtype=np.complex128)
    X.sort_indices()
    ptr = np.ascontiguousarray(X.indptr, dtype=np.int32)
    idx = np.ascontiguousarray(X.indices, dtype=np.int32)
    re = np.ascontiguousarray(X.data.real, dtype=np.float64)
    im = np.ascontiguousarray(X.data.imag, dtype=np.float64)
    return ptr, idx, re, im


def _p(a):
    return None if a is None else a.ctypes.data


def unfold(N, H=None, A=None, gamma=1.0, cols=None, want_k=True):
    """Matrix of X -> -i[H, X] + gamma (A X A^+ - 1/2 {A^+ A, X}) in the generator basis.

    Returns (G, K, max_imag): G a scipy CSR (N^2-1)^2 matrix (only the columns in
    ``cols`` when given), K the image of 1/N, max_imag the largest discarded
    imaginary part (rounding-sized for a Hermiticity-preserving map).
    """
    lib = _load()
    D = N * N - 1
    hp = _csr_parts(H)
    ap = _csr_parts(A)
    hargs = [_p(x) for x in hp] if hp else [None] * 4
    aargs = [_p(x) for x in ap] if ap else [None] * 4
    cols_arr = None if cols is None else np.ascontiguousarray(cols, dtype=np.int64)
    ncols = 0 if cols_arr is None else len(cols_arr)
    mx = np.zeros(1)
    n = lib.oracle_unfold(N, *hargs, *aargs, float(gamma), _p(cols_arr), ncols,
                          None, None, None, None, _p(mx))
    if n < 0:
        raise MemoryError("oracle_unfold: allocation failed")
    row = np.empty(max(n, 1), dtype=np.int32)
    col = np.empty(max(n, 1), dtype=np.int32)
    val = np.empty(max(n, 1), dtype=np.float64)
    K = np.empty(D, dtype=np.float64) if want_k else None
    n2 = lib.oracle_unfold(N, *hargs, *aargs, float(gamma), _p(cols_arr), ncols,
                           _p(row), _p(col), _p(val), _p(K), _p(mx))
    assert n2 == n
    G = sp.csr_matrix((val[:n], (row[:n], col[:n])), shape=(D, D))
    G.sort_indices()
    return G, K, float(mx[0])
