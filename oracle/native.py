"""ctypes wrappers of the C oracle (test infrastructure only).

``build()`` compiles ``csrc/oracle_unfold.c`` and ``csrc/oracle_rk4.c`` with gcc into
``oracle/_build/``.  ``unfold()`` returns the matrix of one Lindbladian term in the generator
basis as a scipy CSR matrix (Eq. 1, Eq. 6, Eq. 8: G_sm = Tr(F_s L(F_m)), K_s = Tr(F_s L(1/N))).
``rk4()`` is the classical RK4 map of Sec. IV step 3.1 on CSR matrices, the rows of every
stage shared out over the host's cores (OpenMP), for the long and large oracle runs.
"""
import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "oracle_unfold.c")
_LIB = os.path.join(_HERE, "_build", "liboracle_unfold.so")
_SRC_RK4 = os.path.join(_HERE, "csrc", "oracle_rk4.c")
_LIB_RK4 = os.path.join(_HERE, "_build", "liboracle_rk4.so")
_lib = None
_lib_rk4 = None


def build(force=False):
    """Compile the C oracle with gcc (portable flags: runs on x86-64 and aarch64)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", _LIB, "-lm"])
    if force or not os.path.exists(_LIB_RK4) or os.path.getmtime(_LIB_RK4) < os.path.getmtime(_SRC_RK4):
        # no contraction of a*b + c into fused multiply-adds, so the sums round like numpy's;
        # without OpenMP the same code runs on one thread
        base = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared", _SRC_RK4, "-o", _LIB_RK4]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:] + ["-lm"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base + ["-lm"])
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


def _load_rk4():
    global _lib_rk4
    if _lib_rk4 is None:
        build()
        lib = ctypes.CDLL(_LIB_RK4)
        P, L, D = ctypes.c_void_p, ctypes.c_longlong, ctypes.c_double
        lib.oracle_rk4.restype = ctypes.c_int
        lib.oracle_rk4.argtypes = [L, P, P, P, P, P, P, P, ctypes.c_int, D, D, D, P, D, D, L, L, P]
        lib.oracle_rk4_threads.restype = ctypes.c_int
        lib.oracle_rk4_threads.argtypes = []
        _lib_rk4 = lib
    return _lib_rk4


def rk4_threads():
    """Threads the C RK4 runs on (OpenMP's default: every host core unless OMP_NUM_THREADS)."""
    return int(_load_rk4().oracle_rk4_threads())


def _real_csr(X, D):
    X = sp.csr_matrix(X, dtype=np.float64)
    X.sort_indices()
    assert X.shape == (D, D)
    return (np.ascontiguousarray(X.indptr, dtype=np.int32), np.ascontiguousarray(X.indices, dtype=np.int32),
            np.ascontiguousarray(X.data, dtype=np.float64))


class Rk4System:
    """CSR arrays of dv/dt = (Q0 + eps(t) Q1) v + K prepared once for repeated ``run`` calls."""

    def __init__(self, Q0, Q1, K, D):
        self.D = D
        self.q0 = _real_csr(Q0, D)
        self.q1 = _real_csr(Q1, D) if Q1 is not None else (None, None, None)
        self.K = None if K is None else np.ascontiguousarray(K, dtype=np.float64)

    def run(self, E, A, omega, v0, h, nsteps, t0=0.0, emit_every=None, drive="sin"):
        """Classical RK4 (Sec. IV step 3.1) from v0; returns (v_final, v every ``emit_every`` steps)."""
        lib = _load_rk4()
        D = self.D
        v = np.array(v0, dtype=np.float64, copy=True)
        ne = int(nsteps) // int(emit_every) if emit_every else 0
        out = np.zeros((max(ne, 1), D))
        st = lib.oracle_rk4(D, *[_p(x) for x in self.q0], *[_p(x) for x in self.q1], _p(self.K),
                            0 if drive == "sin" else 1, float(E), float(A), float(omega), _p(v), float(t0), float(h),
                            int(nsteps), int(emit_every or 0), _p(out))
        if st != 0:
            raise MemoryError("oracle_rk4: allocation failed")
        return v, [out[i].copy() for i in range(ne)]


def rk4(Q0, Q1, K, E, A, omega, v0, h, nsteps, t0=0.0, emit_every=None, drive="sin"):
    """Classical RK4 on dv/dt = (Q0 + eps(t) Q1) v + K (Sec. IV step 3.1) in C over all host
    cores: the same map as ``propagate.rk4`` with eps(t) = E + A sin(omega t) ("sin") or the
    square drive of ``propagate.eps_square_step`` ("square").  Q1, K may be None.
    Returns (v_final, list of v every ``emit_every`` steps)."""
    return Rk4System(Q0, Q1, K, len(v0)).run(E, A, omega, v0, h, nsteps, t0=t0, emit_every=emit_every, drive=drive)
