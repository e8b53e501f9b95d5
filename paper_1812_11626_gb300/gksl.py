"""Thin ctypes binding of libgksl (include/gksl.h): argument marshalling only.

Every ``gksl_*`` function below has the name and argument order of the C entry point.
Array arguments may be numpy arrays (host memory) or CUDA torch tensors (device memory of
the context's GPU); the library decides which by the pointer.  A non-OK status raises
``GkslError`` with the library's message.  There is no fallback: if the shared library is
missing, importing this module raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgksl.so")

GKSL_OK, GKSL_ERR_ARG, GKSL_ERR_CUDA, GKSL_ERR_OOM, GKSL_ERR_STATE, GKSL_ERR_UNSTABLE, GKSL_ERR_DIVERGED, \
    GKSL_ERR_TIMEOUT = range(8)
STATUS_NAMES = ["OK", "ERR_ARG", "ERR_CUDA", "ERR_OOM", "ERR_STATE", "ERR_UNSTABLE", "ERR_DIVERGED", "ERR_TIMEOUT"]
GKSL_MAX_H0 = 8
GKSL_MAX_P = 8
GKSL_STRUCT_F, GKSL_STRUCT_D = 0, 1
GKSL_ASM_FP32, GKSL_ASM_TRANSPOSE, GKSL_ASM_NO_DROP, GKSL_ASM_MATRIX_FREE, GKSL_ASM_NO_FOLD = 1, 2, 4, 8, 16
GKSL_ASM_WIDE_COLUMNS = 32
GKSL_ASM_DENSE_DISSIPATORS = 64
GKSL_MAT_Q0, GKSL_MAT_Q1, GKSL_MAT_H0, GKSL_MAT_R = 0, 1, 16, 32

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libgksl is not built ({LIB_PATH} missing): run __graft_entry__.build() first")
_lib = ctypes.CDLL(LIB_PATH)


class GkslError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"GKSL_{name}: {message}")


class gksl_info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("D", ctypes.c_longlong), ("nnz_q0", ctypes.c_longlong),
                ("nnz_q1", ctypes.c_longlong), ("nnz_r", ctypes.c_longlong * GKSL_MAX_P),
                ("ell_width_q0", ctypes.c_int), ("ell_width_q1", ctypes.c_int), ("long_rows", ctypes.c_longlong),
                ("device_bytes", ctypes.c_longlong), ("assemble_seconds", ctypes.c_double),
                ("max_abs_q0", ctypes.c_double), ("rk4_variant", ctypes.c_int * 2),
                ("rk4_variant_us", (ctypes.c_double * 4) * 2), ("q1_folded", ctypes.c_int),
                ("compact_columns", ctypes.c_int * 2), ("compact_escaped_rows", ctypes.c_longlong),
                ("tail_nnz", ctypes.c_longlong), ("rk4_compact", ctypes.c_int * 2),
                ("rk4_variant_us_c16", (ctypes.c_double * 4) * 2)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_L = ctypes.c_longlong
_D = ctypes.c_double
_U = ctypes.c_uint
_S = ctypes.c_int  # gksl_status

_SIGS = {
    "gksl_create": (_S, [_I, _I, _P, ctypes.POINTER(_P)]),
    "gksl_destroy": (None, [_P]),
    "gksl_last_error": (ctypes.c_char_p, [_P]),
    "gksl_set_h0_component": (_S, [_P, _I, _D, _P, _P, _P, _P, _I]),
    "gksl_set_theta": (_S, [_P, _I, _D]),
    "gksl_set_h1": (_S, [_P, _P, _P, _P, _P, _I]),
    "gksl_set_dissipator": (_S, [_P, _I, _D, _P, _P, _P, _P, _I]),
    "gksl_set_gamma": (_S, [_P, _I, _D]),
    "gksl_set_drive": (_S, [_P, _D, _D, _D]),
    "gksl_set_drive_shape": (_S, [_P, _I]),
    "gksl_set_kossakowski": (_S, [_P, _P, _P, _D]),
    "gksl_expand": (_S, [_P, _P, _P, _P, _P, _I, _P, _P]),
    "gksl_structure_count": (_S, [_I, _I, ctypes.POINTER(_L)]),
    "gksl_structure_enumerate": (_S, [_I, _I, _L, _P, _P, _P, _P, ctypes.POINTER(_L)]),
    "gksl_assemble": (_S, [_P, _U, ctypes.POINTER(_D)]),
    "gksl_get_csr": (_S, [_P, _I, ctypes.POINTER(_L), _P, _P, _P]),
    "gksl_get_k": (_S, [_P, _P]),
    "gksl_get_k_channel": (_S, [_P, _I, _P]),
    "gksl_set_rho0": (_S, [_P, _P, _P]),
    "gksl_set_state": (_S, [_P, _P, _D]),
    "gksl_get_state": (_S, [_P, _P, ctypes.POINTER(_D)]),
    "gksl_min_stable_steps": (_S, [_P, ctypes.POINTER(_L)]),
    "gksl_propagate": (_S, [_P, _L, _L, _I, _L, _L, _P]),
    "gksl_observable_diag": (_S, [_P, _P, _P, _L, _P]),
    "gksl_rho": (_S, [_P, _P, _P, _P]),
    "gksl_adjoint_timeavg": (_S, [_P, _P, _L, _L, _I, ctypes.POINTER(_D), _P, _I]),
    "gksl_batch_create": (_S, [_I, _P, _P, _P, _P, ctypes.POINTER(_P)]),
    "gksl_batch_destroy": (None, [_P]),
    "gksl_batch_last_error": (ctypes.c_char_p, [_P]),
    "gksl_batch_reset": (_S, [_P]),
    "gksl_batch_propagate": (_S, [_P, _P, _P, _L, ctypes.POINTER(_D)]),
    "gksl_batch_get_state": (_S, [_P, _I, _P]),
    "gksl_batch_info": (_S, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "gksl_batch_set_scan": (_S, [_P, _I, _P]),
    "gksl_batch_group_stats": (_S, [_P, _I, ctypes.POINTER(_L), ctypes.POINTER(_I), ctypes.POINTER(_L),
                                    ctypes.POINTER(_L), ctypes.POINTER(_I)]),
    "gksl_batch_asymptotic": (_S, [_P, _P, _L, _L, _D, _L, _P, ctypes.POINTER(_L)]),
    "gksl_get_info": (_S, [_P, ctypes.POINTER(gksl_info)]),
    "gksl_measure_rates": (_S, [_I, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "gksl_propagate_csr_noalloc": (_S, [_L, _P, _P, _P, _P, _P, _P, _P, _P, _D, _D, _L, _D, _D, _D, _P]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = sorted(_SIGS)


def _ptr(a):
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "arrays must be contiguous"
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous(), "tensors must be contiguous"
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _arr(x, dtype):
    """numpy arrays are converted to the C type; tensors are passed through unchanged."""
    if x is None or hasattr(x, "data_ptr"):
        return x
    return np.ascontiguousarray(x, dtype=dtype)


def _check(st, ctx=None, batch=None, batch_create=False):
    if st != GKSL_OK:
        msg = ""
        if ctx is not None:
            msg = _lib.gksl_last_error(ctx).decode()
        elif batch is not None or batch_create:
            msg = _lib.gksl_batch_last_error(batch).decode()
        raise GkslError(st, msg)


# ------------------------------------------------------------------ the C calls, same names

def gksl_create(N, device=0, cuda_stream=None):
    out = _P()
    _check(_lib.gksl_create(int(N), int(device), cuda_stream, ctypes.byref(out)))
    return out.value


def gksl_destroy(ctx):
    _lib.gksl_destroy(ctx)


def gksl_last_error(ctx):
    return _lib.gksl_last_error(ctx).decode()


def _op(rowptr, col, re, im):
    return _arr(rowptr, np.int32), _arr(col, np.int32), _arr(re, np.float64), _arr(im, np.float64)


def gksl_set_h0_component(ctx, k, theta, rowptr, col, re, im, nnz):
    rp, c, r, i = _op(rowptr, col, re, im)
    _check(_lib.gksl_set_h0_component(ctx, k, theta, _ptr(rp), _ptr(c), _ptr(r), _ptr(i), int(nnz)), ctx)


def gksl_set_theta(ctx, k, theta):
    _check(_lib.gksl_set_theta(ctx, k, theta), ctx)


def gksl_set_h1(ctx, rowptr, col, re, im, nnz):
    rp, c, r, i = _op(rowptr, col, re, im)
    _check(_lib.gksl_set_h1(ctx, _ptr(rp), _ptr(c), _ptr(r), _ptr(i), int(nnz)), ctx)


def gksl_set_dissipator(ctx, p, gamma, rowptr, col, re, im, nnz):
    rp, c, r, i = _op(rowptr, col, re, im)
    _check(_lib.gksl_set_dissipator(ctx, p, gamma, _ptr(rp), _ptr(c), _ptr(r), _ptr(i), int(nnz)), ctx)


def gksl_set_gamma(ctx, p, gamma):
    _check(_lib.gksl_set_gamma(ctx, p, gamma), ctx)


def gksl_set_drive(ctx, E, A, omega):
    _check(_lib.gksl_set_drive(ctx, E, A, omega), ctx)


GKSL_DRIVE_SIN, GKSL_DRIVE_SQUARE = 0, 1


def gksl_set_drive_shape(ctx, shape):
    _check(_lib.gksl_set_drive_shape(ctx, int(shape)), ctx)


def gksl_set_kossakowski(ctx, a_re, a_im=None, tol=1e-12):
    a_re, a_im = _arr(a_re, np.float64), _arr(a_im, np.float64)
    _check(_lib.gksl_set_kossakowski(ctx, _ptr(a_re), _ptr(a_im), float(tol)), ctx)


def gksl_expand(ctx, rowptr, col, re, im, nnz, coef_re, coef_im=None):
    rp, c, r, i = _op(rowptr, col, re, im)
    _check(_lib.gksl_expand(ctx, _ptr(rp), _ptr(c), _ptr(r), _ptr(i), int(nnz), _ptr(coef_re), _ptr(coef_im)), ctx)


def gksl_structure_count(N, which):
    n = _L()
    _check(_lib.gksl_structure_count(int(N), int(which), ctypes.byref(n)))
    return n.value


def gksl_structure_enumerate(N, which, capacity, m, n, s, value):
    cnt = _L()
    _check(_lib.gksl_structure_enumerate(int(N), int(which), int(capacity), _ptr(m), _ptr(n), _ptr(s), _ptr(value),
                                         ctypes.byref(cnt)))
    return cnt.value


def gksl_assemble(ctx, flags=0):
    sec = _D()
    _check(_lib.gksl_assemble(ctx, int(flags), ctypes.byref(sec)), ctx)
    return sec.value


def gksl_get_csr(ctx, which, rowptr=None, col=None, val=None):
    nnz = _L()
    _check(_lib.gksl_get_csr(ctx, int(which), ctypes.byref(nnz), _ptr(rowptr), _ptr(col), _ptr(val)), ctx)
    return nnz.value


def gksl_get_k(ctx, K):
    _check(_lib.gksl_get_k(ctx, _ptr(K)), ctx)


def gksl_get_k_channel(ctx, p, K):
    _check(_lib.gksl_get_k_channel(ctx, int(p), _ptr(K)), ctx)


def gksl_set_rho0(ctx, re, im=None):
    re, im = _arr(re, np.float64), _arr(im, np.float64)
    _check(_lib.gksl_set_rho0(ctx, _ptr(re), _ptr(im)), ctx)


def gksl_set_state(ctx, v, t):
    v = _arr(v, np.float64)
    _check(_lib.gksl_set_state(ctx, _ptr(v), float(t)), ctx)


def gksl_get_state(ctx, v):
    t = _D()
    _check(_lib.gksl_get_state(ctx, _ptr(v), ctypes.byref(t)), ctx)
    return t.value


def gksl_min_stable_steps(ctx):
    n = _L()
    _check(_lib.gksl_min_stable_steps(ctx, ctypes.byref(n)), ctx)
    return n.value


def gksl_propagate(ctx, steps_per_period, n_steps, precision=64, correction_every=0, emit_every=0, v_out=None):
    _check(_lib.gksl_propagate(ctx, int(steps_per_period), int(n_steps), int(precision), int(correction_every),
                               int(emit_every), _ptr(v_out)), ctx)


def gksl_observable_diag(ctx, o_diag, v, count, out):
    o_diag = _arr(o_diag, np.float64)
    _check(_lib.gksl_observable_diag(ctx, _ptr(o_diag), _ptr(v), int(count), _ptr(out)), ctx)


def gksl_rho(ctx, v, re, im):
    _check(_lib.gksl_rho(ctx, _ptr(_arr(v, np.float64)), _ptr(re), _ptr(im)), ctx)


def gksl_adjoint_timeavg(ctx, o_diag, steps_per_period, period_index, precision, grad):
    loss = _D()
    o_diag = _arr(o_diag, np.float64)
    _check(_lib.gksl_adjoint_timeavg(ctx, _ptr(o_diag), int(steps_per_period), int(period_index), int(precision),
                                     ctypes.byref(loss), _ptr(grad), len(grad)), ctx)
    return loss.value


def gksl_batch_create(groups, n_inst, A, g):
    arr = (_P * len(groups))(*groups)
    ni = np.ascontiguousarray(n_inst, dtype=np.int32)
    A = np.ascontiguousarray(A, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = _P()
    _check(_lib.gksl_batch_create(len(groups), ctypes.cast(arr, _P), _ptr(ni), _ptr(A), _ptr(g), ctypes.byref(out)),
           batch_create=True)
    return out.value


def gksl_batch_destroy(b):
    _lib.gksl_batch_destroy(b)


def gksl_batch_reset(b):
    _check(_lib.gksl_batch_reset(b), batch=b)


def gksl_batch_propagate(b, steps_per_period, n_steps, correction_every=0):
    spp = np.ascontiguousarray(steps_per_period, dtype=np.int64)
    ns = np.ascontiguousarray(n_steps, dtype=np.int64)
    sec = _D()
    _check(_lib.gksl_batch_propagate(b, _ptr(spp), _ptr(ns), int(correction_every), ctypes.byref(sec)), batch=b)
    return sec.value


def gksl_batch_get_state(b, instance, v):
    _check(_lib.gksl_batch_get_state(b, int(instance), _ptr(v)), batch=b)


def gksl_batch_set_scan(b, component, theta_b):
    th = np.ascontiguousarray(theta_b, dtype=np.float64)
    _check(_lib.gksl_batch_set_scan(b, int(component), _ptr(th)), batch=b)


def gksl_batch_asymptotic(b, steps_per_period, transient, max_periods, tol, correction_every, n_instances):
    """Returns (residual per instance, total periods run)."""
    spp = np.ascontiguousarray(steps_per_period, dtype=np.int64)
    res = np.zeros(int(n_instances))
    per = _L()
    _check(_lib.gksl_batch_asymptotic(b, _ptr(spp), int(transient), int(max_periods), float(tol),
                                      int(correction_every), _ptr(res), ctypes.byref(per)), batch=b)
    return res, per.value


def gksl_batch_group_stats(b, group):
    """(rows D, instances, channel entries, pair-unit entries, FP32 path: 0 16-byte rows, 1 scalar
    rows, 2 pair units) of one group."""
    rows, inst, ent, pent, path = _L(), _I(), _L(), _L(), _I()
    _check(_lib.gksl_batch_group_stats(b, int(group), ctypes.byref(rows), ctypes.byref(inst), ctypes.byref(ent),
                                       ctypes.byref(pent), ctypes.byref(path)), batch=b)
    return rows.value, inst.value, ent.value, pent.value, path.value


def gksl_batch_info(b, group):
    ipl, us = _I(), _D()
    _check(_lib.gksl_batch_info(b, int(group), ctypes.byref(ipl), ctypes.byref(us)), batch=b)
    return ipl.value, us.value


def gksl_get_info(ctx):
    info = gksl_info()
    _check(_lib.gksl_get_info(ctx, ctypes.byref(info)), ctx)
    return info


def gksl_measure_rates(device=0):
    """(FP64 FMA per second, L2-resident read bytes per second) of the GPU, both self-checked."""
    f, l2 = _D(), _D()
    st = _lib.gksl_measure_rates(int(device), ctypes.byref(f), ctypes.byref(l2))
    if st != GKSL_OK:
        raise GkslError(st, "gksl_measure_rates: a rate probe failed its own check or a CUDA call failed")
    return f.value, l2.value


GKSL_NOALLOC_MAX_D = 262144


def _noalloc_check(D, mats, K, v):
    """Reject, before anything is launched, arguments the allocation-free kernels would index out
    of bounds: every array a contiguous CUDA tensor on v's device, CSR rowptr/col int32 and values
    float64, rowptr of D + 1 entries from 0 to at most the length of col and val, K and v float64
    of D entries.  Reads the first and last rowptr entry of each matrix (two 4-byte copies)."""
    import torch

    def bad(msg):
        raise GkslError(GKSL_ERR_ARG, f"gksl_propagate_csr_noalloc: {msg}")

    if not isinstance(v, torch.Tensor) or not v.is_cuda:
        bad("v must be a CUDA tensor")
    dev = v.device

    def tensor(name, x, dtype, n=None):
        if not isinstance(x, torch.Tensor) or not x.is_cuda:
            bad(f"{name} must be a CUDA tensor")
        if x.device != dev:
            bad(f"{name} is on {x.device}, v on {dev}")
        if x.dtype != dtype:
            bad(f"{name} must be {dtype}, got {x.dtype}")
        if not x.is_contiguous():
            bad(f"{name} must be contiguous")
        if n is not None and x.numel() != n:
            bad(f"{name} has {x.numel()} entries, expected {n}")

    if not 1 <= int(D) <= GKSL_NOALLOC_MAX_D:
        bad(f"D = {int(D)} must be in [1, GKSL_NOALLOC_MAX_D = {GKSL_NOALLOC_MAX_D}]")
    tensor("v", v, torch.float64, int(D))
    if K is not None:
        tensor("K", K, torch.float64, int(D))
    for name, (rp, col, val) in mats.items():
        if rp is None and col is None and val is None and name == "A1":
            continue
        if rp is None or col is None or val is None:
            bad(f"{name}: rowptr, col and val must all be given" + (" or all be None" if name == "A1" else ""))
        tensor(f"{name} rowptr", rp, torch.int32, int(D) + 1)
        tensor(f"{name} col", col, torch.int32)
        tensor(f"{name} val", val, torch.float64, col.numel())
        first, last = int(rp[0]), int(rp[-1])
        if first != 0 or last > col.numel():
            bad(f"{name} rowptr must run from 0 to at most {col.numel()} (got {first} .. {last})")


def gksl_propagate_csr_noalloc(D, a0_rowptr, a0_col, a0_val, a1_rowptr, a1_col, a1_val, K, v, t0, h, n_steps, E, A,
                               omega, cuda_stream=None):
    """Allocation-free RK4 on caller-owned device arrays (all array arguments CUDA tensors on one
    device; the A1 triple and K may be None).  The arguments are checked first (``_noalloc_check``);
    the call then runs with v's device current, on ``cuda_stream`` or, when that is None, on torch's
    current stream of that device, so it is ordered after the work that produced its inputs."""
    import torch
    _noalloc_check(D, {"A0": (a0_rowptr, a0_col, a0_val), "A1": (a1_rowptr, a1_col, a1_val)}, K, v)
    with torch.cuda.device(v.device):
        if cuda_stream is None:
            cuda_stream = torch.cuda.current_stream(v.device).cuda_stream
        st = _lib.gksl_propagate_csr_noalloc(int(D), _ptr(a0_rowptr), _ptr(a0_col), _ptr(a0_val), _ptr(a1_rowptr),
                                             _ptr(a1_col), _ptr(a1_val), _ptr(K), _ptr(v), float(t0), float(h),
                                             int(n_steps), float(E), float(A), float(omega), cuda_stream)
    if st == GKSL_ERR_ARG:
        raise GkslError(st, "gksl_propagate_csr_noalloc: h must be > 0 and n_steps >= 0")
    if st != GKSL_OK:
        raise GkslError(st, f"gksl_propagate_csr_noalloc failed with status {st} (a CUDA error was pending or a "
                            f"launch failed)")


# ------------------------------------------------------------------ conveniences over the calls

def set_csr_operator(setter, ctx, *lead, op):
    """Pass a workloads.CSR operator to one of the gksl_set_* calls."""
    setter(ctx, *lead, op.rowptr, op.col, op.re, op.im, op.nnz)


def get_csr_numpy(ctx, which):
    """Copy an assembled matrix to host numpy arrays (rowptr, col, val)."""
    nnz = gksl_get_csr(ctx, which)
    info_D = gksl_get_info(ctx).D
    rp = np.empty(info_D + 1, dtype=np.int32)
    col = np.empty(max(nnz, 1), dtype=np.int32)
    val = np.empty(max(nnz, 1), dtype=np.float64)
    gksl_get_csr(ctx, which, rp, col, val)
    return rp, col[:nnz], val[:nnz]


def dimer_context(d, device=0, stream=None, flags=GKSL_ASM_FP32 | GKSL_ASM_TRANSPOSE, assemble=True):
    """Context for a workloads.Dimer: H0 components (J HJ, U HU), H1 and L at rate gamma/M."""
    p = d.params
    ctx = gksl_create(d.N, device, stream)
    set_csr_operator(gksl_set_h0_component, ctx, 0, p["J"], op=d.HJ)
    set_csr_operator(gksl_set_h0_component, ctx, 1, p["U"], op=d.HU)
    set_csr_operator(gksl_set_h1, ctx, op=d.H1)
    set_csr_operator(gksl_set_dissipator, ctx, 0, d.rate, op=d.L)
    gksl_set_drive(ctx, p["E"], p["A"], p["omega"])
    if assemble:
        gksl_assemble(ctx, flags)
    gksl_set_rho0(ctx, d.rho0_dense().real.copy(), d.rho0_dense().imag.copy())
    return ctx


def dimer_batch(instances, device=0):
    """Batch of dimer instances (dicts with N, A, gamma): one group per N, group contexts at rate
    1/(N-1) so that the per-instance scale g_b = gamma_b gives the rate gamma_b/(N-1).

    Returns (batch, contexts, groups) where groups[i] = (N, [instance indices], stable steps per
    period for the group's largest A and gamma)."""
    from . import workloads as W
    by_n = {}
    for i, x in enumerate(instances):
        by_n.setdefault(x["N"], []).append(i)
    ctxs, n_inst, A, g, groups = [], [], [], [], []
    for N in sorted(by_n):
        idx = by_n[N]
        d = W.dimer(N)
        d.rate = 1.0 / (N - 1)
        c = dimer_context(d, device=device, flags=GKSL_ASM_FP32)
        p = d.params
        gksl_set_drive(c, p["E"], max(instances[i]["A"] for i in idx), p["omega"])
        gksl_set_gamma(c, 0, max(instances[i]["gamma"] for i in idx) / (N - 1))
        spp = gksl_min_stable_steps(c)
        gksl_set_gamma(c, 0, 1.0 / (N - 1))
        gksl_set_drive(c, p["E"], p["A"], p["omega"])
        gksl_assemble(c, GKSL_ASM_FP32)
        ctxs.append(c)
        n_inst.append(len(idx))
        A += [instances[i]["A"] for i in idx]
        g += [instances[i]["gamma"] for i in idx]
        groups.append((N, idx, spp))
    return gksl_batch_create(ctxs, n_inst, A, g), ctxs, groups


def bifurcation_scan(N, U_values, transient=10, tol=0.0, max_periods=1, steps_per_period=None, device=0,
                     params=None, correction_every=None):
    """Populations diag rho at phase 0 of the driven dimer's long-time state for every interaction U
    in U_values, propagated together as one batch (the quantum bifurcation diagram of Sec. III /
    Sec. V): `transient` periods, then period by period until every instance's period-map residual
    max_s |v(kT) - v((k-1)T)| is <= tol or `max_periods` more periods have run
    (gksl_batch_asymptotic).  FP32 bulk with one FP64 step per period unless `correction_every`
    says otherwise (1: FP64 throughout).
    Returns (populations [len(U), N], steps per period, residual per U, total periods run)."""
    from . import workloads as W
    d = W.dimer(N, params)
    ctx = dimer_context(d, device=device, flags=GKSL_ASM_FP32)
    b = None
    try:
        p = d.params
        n = len(U_values)
        if steps_per_period is None:
            gksl_set_theta(ctx, 1, float(np.max(np.abs(U_values))))
            steps_per_period = gksl_min_stable_steps(ctx)
            steps_per_period += steps_per_period % 2
            gksl_set_theta(ctx, 1, p["U"])
            gksl_assemble(ctx, GKSL_ASM_FP32)
        if correction_every is None:
            correction_every = steps_per_period
        b = gksl_batch_create([ctx], [n], [p["A"]] * n, [1.0] * n)
        gksl_batch_set_scan(b, 1, U_values)
        residual, periods = gksl_batch_asymptotic(b, [steps_per_period], transient, max_periods, tol,
                                                  correction_every, n)
        D = N * N - 1
        pops = np.zeros((n, N))
        v = np.zeros(D)
        re, im = np.zeros((N, N)), np.zeros((N, N))
        for i in range(n):
            gksl_batch_get_state(b, i, v)
            gksl_rho(ctx, v, re, im)
            pops[i] = np.diag(re)
        return pops, steps_per_period, residual, periods
    finally:
        if b is not None:
            gksl_batch_destroy(b)
        gksl_destroy(ctx)


class TimeAvgObservable:
    """torch.autograd.Function factory: loss(theta) = period mean of <O> with the adjoint gradient.

    ``make(ctx, o_diag, spp, period, precision)`` returns a function of a float64 tensor
    theta = [A, gamma_0.., theta_0..] (the order of gksl_adjoint_timeavg) whose backward is
    the library's discrete adjoint of the RK4 map.
    """

    @staticmethod
    def make(ctx, o_diag, steps_per_period, period_index, precision=64):
        import torch

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(fctx, theta):
                th = theta.detach().cpu().numpy().astype(np.float64)
                info = gksl_get_info(ctx)
                del info
                grad = np.zeros(len(th))
                _apply_params(ctx, th)
                loss = gksl_adjoint_timeavg(ctx, o_diag, steps_per_period, period_index, precision, grad)
                fctx.save_for_backward(torch.as_tensor(grad, dtype=theta.dtype, device=theta.device))
                return torch.as_tensor(loss, dtype=theta.dtype, device=theta.device)

            @staticmethod
            def backward(fctx, gout):
                (g,) = fctx.saved_tensors
                return gout * g

        return _Fn.apply


_PARAM_LAYOUT = {}


def set_param_layout(ctx, A_drive, E, omega, channels, components):
    """Record which channel / component indices theta maps to for TimeAvgObservable."""
    _PARAM_LAYOUT[ctx] = (E, omega, list(channels), list(components))


def _apply_params(ctx, th):
    E, omega, channels, comps = _PARAM_LAYOUT[ctx]
    gksl_set_drive(ctx, E, float(th[0]), omega)
    for i, p in enumerate(channels):
        gksl_set_gamma(ctx, p, float(th[1 + i]))
    for i, k in enumerate(comps):
        gksl_set_theta(ctx, k, float(th[1 + len(channels) + i]))
    gksl_assemble(ctx, GKSL_ASM_FP32 | GKSL_ASM_TRANSPOSE)
