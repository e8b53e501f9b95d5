"""Unfolded dimer system by the definition route (test infrastructure only).

For the driven dimer, H(t) = J HJ + U HU + eps(t) H1 and one dissipator L with
rate g, the unfolded system (Eq. 8) is linear in every parameter:
    dv/dt = (J Q_J + U Q_U + g R1 + eps(t) Q1) v + g K1,
where Q_X is the matrix of X -> -i[X_op, .] and (R1, K1) the matrix and image of
1/N of the unit-rate dissipator, all by Q_sm = Tr(F_s L(F_m)) (``native.unfold``).
"""
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import native
from . import propagate as _p


@dataclass
class Unfolded:
    N: int
    QJ: sp.csr_matrix
    QU: sp.csr_matrix
    Q1: sp.csr_matrix
    R1: sp.csr_matrix
    K1: np.ndarray
    max_imag: float

    def q0(self, J, U, rate):
        """J Q_J + U Q_U + rate R1 (everything but the eps(t) Q1 term)."""
        return (J * self.QJ + U * self.QU + rate * self.R1).tocsr()


def unfold_dimer(d):
    """Components of the unfolded dimer of ``workloads.dimer`` (definition route)."""
    N = d.N
    QJ, _, i1 = native.unfold(N, H=d.HJ.to_scipy(), want_k=False)
    QU, _, i2 = native.unfold(N, H=d.HU.to_scipy(), want_k=False)
    Q1, _, i3 = native.unfold(N, H=d.H1.to_scipy(), want_k=False)
    R1, K1, i4 = native.unfold(N, A=d.L.to_scipy(), gamma=1.0)
    return Unfolded(N, QJ, QU, Q1, R1, K1, max(i1, i2, i3, i4))


def initial_v(d):
    """v(0) = Tr(F_j rho0) for rho0 = |k><k| (Sec. IV step 2.6)."""
    from . import basis as _b
    rho0 = sp.csr_matrix(([1.0 + 0j], ([d.rho0_index], [d.rho0_index])), shape=(d.N, d.N))
    return _b.expand_sparse(rho0).real


def propagate_dimer(d, u, steps_per_period, nsteps, emit_every=None, v0=None, t0=0.0, drive="sin", threaded=False):
    """RK4 of the dimer from v0 (default v(0)); returns (v_final, emitted list).

    drive: "sin" (theta = sin(omega t)) or "square" (theta = +-1, Sec. III driving (i)).
    threaded: run the same map with the C RK4 on every host core (``native.rk4``)."""
    p = d.params
    T = 2 * np.pi / p["omega"]
    h = T / steps_per_period
    Q0 = u.q0(p["J"], p["U"], d.rate)
    K = d.rate * u.K1
    if v0 is None:
        v0 = initial_v(d)
    if threaded:
        return native.rk4(Q0, u.Q1, K, p["E"], p["A"], p["omega"], v0, h, nsteps, t0=t0, emit_every=emit_every,
                          drive=drive)
    step = _p.eps_square_step(p["E"], p["A"], p["omega"]) if drive == "square" else None
    return _p.rk4(Q0, u.Q1, K, _p.eps_fn(p["E"], p["A"], p["omega"]), v0, h, nsteps, t0=t0,
                  emit_every=emit_every, eps_step=step)
