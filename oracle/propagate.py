"""Propagation of dv/dt = A(t) v + b by classical RK4, its discrete adjoint, and rho-space checks.

TEST INFRASTRUCTURE ONLY. Sec. IV step 3.1 integrates Eq. 8 with the fourth-order
Runge-Kutta method; the paper gives no step size, so the time grid is a reading:
t_n = t0 + n h, stages at t_n, t_n + h/2 (twice) and t_n + h, and
A(t) = Q0 + eps(t) Q1 with eps(t) = E + A_drive sin(omega t).

The discrete adjoint differentiates exactly this discrete map (a reading: the
paper has no gradient); with Y1 = v, Y2 = v + h/2 k1, Y3 = v + h/2 k2,
Y4 = v + h k3, k_i = A_i Y_i + b and v' = v + h/6 (k1 + 2 k2 + 2 k3 + k4),
the reverse sweep for an output adjoint lam' is
    kb4 = h/6 lam'            Yb4 = A4^T kb4
    kb3 = h/3 lam' + h Yb4    Yb3 = A3^T kb3
    kb2 = h/3 lam' + h/2 Yb3  Yb2 = A2^T kb2
    kb1 = h/6 lam' + h/2 Yb2  Yb1 = A1^T kb1
    lam = lam' + Yb1 + Yb2 + Yb3 + Yb4,
and a parameter theta gains sum_i kb_i . (dA_i/dtheta Y_i + db/dtheta).
"""
import numpy as np
import scipy.linalg as sla

from . import basis as _b
from . import lindblad as _l


def eps_fn(E, A, omega):
    return lambda t: E + A * np.sin(omega * t)


def square_theta(t, omega):
    """Sec. III driving (i): theta = +1 on [0, T/2), -1 on [T/2, T), periodic, T = 2 pi / omega."""
    T = 2 * np.pi / omega
    return 1.0 if (t % T) < 0.5 * T else -1.0


def eps_square_step(E, A, omega):
    """Stage values of eps for the square drive (reading): the drive is constant on every step of a
    grid that contains its jumps, so all stages of the step use theta at the step's midpoint."""
    def stages(t, h):
        e = E + A * square_theta(t + 0.5 * h, omega)
        return e, e, e
    return stages


def rk4(Q0, Q1, K, eps, v0, h, nsteps, t0=0.0, emit_every=None, emit_fn=None, eps_step=None):
    """Classical RK4 on dv/dt = (Q0 + eps(t) Q1) v + K.

    Q0, Q1 are anything with ``@`` (scipy sparse or dense). Returns the final v and
    the list of emitted values (v, or emit_fn(v), every ``emit_every`` steps).
    ``eps_step(t_n, h)``, when given, supplies the three stage values (t_n, t_n + h/2, t_n + h)
    instead of eps(t) at the stage times.  Works in complex arithmetic too (complex-step).
    """
    v = np.array(v0, copy=True)
    out = []

    def f(e, y):
        return Q0 @ y + e * (Q1 @ y) + K

    for n in range(nsteps):
        t = t0 + n * h
        if eps_step is not None:
            e1, e2, e4 = eps_step(t, h)
        else:
            e1, e2, e4 = eps(t), eps(t + 0.5 * h), eps(t + h)
        k1 = f(e1, v)
        k2 = f(e2, v + 0.5 * h * k1)
        k3 = f(e2, v + 0.5 * h * k2)
        k4 = f(e4, v + h * k3)
        v = v + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        if emit_every and (n + 1) % emit_every == 0:
            out.append(emit_fn(v) if emit_fn else v.copy())
    return v, out


def trapezoid_weights(steps_per_period):
    """Weights of the trapezoid mean over the S+1 grid points of one period."""
    S = steps_per_period
    w = np.full(S + 1, 1.0 / S)
    w[0] = w[-1] = 0.5 / S
    return w


def timeavg_loss(Q0, Q1, K, eps, v0, w_obs, c_obs, h, steps_per_period, period_index, t0=0.0):
    """Trapezoid mean of <O> = c_obs + w_obs.v over period `period_index` (1-based).

    The forward trajectory starts at t0 with v0 and runs period_index periods.
    """
    S = steps_per_period
    wt = trapezoid_weights(S)
    first = (period_index - 1) * S
    v = np.array(v0, copy=True)
    acc = 0.0
    if first == 0:
        acc = acc + wt[0] * (c_obs + w_obs @ v)
    for n in range(period_index * S):
        v, _ = rk4(Q0, Q1, K, eps, v, h, 1, t0=t0 + n * h)
        m = n + 1 - first
        if m >= 0:
            acc = acc + wt[m] * (c_obs + w_obs @ v)
    return acc


def timeavg_adjoint(Q0, Q1, K, eps, v0, w_obs, c_obs, h, steps_per_period, period_index,
                    dQ0, dQ1, dK, t0=0.0):
    """Loss and gradient of ``timeavg_loss`` by the discrete adjoint of RK4.

    dQ0, dQ1, dK are lists (one entry per parameter) of the derivatives of Q0, of
    the coefficient matrix multiplying eps(t) -- given as a pair (matrix, deps)
    with deps(t) = d eps(t) / d theta -- and of K. Entries may be None.
    Returns (loss, grad).
    """
    S = steps_per_period
    wt = trapezoid_weights(S)
    first = (period_index - 1) * S
    nsteps = period_index * S
    traj = [np.array(v0, copy=True)]
    v = traj[0]
    for n in range(nsteps):
        v, _ = rk4(Q0, Q1, K, eps, v, h, 1, t0=t0 + n * h)
        traj.append(v)
    loss = sum(wt[m] * (c_obs + w_obs @ traj[first + m]) for m in range(S + 1))

    Q0T = Q0.T
    Q1T = Q1.T
    P = len(dQ0)
    grad = np.zeros(P)
    lam = wt[S] * w_obs
    for n in range(nsteps - 1, -1, -1):
        t = t0 + n * h
        v = traj[n]
        ts = (t, t + 0.5 * h, t + 0.5 * h, t + h)

        def Aop(tt, y):
            return Q0 @ y + eps(tt) * (Q1 @ y)

        def ATop(tt, y):
            return Q0T @ y + eps(tt) * (Q1T @ y)

        Y1 = v
        k1 = Aop(ts[0], Y1) + K
        Y2 = v + 0.5 * h * k1
        k2 = Aop(ts[1], Y2) + K
        Y3 = v + 0.5 * h * k2
        k3 = Aop(ts[2], Y3) + K
        Y4 = v + h * k3
        kb4 = (h / 6.0) * lam
        Yb4 = ATop(ts[3], kb4)
        kb3 = (h / 3.0) * lam + h * Yb4
        Yb3 = ATop(ts[2], kb3)
        kb2 = (h / 3.0) * lam + 0.5 * h * Yb3
        Yb2 = ATop(ts[1], kb2)
        kb1 = (h / 6.0) * lam + 0.5 * h * Yb2
        Yb1 = ATop(ts[0], kb1)
        for p in range(P):
            for kb, Y, tt in ((kb1, Y1, ts[0]), (kb2, Y2, ts[1]), (kb3, Y3, ts[2]), (kb4, Y4, ts[3])):
                g = 0.0
                if dQ0[p] is not None:
                    g += kb @ (dQ0[p] @ Y)
                if dQ1[p] is not None:
                    M1, deps = dQ1[p]
                    g += deps(tt) * (kb @ (M1 @ Y))
                if dK[p] is not None:
                    g += kb @ dK[p]
                grad[p] += g
        lam = lam + Yb1 + Yb2 + Yb3 + Yb4
        m = n - first
        if 0 <= m <= S:
            lam = lam + wt[m] * w_obs
    return loss, grad


def observable_weights(o_diag):
    """<O> = Tr(O)/N + sum_j v_j Tr(O F_j) for a diagonal O (Eq. 6); returns (w, c0)."""
    N = len(o_diag)
    O = np.diag(np.asarray(o_diag, dtype=np.complex128))
    w = _b.expand_sparse(O).real
    return w, float(np.sum(o_diag) / N)


# ------------------------------------------------------------- rho-space checks

def rho_rk4(H0, H1, Ls, gammas, eps, rho0, h, nsteps, t0=0.0):
    """RK4 applied directly to vec(rho) with the dense Liouvillian of Eq. 1 (no generator basis).

    RK4 commutes with the affine change of variables v = Tr(F rho), so this must
    reproduce the v-space map up to rounding.
    """
    N = rho0.shape[0]
    S0 = _l.liouvillian_vec(H0, Ls, gammas)
    S1 = _l.liouvillian_vec(H1)
    x = _l.vec(rho0).astype(np.complex128)
    for n in range(nsteps):
        t = t0 + n * h

        def f(tt, y):
            return S0 @ y + eps(tt) * (S1 @ y)

        k1 = f(t, x)
        k2 = f(t + 0.5 * h, x + 0.5 * h * k1)
        k3 = f(t + 0.5 * h, x + 0.5 * h * k2)
        k4 = f(t + h, x + h * k3)
        x = x + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
    return _l.unvec(x, N)


def rho_expm(H, Ls, gammas, rho0, t):
    """Exact rho(t) = exp(t L) rho0 for a time-independent Lindbladian (matrix exponential)."""
    N = rho0.shape[0]
    S = _l.liouvillian_vec(H, Ls, gammas)
    return _l.unvec(sla.expm(t * S) @ _l.vec(rho0), N)
