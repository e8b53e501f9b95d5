/*
 * Threaded CPU RK4 of the unfolded system.  TEST INFRASTRUCTURE ONLY -- called from the
 * oracle's Python wrapper (and timed as the CPU baseline); the product library never links it.
 *
 * Sec. IV step 3.1 integrates Eq. 8, dv/dt = (Q0 + eps(t) Q1) v + K, with the classical
 * fourth-order Runge-Kutta method.  The paper gives no time grid; the reading used throughout
 * the oracle is t_n = t0 + n h with stages at t_n, t_n + h/2 (twice) and t_n + h, and
 *     eps(t) = E + A sin(omega t)                       (drive 0, Sec. III driving (ii)),
 *     eps    = E + A theta(t_n + h/2), theta = +-1      (drive 1, Sec. III driving (i): the
 *              drive is constant on every step of a grid that holds its jumps).
 * One step:
 *     k1 = f(t_n, v),            y = v + (h/2) k1
 *     k2 = f(t_n + h/2, y),      y = v + (h/2) k2
 *     k3 = f(t_n + h/2, y),      y = v + h k3
 *     k4 = f(t_n + h, y),        v = v + (h/6) (k1 + 2 k2 + 2 k3 + k4)
 * with f(t, y)_r = sum_e Q0[r,e] y[col e] + eps(t) sum_e Q1[r,e] y[col e] + K_r, the entries of
 * a row summed in stored order.  Rows are shared out over OpenMP threads; that changes no sum.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_rk4_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static double drive_eps(int drive, double E, double A, double omega, double t) {
    if (drive == 0) return E + A * sin(omega * t);
    double T = 2.0 * M_PI / omega;
    return E + A * (fmod(t, T) < 0.5 * T ? 1.0 : -1.0);
}

/* k = Q0 y + eps Q1 y + K (Q1 and K may be absent); the rows are shared out over the threads of
 * the enclosing parallel region (an orphaned work-sharing loop, ending in a barrier) */
static void f_eval(long long D, const int *p0, const int *c0, const double *v0,
                   const int *p1, const int *c1, const double *v1, const double *K,
                   double eps, const double *y, double *k) {
    long long r;
#pragma omp for schedule(static)
    for (r = 0; r < D; ++r) {
        double a = 0.0;
        for (int e = p0[r]; e < p0[r + 1]; ++e) a += v0[e] * y[c0[e]];
        double b = 0.0;
        if (p1)
            for (int e = p1[r]; e < p1[r + 1]; ++e) b += v1[e] * y[c1[e]];
        double s = a + eps * b;
        k[r] = K ? s + K[r] : s;
    }
}

/* y = v + c k */
static void axpy(long long D, const double *v, double c, const double *k, double *y) {
    long long r;
#pragma omp for schedule(static)
    for (r = 0; r < D; ++r) y[r] = v[r] + c * k[r];
}

/*
 * Runs n_steps RK4 steps of size h from time t0 on v (length D, updated in place).  Every
 * emit_every steps (0: never) v is copied to the next row of out (D doubles per row).
 * Returns 0, or -1 when the work vectors cannot be allocated.  One parallel region covers the
 * whole call; every thread walks the same steps and shares out the rows of each sweep.
 */
int oracle_rk4(long long D, const int *q0_ptr, const int *q0_col, const double *q0_val,
               const int *q1_ptr, const int *q1_col, const double *q1_val, const double *K,
               int drive, double E, double A, double omega,
               double *v, double t0, double h, long long n_steps, long long emit_every, double *out) {
    double *k1 = malloc(sizeof(double) * (size_t)D), *k2 = malloc(sizeof(double) * (size_t)D);
    double *k3 = malloc(sizeof(double) * (size_t)D), *k4 = malloc(sizeof(double) * (size_t)D);
    double *y = malloc(sizeof(double) * (size_t)D);
    if (!k1 || !k2 || !k3 || !k4 || !y) {
        free(k1); free(k2); free(k3); free(k4); free(y);
        return -1;
    }
    const double hh = 0.5 * h, h6 = h / 6.0;
#pragma omp parallel
    {
        for (long long n = 0; n < n_steps; ++n) {
            double t = t0 + (double)n * h;
            double e1, e2, e4;
            if (drive == 0) {
                e1 = drive_eps(0, E, A, omega, t);
                e2 = drive_eps(0, E, A, omega, t + 0.5 * h);
                e4 = drive_eps(0, E, A, omega, t + h);
            } else {
                e1 = e2 = e4 = drive_eps(1, E, A, omega, t + 0.5 * h);
            }
            f_eval(D, q0_ptr, q0_col, q0_val, q1_ptr, q1_col, q1_val, K, e1, v, k1);
            axpy(D, v, hh, k1, y);
            f_eval(D, q0_ptr, q0_col, q0_val, q1_ptr, q1_col, q1_val, K, e2, y, k2);
            axpy(D, v, hh, k2, y);
            f_eval(D, q0_ptr, q0_col, q0_val, q1_ptr, q1_col, q1_val, K, e2, y, k3);
            axpy(D, v, h, k3, y);
            f_eval(D, q0_ptr, q0_col, q0_val, q1_ptr, q1_col, q1_val, K, e4, y, k4);
            long long r;
#pragma omp for schedule(static)
            for (r = 0; r < D; ++r) v[r] = v[r] + h6 * (k1[r] + 2.0 * k2[r] + 2.0 * k3[r] + k4[r]);
            if (emit_every > 0 && (n + 1) % emit_every == 0 && out) {
#pragma omp single
                memcpy(out + (size_t)((n + 1) / emit_every - 1) * (size_t)D, v, sizeof(double) * (size_t)D);
            }
        }
    }
    free(k1); free(k2); free(k3); free(k4); free(y);
    return 0;
}
