/*
 * Sparse CPU oracle: the matrix of a Lindbladian in the SU(N) generator basis,
 * by definition, column by column.  TEST INFRASTRUCTURE ONLY -- called from the
 * oracle's Python wrapper; the product library never links it.
 *
 * Definition (Eq. 1, Eq. 6, Eq. 8 of arXiv:1812.11626):
 *     G_sm = Re Tr(F_s L(F_m)),      K_s = Re Tr(F_s L(1/N)),
 * with L(X) = -i[H, X] + gamma (A X A^+ - 1/2 {A^+ A, X}) for one Hamiltonian H
 * and one dissipator A (either may be absent).  Column m is obtained by forming
 * Y = L(F_m) as a sparse N x N matrix and reading off Tr(F_s Y) for every
 * generator s with the entry formulas of the Sec. II basis:
 *     S^(j,k): (Y_jk + Y_kj)/sqrt2,  J^(j,k): i (Y_jk - Y_kj)/sqrt2,
 *     D^l:     c_l (sum_{k<l} Y_kk - l Y_ll),  c_l = 1/sqrt(l(l+1)).
 * The basis order is S (pairs j<k lexicographic), then J, then D^1..D^{N-1}.
 * No structure constant is used anywhere in this file.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct { int n; int *ptr, *idx; double *re, *im; } csr_t;

static void csr_free(csr_t *a) { free(a->ptr); free(a->idx); free(a->re); free(a->im); }

/* transpose (no conjugation) of an n x n CSR matrix */
static csr_t csr_transpose(int n, const int *ptr, const int *idx, const double *re, const double *im) {
    csr_t t; int nnz = ptr[n];
    t.n = n;
    t.ptr = calloc((size_t)n + 1, sizeof(int));
    t.idx = malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    t.re = malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    t.im = malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    for (int e = 0; e < nnz; ++e) t.ptr[idx[e] + 1]++;
    for (int i = 0; i < n; ++i) t.ptr[i + 1] += t.ptr[i];
    int *fill = malloc(sizeof(int) * (size_t)n);
    memcpy(fill, t.ptr, sizeof(int) * (size_t)n);
    for (int r = 0; r < n; ++r)
        for (int e = ptr[r]; e < ptr[r + 1]; ++e) {
            int p = fill[idx[e]]++;
            t.idx[p] = r; t.re[p] = re[e]; t.im[p] = im[e];
        }
    free(fill);
    return t;
}

/* dense-backed sparse accumulator for an N x N complex matrix */
typedef struct { int N; double *re, *im; char *mark; int *list; int cnt; int diag; } acc_t;

static void acc_add(acc_t *a, int i, int j, double xr, double xi) {
    size_t p = (size_t)i * a->N + j;
    if (!a->mark[p]) { a->mark[p] = 1; a->list[a->cnt++] = (int)p; }
    a->re[p] += xr; a->im[p] += xi;
    if (i == j) a->diag = 1;
}

static void acc_clear(acc_t *a) {
    for (int t = 0; t < a->cnt; ++t) { size_t p = (size_t)a->list[t]; a->mark[p] = 0; a->re[p] = 0; a->im[p] = 0; }
    a->cnt = 0; a->diag = 0;
}

/* generator F_m as a list of (i, j, value) entries */
static int generator_entries(int N, long long m, int *ei, int *ej, double *er, double *eim) {
    long long P2 = (long long)N * (N - 1) / 2;
    const double r2 = 1.0 / sqrt(2.0);
    if (m < 2 * P2) {
        long long p = m < P2 ? m : m - P2;
        int j = 0;                                    /* invert the lexicographic pair index */
        while (p >= (long long)(N - 1 - j)) { p -= N - 1 - j; ++j; }
        int k = j + 1 + (int)p;
        ei[0] = j; ej[0] = k; ei[1] = k; ej[1] = j;
        if (m < P2) { er[0] = r2; eim[0] = 0; er[1] = r2; eim[1] = 0; }
        else        { er[0] = 0; eim[0] = -r2; er[1] = 0; eim[1] = r2; }
        return 2;
    }
    int l = (int)(m - 2 * P2) + 1;
    double c = 1.0 / sqrt((double)l * (l + 1.0));
    for (int k = 0; k < l; ++k) { ei[k] = k; ej[k] = k; er[k] = c; eim[k] = 0; }
    ei[l] = l; ej[l] = l; er[l] = -l * c; eim[l] = 0;
    return l + 1;
}

typedef struct {
    int N;
    int hasH; csr_t H, HT;          /* H in CSR and its transpose (columns of H) */
    int hasA; csr_t A, AT, M, MT;   /* dissipator, its transpose, M = A^+ A and M^T */
    double gamma;
} gen_t;

/* Y += L(X) for X given as entries (i, j, x) */
static void apply_L(const gen_t *g, acc_t *Y, int ne, const int *ei, const int *ej, const double *er, const double *eim) {
    for (int t = 0; t < ne; ++t) {
        int i = ei[t], j = ej[t];
        double xr = er[t], xi = eim[t];
        if (g->hasH) {
            /* -i (H X)_{kj} = -i sum_i H_ki X_ij : column i of H is row i of H^T */
            for (int e = g->HT.ptr[i]; e < g->HT.ptr[i + 1]; ++e) {
                int k = g->HT.idx[e]; double hr = g->HT.re[e], hi = g->HT.im[e];
                double pr = hr * xr - hi * xi, pi = hr * xi + hi * xr;
                acc_add(Y, k, j, pi, -pr);             /* -i * (pr + i pi) = pi - i pr */
            }
            /* +i (X H)_{ik} = +i sum_j X_ij H_jk : row j of H */
            for (int e = g->H.ptr[j]; e < g->H.ptr[j + 1]; ++e) {
                int k = g->H.idx[e]; double hr = g->H.re[e], hi = g->H.im[e];
                double pr = xr * hr - xi * hi, pi = xr * hi + xi * hr;
                acc_add(Y, i, k, -pi, pr);             /* +i * (pr + i pi) = -pi + i pr */
            }
        }
        if (g->hasA) {
            double gm = g->gamma;
            /* gamma (A X A^+)_{ab} = gamma sum A_ai X_ij conj(A_bj) : columns i and j of A */
            for (int e = g->AT.ptr[i]; e < g->AT.ptr[i + 1]; ++e) {
                int a = g->AT.idx[e]; double ar = g->AT.re[e], ai = g->AT.im[e];
                double tr = ar * xr - ai * xi, ti = ar * xi + ai * xr;
                for (int f = g->AT.ptr[j]; f < g->AT.ptr[j + 1]; ++f) {
                    int b = g->AT.idx[f]; double br = g->AT.re[f], bi = -g->AT.im[f];
                    acc_add(Y, a, b, gm * (tr * br - ti * bi), gm * (tr * bi + ti * br));
                }
            }
            /* -gamma/2 (M X)_{kj} = -gamma/2 sum_i M_ki X_ij : column i of M */
            for (int e = g->MT.ptr[i]; e < g->MT.ptr[i + 1]; ++e) {
                int k = g->MT.idx[e]; double mr = g->MT.re[e], mi = g->MT.im[e];
                acc_add(Y, k, j, -0.5 * gm * (mr * xr - mi * xi), -0.5 * gm * (mr * xi + mi * xr));
            }
            /* -gamma/2 (X M)_{ik} = -gamma/2 sum_j X_ij M_jk : row j of M */
            for (int e = g->M.ptr[j]; e < g->M.ptr[j + 1]; ++e) {
                int k = g->M.idx[e]; double mr = g->M.re[e], mi = g->M.im[e];
                acc_add(Y, i, k, -0.5 * gm * (xr * mr - xi * mi), -0.5 * gm * (xr * mi + xi * mr));
            }
        }
    }
}

/* coefficients Tr(F_s Y) of the accumulated Y; calls emit(s, re, im) for every touched s */
typedef struct { double *re, *im; char *mark; long long *list; long long cnt; } vacc_t;

static void vacc_add(vacc_t *v, long long s, double xr, double xi) {
    if (!v->mark[s]) { v->mark[s] = 1; v->list[v->cnt++] = s; }
    v->re[s] += xr; v->im[s] += xi;
}

static void expand_Y(int N, const acc_t *Y, vacc_t *v) {
    long long P2 = (long long)N * (N - 1) / 2;
    const double r2 = 1.0 / sqrt(2.0);
    for (int t = 0; t < Y->cnt; ++t) {
        size_t p = (size_t)Y->list[t];
        int i = (int)(p / (size_t)N), j = (int)(p % (size_t)N);
        if (i == j) continue;
        int a = i < j ? i : j, b = i < j ? j : i;
        long long q = (long long)a * N - (long long)a * (a + 1) / 2 + (b - a - 1);
        double yr = Y->re[p], yi = Y->im[p];
        vacc_add(v, q, yr * r2, yi * r2);
        if (i < j) vacc_add(v, P2 + q, -yi * r2, yr * r2);   /* +i y / sqrt2 */
        else       vacc_add(v, P2 + q, yi * r2, -yr * r2);   /* -i y / sqrt2 */
    }
    if (Y->diag) {
        double sr = 0, si = 0;                                /* sum_{k<l} Y_kk */
        for (int l = 1; l < N; ++l) {
            size_t pp = (size_t)(l - 1) * N + (l - 1);
            sr += Y->re[pp]; si += Y->im[pp];
            size_t pl = (size_t)l * N + l;
            double c = 1.0 / sqrt((double)l * (l + 1.0));
            double vr = c * (sr - l * Y->re[pl]), vi = c * (si - l * Y->im[pl]);
            if (vr != 0.0 || vi != 0.0) vacc_add(v, 2 * P2 + l - 1, vr, vi);
        }
    }
}

static void vacc_clear(vacc_t *v) {
    for (long long t = 0; t < v->cnt; ++t) { long long s = v->list[t]; v->mark[s] = 0; v->re[s] = 0; v->im[s] = 0; }
    v->cnt = 0;
}

/*
 * Columns `cols[0..ncols)` (all columns when cols == NULL) of G = [Re Tr(F_s L(F_m))],
 * as COO triplets (row s, column m, value); exact zeros are not emitted.
 * With out_* == NULL only counts.  K (length N^2-1) receives Re Tr(F_s L(1/N)) when
 * non-NULL.  *max_imag receives the largest |Im| met (must be rounding-sized).
 * Returns the number of triplets, or -1 on allocation failure.
 */
long long oracle_unfold(int N,
                        const int *h_ptr, const int *h_idx, const double *h_re, const double *h_im,
                        const int *a_ptr, const int *a_idx, const double *a_re, const double *a_im, double gamma,
                        const long long *cols, long long ncols,
                        int *out_row, int *out_col, double *out_val, double *K, double *max_imag) {
    long long D = (long long)N * N - 1;
    gen_t g; memset(&g, 0, sizeof g);
    g.N = N; g.gamma = gamma;
    if (h_ptr) {
        g.hasH = 1;
        g.H.n = N; g.H.ptr = (int *)h_ptr; g.H.idx = (int *)h_idx; g.H.re = (double *)h_re; g.H.im = (double *)h_im;
        g.HT = csr_transpose(N, h_ptr, h_idx, h_re, h_im);
    }
    if (a_ptr) {
        g.hasA = 1;
        g.A.n = N; g.A.ptr = (int *)a_ptr; g.A.idx = (int *)a_idx; g.A.re = (double *)a_re; g.A.im = (double *)a_im;
        g.AT = csr_transpose(N, a_ptr, a_idx, a_re, a_im);
        /* M = A^+ A, M_ab = sum_k conj(A_ka) A_kb, accumulated densely then compressed */
        double *mr = calloc((size_t)N * N, sizeof(double)), *mi = calloc((size_t)N * N, sizeof(double));
        if (!mr || !mi) return -1;
        for (int k = 0; k < N; ++k)
            for (int e = a_ptr[k]; e < a_ptr[k + 1]; ++e)
                for (int f = a_ptr[k]; f < a_ptr[k + 1]; ++f) {
                    int a = a_idx[e], b = a_idx[f];
                    double xr = a_re[e], xi = -a_im[e], yr = a_re[f], yi = a_im[f];
                    mr[(size_t)a * N + b] += xr * yr - xi * yi;
                    mi[(size_t)a * N + b] += xr * yi + xi * yr;
                }
        int nnz = 0;
        for (size_t p = 0; p < (size_t)N * N; ++p) nnz += (mr[p] != 0.0 || mi[p] != 0.0);
        g.M.n = N; g.M.ptr = calloc((size_t)N + 1, sizeof(int));
        g.M.idx = malloc(sizeof(int) * (size_t)(nnz + 1));
        g.M.re = malloc(sizeof(double) * (size_t)(nnz + 1)); g.M.im = malloc(sizeof(double) * (size_t)(nnz + 1));
        int q = 0;
        for (int a = 0; a < N; ++a) {
            for (int b = 0; b < N; ++b) {
                size_t p = (size_t)a * N + b;
                if (mr[p] != 0.0 || mi[p] != 0.0) { g.M.idx[q] = b; g.M.re[q] = mr[p]; g.M.im[q] = mi[p]; ++q; }
            }
            g.M.ptr[a + 1] = q;
        }
        free(mr); free(mi);
        g.MT = csr_transpose(N, g.M.ptr, g.M.idx, g.M.re, g.M.im);
    }

    acc_t Y; Y.N = N; Y.cnt = 0; Y.diag = 0;
    Y.re = calloc((size_t)N * N, sizeof(double)); Y.im = calloc((size_t)N * N, sizeof(double));
    Y.mark = calloc((size_t)N * N, 1); Y.list = malloc(sizeof(int) * (size_t)N * N);
    vacc_t v; v.cnt = 0;
    v.re = calloc((size_t)D, sizeof(double)); v.im = calloc((size_t)D, sizeof(double));
    v.mark = calloc((size_t)D, 1); v.list = malloc(sizeof(long long) * (size_t)D);
    int *ei = malloc(sizeof(int) * (size_t)N), *ej = malloc(sizeof(int) * (size_t)N);
    double *er = malloc(sizeof(double) * (size_t)N), *eim = malloc(sizeof(double) * (size_t)N);
    if (!Y.re || !Y.im || !Y.mark || !Y.list || !v.re || !v.im || !v.mark || !v.list) return -1;

    double mx = 0.0;
    long long out = 0;
    long long nc = cols ? ncols : D;
    for (long long c = 0; c < nc; ++c) {
        long long m = cols ? cols[c] : c;
        int ne = generator_entries(N, m, ei, ej, er, eim);
        apply_L(&g, &Y, ne, ei, ej, er, eim);
        expand_Y(N, &Y, &v);
        for (long long t = 0; t < v.cnt; ++t) {
            long long s = v.list[t];
            if (fabs(v.im[s]) > mx) mx = fabs(v.im[s]);
            if (v.re[s] == 0.0) continue;
            if (out_row) { out_row[out] = (int)s; out_col[out] = (int)m; out_val[out] = v.re[s]; }
            ++out;
        }
        vacc_clear(&v);
        acc_clear(&Y);
    }
    if (K) {
        /* L(1/N): identity entries scaled by 1/N */
        for (int k = 0; k < N; ++k) { ei[k] = k; ej[k] = k; er[k] = 1.0 / N; eim[k] = 0.0; }
        apply_L(&g, &Y, N, ei, ej, er, eim);
        expand_Y(N, &Y, &v);
        memset(K, 0, sizeof(double) * (size_t)D);
        for (long long t = 0; t < v.cnt; ++t) {
            long long s = v.list[t];
            if (fabs(v.im[s]) > mx) mx = fabs(v.im[s]);
            K[s] = v.re[s];
        }
        vacc_clear(&v);
        acc_clear(&Y);
    }
    if (max_imag) *max_imag = mx;

    free(Y.re); free(Y.im); free(Y.mark); free(Y.list);
    free(v.re); free(v.im); free(v.mark); free(v.list);
    free(ei); free(ej); free(er); free(eim);
    if (g.hasH) csr_free(&g.HT);
    if (g.hasA) { csr_free(&g.AT); csr_free(&g.M); csr_free(&g.MT); }
    return out;
}
