// C-ABI entry points of libgksl (include/gksl.h).  Each call validates its arguments, runs its
// work on the context's stream and converts internal errors into a gksl_status.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>

#include "internal.cuh"
#include "prim.cuh"

namespace gk {

[[noreturn]] void throw_cuda(cudaError_t e, const char *what, const char *file, int line) {
    cudaGetLastError();
    throw Error{e == cudaErrorMemoryAllocation ? GKSL_ERR_OOM : GKSL_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" + std::to_string(line) + ")"};
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool device_local_ptr(const void *p, int device) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == device);
}

void copy_in(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return;
    GK_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
    if (!is_device_ptr(src)) GK_CUDA(cudaStreamSynchronize(s));
}

void copy_out(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return;
    GK_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
    if (!is_device_ptr(dst)) GK_CUDA(cudaStreamSynchronize(s));
}

template <typename T>
std::vector<T> to_host(const T *p, size_t n, cudaStream_t s) {
    std::vector<T> h(n);
    if (n) {
        GK_CUDA(cudaMemcpyAsync(h.data(), p, n * sizeof(T), cudaMemcpyDefault, s));
        GK_CUDA(cudaStreamSynchronize(s));
    }
    return h;
}

}  // namespace gk

using namespace gk;

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

template <typename F>
gksl_status guarded(gksl_ctx *c, F &&f) {
    if (!c) return GKSL_ERR_ARG;
    try {
        DeviceGuard g(c->device);
        c->err.clear();
        f();
        return GKSL_OK;
    } catch (const Error &e) {
        c->err = e.msg;
        return e.st;
    } catch (const std::bad_alloc &) {
        c->err = "host allocation failed";
        return GKSL_ERR_OOM;
    } catch (const std::exception &e) {
        c->err = e.what();
        return GKSL_ERR_ARG;
    }
}

// validate a host copy of an N x N CSR operator; optionally check Hermiticity
void validate_csr(int N, const std::vector<int> &rp, const std::vector<int> &col, const std::vector<double> &re,
                  const std::vector<double> &im, int nnz, bool hermitian) {
    GK_REQUIRE(rp[0] == 0 && rp[N] == nnz, GKSL_ERR_ARG, "CSR rowptr must start at 0 and end at nnz");
    std::map<std::pair<int, int>, std::pair<double, double>> ent;
    double mx = 0.0;
    for (int r = 0; r < N; ++r) {
        GK_REQUIRE(rp[r] <= rp[r + 1], GKSL_ERR_ARG, "CSR rowptr must be non-decreasing");
        for (int e = rp[r]; e < rp[r + 1]; ++e) {
            GK_REQUIRE(col[e] >= 0 && col[e] < N, GKSL_ERR_ARG, "CSR column index out of range");
            GK_REQUIRE(std::isfinite(re[e]) && std::isfinite(im[e]), GKSL_ERR_ARG, "non-finite operator entry");
            bool fresh = ent.emplace(std::make_pair(r, col[e]), std::make_pair(re[e], im[e])).second;
            GK_REQUIRE(fresh, GKSL_ERR_ARG, "duplicate (row, column) entry in CSR operator");
            mx = std::max(mx, std::hypot(re[e], im[e]));
        }
    }
    if (!hermitian) return;
    double tol = 1e-12 * (mx > 0 ? mx : 1.0);
    for (auto &kv : ent) {
        int r = kv.first.first, c = kv.first.second;
        auto it = ent.find({c, r});
        double yr = 0, yi = 0;
        if (it != ent.end()) { yr = it->second.first; yi = it->second.second; }
        GK_REQUIRE(std::fabs(kv.second.first - yr) <= tol && std::fabs(kv.second.second + yi) <= tol, GKSL_ERR_ARG,
                   "Hamiltonian operator is not Hermitian");
    }
}

// copy and validate an operator into `op` (no effect on the context's state)
void fill_op(gksl_ctx *c, Op &op, const int *rowptr, const int *col, const double *re, const double *im, int nnz,
             bool hermitian) {
    GK_REQUIRE(nnz > 0 && rowptr && col && re, GKSL_ERR_ARG, "operator arrays must not be null (nnz > 0)");
    int N = c->N;
    Op o;
    o.nnz = nnz;
    o.h_rowptr = to_host(rowptr, (size_t)N + 1, c->stream);
    o.h_col = to_host(col, (size_t)nnz, c->stream);
    o.h_re = to_host(re, (size_t)nnz, c->stream);
    o.h_im = im ? to_host(im, (size_t)nnz, c->stream) : std::vector<double>((size_t)nnz, 0.0);
    validate_csr(N, o.h_rowptr, o.h_col, o.h_re, o.h_im, nnz, hermitian);
    o.rowptr.alloc((size_t)N + 1);
    o.col.alloc((size_t)nnz);
    o.re.alloc((size_t)nnz);
    o.im.alloc((size_t)nnz);
    copy_in(o.rowptr.p, o.h_rowptr.data(), sizeof(int) * (N + 1), c->stream);
    copy_in(o.col.p, o.h_col.data(), sizeof(int) * nnz, c->stream);
    copy_in(o.re.p, o.h_re.data(), sizeof(double) * nnz, c->stream);
    copy_in(o.im.p, o.h_im.data(), sizeof(double) * nnz, c->stream);
    GK_CUDA(cudaStreamSynchronize(c->stream));
    o.set = true;
    o.weight = op.weight;
    op = std::move(o);
}

void set_op(gksl_ctx *c, Op &op, const int *rowptr, const int *col, const double *re, const double *im, int nnz,
            bool hermitian) {
    if (nnz == 0) op = Op();
    else fill_op(c, op, rowptr, col, re, im, nnz, hermitian);
    c->comp_dirty = true;
    c->assembled = false;
}

void ensure_state(gksl_ctx *c) {
    if (c->v.n < (size_t)c->D + 1) {
        c->v.alloc((size_t)c->D + 1);
        double one = 1.0;
        GK_CUDA(cudaMemcpyAsync(c->v.p + c->D, &one, sizeof(double), cudaMemcpyHostToDevice, c->stream));
        GK_CUDA(cudaStreamSynchronize(c->stream));
        clear_graphs(c);
    }
}

// Gershgorin interval of the Hermitian H(eps) = sum theta_k H0_k + eps H1 (host copies)
void gershgorin(const gksl_ctx *c, double eps, double &lo, double &hi) {
    int N = c->N;
    std::vector<std::map<int, std::pair<double, double>>> rows((size_t)N);
    auto add = [&](const Op &o, double w) {
        if (!o.set) return;
        for (int r = 0; r < N; ++r)
            for (int e = o.h_rowptr[r]; e < o.h_rowptr[r + 1]; ++e) {
                auto &x = rows[r][o.h_col[e]];
                x.first += w * o.h_re[e];
                x.second += w * o.h_im[e];
            }
    };
    for (int k = 0; k < GKSL_MAX_H0; ++k) add(c->h0[k], c->h0[k].weight);
    add(c->h1, eps);
    lo = 1e300;
    hi = -1e300;
    for (int r = 0; r < N; ++r) {
        double center = 0.0, rad = 0.0;
        for (auto &kv : rows[r]) {
            if (kv.first == r) center = kv.second.first;
            else rad += std::hypot(kv.second.first, kv.second.second);
        }
        lo = std::min(lo, center - rad);
        hi = std::max(hi, center + rad);
    }
}

}  // namespace

// ====================================================================== lifetime

extern "C" gksl_status gksl_create(int N, int device, void *cuda_stream, gksl_ctx **out) {
    if (!out || N < 2 || N > 4096) return GKSL_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return GKSL_ERR_CUDA;
    }
    gksl_ctx *c = new (std::nothrow) gksl_ctx();
    if (!c) return GKSL_ERR_OOM;
    c->N = N;
    c->P2 = (long long)N * (N - 1) / 2;
    c->D = (long long)N * N - 1;
    c->device = device;
    gksl_status st = guarded(c, [&] {
        if (cuda_stream) {
            c->stream = (cudaStream_t)cuda_stream;
        } else {
            GK_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
            c->own_stream = true;
        }
    });
    if (st != GKSL_OK) {
        delete c;
        return st;
    }
    *out = c;
    return GKSL_OK;
}

extern "C" void gksl_destroy(gksl_ctx *c) {
    if (!c) return;
    {
        DeviceGuard g(c->device);
        cudaStreamSynchronize(c->stream);
        clear_graphs(c);
        if (c->own_stream) cudaStreamDestroy(c->stream);
    }
    delete c;
}

extern "C" const char *gksl_last_error(const gksl_ctx *c) { return c ? c->err.c_str() : "null context"; }

// ====================================================================== inputs

extern "C" gksl_status gksl_set_h0_component(gksl_ctx *c, int k, double theta, const int *rowptr, const int *col,
                                             const double *re, const double *im, int nnz) {
    return guarded(c, [&] {
        GK_REQUIRE(k >= 0 && k < GKSL_MAX_H0, GKSL_ERR_ARG, "component index out of range");
        GK_REQUIRE(std::isfinite(theta), GKSL_ERR_ARG, "theta must be finite");
        set_op(c, c->h0[k], rowptr, col, re, im, nnz, true);
        c->h0[k].weight = theta;
    });
}

extern "C" gksl_status gksl_set_theta(gksl_ctx *c, int k, double theta) {
    return guarded(c, [&] {
        GK_REQUIRE(k >= 0 && k < GKSL_MAX_H0 && c->h0[k].set, GKSL_ERR_ARG, "component not set");
        GK_REQUIRE(std::isfinite(theta), GKSL_ERR_ARG, "theta must be finite");
        c->h0[k].weight = theta;
        c->assembled = false;
    });
}

extern "C" gksl_status gksl_set_h1(gksl_ctx *c, const int *rowptr, const int *col, const double *re, const double *im,
                                   int nnz) {
    return guarded(c, [&] { set_op(c, c->h1, rowptr, col, re, im, nnz, true); });
}

extern "C" gksl_status gksl_set_dissipator(gksl_ctx *c, int p, double gamma, const int *rowptr, const int *col,
                                           const double *re, const double *im, int nnz) {
    return guarded(c, [&] {
        GK_REQUIRE(p >= 0 && p < GKSL_MAX_P, GKSL_ERR_ARG, "channel index out of range");
        GK_REQUIRE(std::isfinite(gamma) && gamma >= 0.0, GKSL_ERR_ARG, "gamma_p must be finite and >= 0");
        if (c->diss[p].km) c->km_A.release();   // the Kossakowski matrix this channel held
        set_op(c, c->diss[p], rowptr, col, re, im, nnz, false);
        c->diss[p].weight = gamma;
    });
}

extern "C" gksl_status gksl_set_gamma(gksl_ctx *c, int p, double gamma) {
    return guarded(c, [&] {
        GK_REQUIRE(p >= 0 && p < GKSL_MAX_P && c->diss[p].set, GKSL_ERR_ARG, "channel not set");
        GK_REQUIRE(std::isfinite(gamma) && gamma >= 0.0, GKSL_ERR_ARG, "gamma_p must be finite and >= 0");
        c->diss[p].weight = gamma;
        c->assembled = false;
    });
}

extern "C" gksl_status gksl_set_drive(gksl_ctx *c, double E, double A, double omega) {
    return guarded(c, [&] {
        GK_REQUIRE(std::isfinite(E) && std::isfinite(A) && std::isfinite(omega) && omega > 0.0, GKSL_ERR_ARG,
                   "drive parameters must be finite with omega > 0");
        if (c->E != E) c->assembled = false;
        c->E = E;
        c->A = A;
        c->omega = omega;
        c->drive_set = true;
        clear_graphs(c);
    });
}

// Kossakowski matrix (Eq. 8).  A = sum_p c_p c_p^+ by a diagonally pivoted Cholesky factorisation
// (exact for a positive semidefinite A of rank <= GKSL_MAX_P); then gamma_p = |c_p|^2,
// l_p = c_p / |c_p|, L_p = sum_j l_pj F_j.  Any such rank factorisation gives the same Lindbladian
// as the eigen-decomposition of Eq. 9 (the dissipator is invariant under a unitary remixing of its
// channels).  A matrix of higher rank, or any A at N > 64, is kept whole on the device and
// assembled by the dense route (dense_diss.cu) as channel 0 at unit weight; at N > 64 it is
// copied and checked on the device (kossakowski_upload_checked), below on the host.
extern "C" gksl_status gksl_set_kossakowski(gksl_ctx *c, const double *a_re, const double *a_im, double tol) {
    return guarded(c, [&] {
        GK_REQUIRE(a_re && tol >= 0.0, GKSL_ERR_ARG, "a_re must not be null and tol >= 0");
        const long long D = c->D;
        const int N = c->N;
        GK_REQUIRE(N <= kDenseKmMaxN, GKSL_ERR_ARG, "the Kossakowski form is limited to N <= 128");
        if (N > 64) {
            // dense route without a rank factorisation: the matrix goes to the device and is
            // checked there (the same conditions and messages as below), then replaces the channels
            DBuf<double2> A;
            const double tr = kossakowski_upload_checked(c, a_re, a_im, A);
            for (int p = 0; p < GKSL_MAX_P; ++p)
                if (c->diss[p].set) c->diss[p] = Op();
            c->km_A = std::move(A);
            c->comp_dirty = true;
            c->assembled = false;
            Op &o = c->diss[0];
            o.set = true;
            o.km = true;
            o.km_trace = tr;
            o.weight = 1.0;
            return;
        }
        size_t DD = (size_t)D * D;
        std::vector<double> ar = to_host(a_re, DD, c->stream), ai = a_im ? to_host(a_im, DD, c->stream)
                                                                         : std::vector<double>(DD, 0.0);
        double mx = 0.0;
        for (size_t i = 0; i < DD; ++i) {
            GK_REQUIRE(std::isfinite(ar[i]) && std::isfinite(ai[i]), GKSL_ERR_ARG, "non-finite Kossakowski entry");
            mx = std::max(mx, std::hypot(ar[i], ai[i]));
        }
        for (long long j = 0; j < D; ++j)
            for (long long k = j; k < D; ++k)
                GK_REQUIRE(std::fabs(ar[j * D + k] - ar[k * D + j]) <= 1e-12 * mx &&
                               std::fabs(ai[j * D + k] + ai[k * D + j]) <= 1e-12 * mx,
                           GKSL_ERR_ARG, "Kossakowski matrix is not Hermitian");
        double dmax0 = 0.0;
        for (long long j = 0; j < D; ++j) dmax0 = std::max(dmax0, ar[j * D + j]);
        const double thr = tol * std::max(dmax0, 1e-300);
        // pivoted Cholesky on the residual R = A - sum c c^+, at most GKSL_MAX_P pivots (N <= 64)
        std::vector<std::vector<double>> cr, ci;
        bool low_rank = false;
        if (N <= 64) {
            std::vector<double> rr = ar, ri = ai;
            for (;;) {
                long long piv = -1;
                double best = thr;
                for (long long j = 0; j < D; ++j)
                    if (rr[j * D + j] > best) { best = rr[j * D + j]; piv = j; }
                if (piv < 0) { low_rank = true; break; }
                if ((int)cr.size() == GKSL_MAX_P) break;   // rank above the channel count: dense route
                double sc = 1.0 / std::sqrt(best);
                std::vector<double> vr((size_t)D), vi((size_t)D);
                for (long long i = 0; i < D; ++i) {   // c = R[:, piv] / sqrt(R[piv, piv])
                    vr[i] = rr[i * D + piv] * sc;
                    vi[i] = ri[i * D + piv] * sc;
                }
                for (long long i = 0; i < D; ++i)
                    for (long long k = 0; k < D; ++k) {   // R -= c c^+
                        rr[i * D + k] -= vr[i] * vr[k] + vi[i] * vi[k];
                        ri[i * D + k] -= vi[i] * vr[k] - vr[i] * vi[k];
                    }
                cr.push_back(std::move(vr));
                ci.push_back(std::move(vi));
            }
            if (low_rank)
                for (long long j = 0; j < D; ++j)
                    GK_REQUIRE(rr[j * D + j] >= -std::max(thr, 1e-12 * dmax0), GKSL_ERR_ARG,
                               "Kossakowski matrix is not positive semidefinite");
        }
        // dense route: necessary conditions of positive semidefiniteness, checked before the
        // context changes (a rejected matrix leaves the previous channels in place)
        double tr = 0.0;
        if (!low_rank) {
            const double eps = 1e-12 * mx;
            for (long long j = 0; j < D; ++j) {
                GK_REQUIRE(ar[j * D + j] >= -eps, GKSL_ERR_ARG, "Kossakowski matrix is not positive semidefinite");
                tr += ar[j * D + j];
            }
            for (long long j = 0; j < D; ++j)
                for (long long k = j + 1; k < D; ++k) {
                    double m2 = ar[j * D + k] * ar[j * D + k] + ai[j * D + k] * ai[j * D + k];
                    double dd = std::max(ar[j * D + j], 0.0) * std::max(ar[k * D + k], 0.0);
                    GK_REQUIRE(m2 <= dd + eps * mx * 4.0, GKSL_ERR_ARG,
                               "Kossakowski matrix is not positive semidefinite (a 2 x 2 principal minor is negative)");
                }
        }
        c->km_A.release();
        for (int p = 0; p < GKSL_MAX_P; ++p)
            if (c->diss[p].set) c->diss[p] = Op();
        c->comp_dirty = true;
        c->assembled = false;
        if (!low_rank) {   // A kept whole on the device, channel 0 at unit weight
            std::vector<double2> h(DD);
            for (size_t i = 0; i < DD; ++i) h[i] = make_double2(ar[i], ai[i]);
            c->km_A.alloc(DD);
            GK_CUDA(cudaMemcpy(c->km_A.p, h.data(), sizeof(double2) * DD, cudaMemcpyHostToDevice));
            Op &o = c->diss[0];
            o.set = true;
            o.km = true;
            o.km_trace = tr;
            o.weight = 1.0;
            return;
        }
        // channels L_p = sum_j l_pj F_j as dense N x N matrices, then CSR
        Basis B(N);
        const double r2 = GK_RSQRT2;
        for (int p = 0; p < (int)cr.size(); ++p) {
            double g = 0.0;
            for (long long j = 0; j < D; ++j) g += cr[p][j] * cr[p][j] + ci[p][j] * ci[p][j];
            double inv = 1.0 / std::sqrt(g);
            std::vector<double> Lr((size_t)N * N, 0.0), Li((size_t)N * N, 0.0);
            for (long long j = 0; j < D; ++j) {
                double xr = cr[p][j] * inv, xi = ci[p][j] * inv;
                if (xr == 0.0 && xi == 0.0) continue;
                El e = B.decode(j);
                if (e.kind == 0) {          // S: 1/sqrt2 at (a,b), (b,a)
                    Lr[e.a * N + e.b] += xr * r2; Li[e.a * N + e.b] += xi * r2;
                    Lr[e.b * N + e.a] += xr * r2; Li[e.b * N + e.a] += xi * r2;
                } else if (e.kind == 1) {   // J: -i/sqrt2 at (a,b), +i/sqrt2 at (b,a)
                    Lr[e.a * N + e.b] += xi * r2; Li[e.a * N + e.b] -= xr * r2;
                    Lr[e.b * N + e.a] -= xi * r2; Li[e.b * N + e.a] += xr * r2;
                } else {                    // D^l: c_l on k < l, -l c_l at l
                    for (int k = 0; k <= e.a; ++k) {
                        double dk = dl_diag(e.a, k);
                        Lr[k * N + k] += xr * dk;
                        Li[k * N + k] += xi * dk;
                    }
                }
            }
            std::vector<int> rp((size_t)N + 1, 0), cc;
            std::vector<double> vr, vi;
            for (int r = 0; r < N; ++r) {
                for (int k = 0; k < N; ++k)
                    if (Lr[r * N + k] != 0.0 || Li[r * N + k] != 0.0) {
                        cc.push_back(k);
                        vr.push_back(Lr[r * N + k]);
                        vi.push_back(Li[r * N + k]);
                    }
                rp[r + 1] = (int)cc.size();
            }
            set_op(c, c->diss[p], rp.data(), cc.data(), vr.data(), vi.data(), (int)cc.size(), false);
            c->diss[p].weight = g;
        }
    });
}

extern "C" gksl_status gksl_set_drive_shape(gksl_ctx *c, int shape) {
    return guarded(c, [&] {
        GK_REQUIRE(shape == GKSL_DRIVE_SIN || shape == GKSL_DRIVE_SQUARE, GKSL_ERR_ARG, "unknown drive shape");
        c->drive_shape = shape;
        clear_graphs(c);
    });
}

// ====================================================================== expansion

extern "C" gksl_status gksl_expand(gksl_ctx *c, const int *rowptr, const int *col, const double *re, const double *im,
                                   int nnz, double *coef_re, double *coef_im) {
    return guarded(c, [&] {
        GK_REQUIRE(coef_re, GKSL_ERR_ARG, "coef_re must not be null");
        Op o;
        if (nnz > 0) fill_op(c, o, rowptr, col, re, im, nnz, false);
        else {
            o.rowptr.alloc((size_t)c->N + 1);
            GK_CUDA(cudaMemsetAsync(o.rowptr.p, 0, sizeof(int) * (c->N + 1), c->stream));
        }
        DBuf<double2> coef;
        expand_op(c, o, coef);
        std::vector<double2> h = to_host(coef.p, (size_t)c->D, c->stream);
        std::vector<double> r((size_t)c->D), i((size_t)c->D);
        for (long long s = 0; s < c->D; ++s) { r[s] = h[s].x; i[s] = h[s].y; }
        copy_out(coef_re, r.data(), sizeof(double) * c->D, c->stream);
        if (coef_im) copy_out(coef_im, i.data(), sizeof(double) * c->D, c->stream);
    });
}

// ====================================================================== structure constants

extern "C" gksl_status gksl_structure_count(int N, int which, long long *count) {
    if (!count || N < 2 || N > 4096 || (which != 0 && which != 1)) return GKSL_ERR_ARG;
    try {
        *count = structure_count(N, which, 0);
        return GKSL_OK;
    } catch (const Error &e) {
        return e.st;
    }
}

extern "C" gksl_status gksl_structure_enumerate(int N, int which, long long capacity, int *m, int *n, int *s,
                                                double *value, long long *count) {
    if (!count || N < 2 || N > 4096 || (which != 0 && which != 1)) return GKSL_ERR_ARG;
    try {
        long long total = structure_count(N, which, 0);
        *count = total;
        if (total > capacity || !m || !n || !s || !value) return GKSL_ERR_ARG;
        DBuf<int> dm((size_t)total), dn((size_t)total), ds((size_t)total);
        DBuf<double> dv((size_t)total);
        long long got = structure_enumerate(N, which, total, dm.p, dn.p, ds.p, dv.p, 0);
        if (got != total) return GKSL_ERR_CUDA;
        copy_out(m, dm.p, sizeof(int) * total, 0);
        copy_out(n, dn.p, sizeof(int) * total, 0);
        copy_out(s, ds.p, sizeof(int) * total, 0);
        copy_out(value, dv.p, sizeof(double) * total, 0);
        GK_CUDA(cudaDeviceSynchronize());
        return GKSL_OK;
    } catch (const Error &e) {
        return e.st;
    }
}

// ====================================================================== assembly

extern "C" gksl_status gksl_assemble(gksl_ctx *c, unsigned flags, double *seconds) {
    return guarded(c, [&] {
        NvtxRange r("gksl_assemble");
        assemble(c, flags);
        if (seconds) *seconds = c->assemble_seconds;
    });
}

extern "C" gksl_status gksl_get_csr(gksl_ctx *c, int which, long long *nnz, int *rowptr, int *col, double *val) {
    return guarded(c, [&] {
        GK_REQUIRE(nnz, GKSL_ERR_ARG, "nnz must not be null");
        GK_REQUIRE(c->assembled, GKSL_ERR_STATE, "gksl_assemble must be called first");
        GK_REQUIRE(!(c->asm_flags & GKSL_ASM_MATRIX_FREE), GKSL_ERR_STATE, "assembled matrix-free: no CSR matrix");
        const CsrR *m = nullptr;
        if (which == GKSL_MAT_Q0) m = &c->Q0;
        else if (which == GKSL_MAT_Q1) m = &c->Q1;
        else if (which >= GKSL_MAT_H0 && which < GKSL_MAT_H0 + GKSL_MAX_H0 && c->has_h0[which - GKSL_MAT_H0])
            m = &c->QH0[which - GKSL_MAT_H0];
        else if (which >= GKSL_MAT_R && which < GKSL_MAT_R + GKSL_MAX_P && c->has_r[which - GKSL_MAT_R])
            m = &c->R[which - GKSL_MAT_R];
        GK_REQUIRE(m, GKSL_ERR_ARG, "no such matrix");
        csr_copy_out(c, *m, nnz, rowptr, col, val);
    });
}

extern "C" gksl_status gksl_get_k(gksl_ctx *c, double *K) {
    return guarded(c, [&] {
        GK_REQUIRE(K, GKSL_ERR_ARG, "K must not be null");
        GK_REQUIRE(c->assembled, GKSL_ERR_STATE, "gksl_assemble must be called first");
        GK_REQUIRE(!(c->asm_flags & GKSL_ASM_MATRIX_FREE), GKSL_ERR_STATE, "assembled matrix-free: no K vector");
        copy_out(K, c->K.p, sizeof(double) * c->D, c->stream);
    });
}

extern "C" gksl_status gksl_get_k_channel(gksl_ctx *c, int p, double *K) {
    return guarded(c, [&] {
        GK_REQUIRE(K, GKSL_ERR_ARG, "K must not be null");
        GK_REQUIRE(c->assembled, GKSL_ERR_STATE, "gksl_assemble must be called first");
        GK_REQUIRE(!(c->asm_flags & GKSL_ASM_MATRIX_FREE), GKSL_ERR_STATE, "assembled matrix-free: no K vector");
        GK_REQUIRE(p >= 0 && p < GKSL_MAX_P && c->has_r[p], GKSL_ERR_ARG, "channel not set");
        copy_out(K, c->Kp[p].p, sizeof(double) * c->D, c->stream);
    });
}

// ====================================================================== state

extern "C" gksl_status gksl_set_rho0(gksl_ctx *c, const double *re, const double *im) {
    return guarded(c, [&] {
        GK_REQUIRE(re, GKSL_ERR_ARG, "re must not be null");
        ensure_state(c);
        size_t n2 = (size_t)c->N * c->N;
        DBuf<double> dre(n2), dim(n2);
        copy_in(dre.p, re, sizeof(double) * n2, c->stream);
        if (im) copy_in(dim.p, im, sizeof(double) * n2, c->stream);
        expand_dense(c, dre.p, im ? dim.p : nullptr, c->v.p);
        c->t = 0.0;
        c->state_set = true;
    });
}

extern "C" gksl_status gksl_set_state(gksl_ctx *c, const double *v, double t) {
    return guarded(c, [&] {
        GK_REQUIRE(v && std::isfinite(t), GKSL_ERR_ARG, "v must not be null and t finite");
        ensure_state(c);
        copy_in(c->v.p, v, sizeof(double) * c->D, c->stream);
        GK_CUDA(cudaStreamSynchronize(c->stream));
        c->t = t;
        c->state_set = true;
    });
}

extern "C" gksl_status gksl_get_state(gksl_ctx *c, double *v, double *t) {
    return guarded(c, [&] {
        GK_REQUIRE(c->state_set, GKSL_ERR_STATE, "no state set");
        if (v) copy_out(v, c->v.p, sizeof(double) * c->D, c->stream);
        GK_CUDA(cudaStreamSynchronize(c->stream));
        if (t) *t = c->t;
    });
}

// ====================================================================== propagation

extern "C" gksl_status gksl_min_stable_steps(gksl_ctx *c, long long *spp) {
    return guarded(c, [&] {
        GK_REQUIRE(spp, GKSL_ERR_ARG, "steps_per_period must not be null");
        GK_REQUIRE(c->drive_set, GKSL_ERR_STATE, "drive not set");
        // ||L_H|| <= spread of H(t) (Gershgorin, extreme at eps = E +- A); ||L_D|| <= 2 sum gamma ||L||^2
        double spread = 0.0;
        for (double eps : {c->E - c->A, c->E + c->A}) {
            double lo, hi;
            gershgorin(c, eps, lo, hi);
            spread = std::max(spread, hi - lo);
        }
        double diss = 0.0;
        for (int p = 0; p < GKSL_MAX_P; ++p) {
            const Op &o = c->diss[p];
            if (!o.set) continue;
            if (o.km) {   // sum_p gamma_p |L_p|_2^2 <= sum_p gamma_p |L_p|_F^2 = Tr A for any factorisation
                diss += 2.0 * o.weight * o.km_trace;
                continue;
            }
            std::vector<double> rs((size_t)c->N, 0.0), cs((size_t)c->N, 0.0);
            for (int r = 0; r < c->N; ++r)
                for (int e = o.h_rowptr[r]; e < o.h_rowptr[r + 1]; ++e) {
                    double a = std::hypot(o.h_re[e], o.h_im[e]);
                    rs[r] += a;
                    cs[o.h_col[e]] += a;
                }
            double n1 = *std::max_element(cs.begin(), cs.end()), ni = *std::max_element(rs.begin(), rs.end());
            diss += 2.0 * o.weight * n1 * ni;
        }
        double bound = spread + diss;
        double T = 2.0 * M_PI / c->omega;
        long long n = (long long)std::ceil(T * bound / 2.6);
        *spp = n < 1 ? 1 : n;
    });
}

extern "C" gksl_status gksl_propagate(gksl_ctx *c, long long spp, long long n_steps, int precision,
                                      long long correction_every, long long emit_every, double *v_out) {
    return guarded(c, [&] {
        NvtxRange r("gksl_propagate");
        bool dev = is_device_ptr(v_out);
        propagate(c, spp, n_steps, precision, correction_every, emit_every, v_out, dev);
    });
}

// ====================================================================== observables

extern "C" gksl_status gksl_observable_diag(gksl_ctx *c, const double *o_diag, const double *v, long long count,
                                            double *out) {
    return guarded(c, [&] {
        GK_REQUIRE(o_diag && v && out && count >= 0, GKSL_ERR_ARG, "null argument");
        DBuf<double> o((size_t)c->N), res((size_t)(count > 0 ? count : 1));
        copy_in(o.p, o_diag, sizeof(double) * c->N, c->stream);
        const double *vd = v;
        DBuf<double> vtmp;
        if (!device_local_ptr(v, c->device)) {   // host memory or another GPU's: copy it here first
            vtmp.alloc((size_t)(count * c->D));
            copy_in(vtmp.p, v, sizeof(double) * count * c->D, c->stream);
            vd = vtmp.p;
        }
        observable_diag(c, o.p, vd, count, c->D, res.p);
        copy_out(out, res.p, sizeof(double) * count, c->stream);
    });
}

extern "C" gksl_status gksl_rho(gksl_ctx *c, const double *v, double *re, double *im) {
    return guarded(c, [&] {
        GK_REQUIRE(v && re && im, GKSL_ERR_ARG, "null argument");
        size_t n2 = (size_t)c->N * c->N;
        DBuf<double> vd((size_t)c->D), dre(n2), dim(n2);
        copy_in(vd.p, v, sizeof(double) * c->D, c->stream);
        rho_dense(c, vd.p, dre.p, dim.p);
        copy_out(re, dre.p, sizeof(double) * n2, c->stream);
        copy_out(im, dim.p, sizeof(double) * n2, c->stream);
    });
}

// ====================================================================== adjoint

extern "C" gksl_status gksl_adjoint_timeavg(gksl_ctx *c, const double *o_diag, long long spp, long long period,
                                            int precision, double *loss, double *grad, int n_grad) {
    return guarded(c, [&] {
        NvtxRange r("gksl_adjoint_timeavg");
        GK_REQUIRE(o_diag && loss && (grad || n_grad == 0), GKSL_ERR_ARG, "null argument");
        GK_REQUIRE(spp > 0 && period >= 1, GKSL_ERR_ARG, "steps_per_period > 0 and period_index >= 1 required");
        DBuf<double> o((size_t)c->N);
        copy_in(o.p, o_diag, sizeof(double) * c->N, c->stream);
        adjoint_timeavg(c, o.p, spp, period, precision, loss, grad, n_grad);
    });
}

// ====================================================================== introspection

extern "C" gksl_status gksl_get_info(gksl_ctx *c, gksl_info *out) {
    return guarded(c, [&] {
        GK_REQUIRE(out, GKSL_ERR_ARG, "null argument");
        memset(out, 0, sizeof *out);
        out->N = c->N;
        out->D = c->D;
        out->nnz_q0 = c->nnz_q0e;
        out->nnz_q1 = c->Q1.nnz;
        for (int p = 0; p < GKSL_MAX_P; ++p) out->nnz_r[p] = c->has_r[p] ? c->R[p].nnz : 0;
        out->ell_width_q0 = c->hyb0.width;
        out->ell_width_q1 = c->hyb1.width;
        out->long_rows = c->hyb0.n_long;
        size_t b = c->Q0.bytes() + c->Q1.bytes() + c->K.bytes() + c->hyb0.bytes() + c->hyb1.bytes() + c->hyb0f.bytes() +
                   c->q1v.bytes() + c->q1vf.bytes() +
                   c->hyb1f.bytes() + c->v.bytes() + c->yA.bytes() + c->yB.bytes() + c->acc.bytes() + c->v32.bytes() +
                   c->yA32.bytes() + c->yB32.bytes() + c->acc32.bytes() + c->eps_tab.bytes();
        for (int k = 0; k < GKSL_MAX_H0; ++k) b += c->QH0[k].bytes();
        for (int p = 0; p < GKSL_MAX_P; ++p) b += c->R[p].bytes() + c->Kp[p].bytes();
        for (int i = 0; i < c->adj_n; ++i) b += c->adj[i].bytes() + c->adjf[i].bytes();
        const MfBands &m = c->mf;
        b += m.h0.bytes() + m.h1.bytes() + m.g.bytes() + m.l.bytes() + m.r32.bytes() + m.h1o32.bytes() +
             m.dg32.bytes() + m.lo32.bytes() + m.ld32.bytes() + m.tiles.bytes();
        for (int i = 0; i < 4; ++i) b += m.img64[i].bytes() + m.img32[i].bytes();
        out->device_bytes = (long long)b;
        out->assemble_seconds = c->assemble_seconds;
        out->max_abs_q0 = c->max_abs_q0;
        out->q1_folded = c->q1_folded ? 1 : 0;
        out->compact_columns[0] = c->hyb0.ell_c16.p ? 1 : 0;
        out->compact_columns[1] = c->hyb0f.ell_c16.p ? 1 : 0;
        out->compact_escaped_rows = c->hyb0.ell_c16.p ? c->hyb0.n_esc : 0;
        out->tail_nnz = c->hyb0.tail_nnz;
        for (int p = 0; p < 2; ++p) {
            out->rk4_variant[p] = c->rk4_var[p];
            out->rk4_compact[p] = c->rk4_c16[p] && c->rk4_var[p] != 2 ? 1 : 0;
            for (int v = 0; v < 4; ++v) {
                out->rk4_variant_us[p][v] = c->rk4_var_us[p][v];
                out->rk4_variant_us_c16[p][v] = c->rk4_var_us_c16[p][v];
            }
        }
    });
}
