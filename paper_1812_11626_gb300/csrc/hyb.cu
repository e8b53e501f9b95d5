// CSR -> hybrid propagation format.  Most rows of the unfolded dimer have the same length
// (18 entries at N = 1000), so an ELL block stored slot-major gives fully coalesced loads
// with one thread per row; the few long rows (the S^(j,j+1) rows that reach every D^l) go
// to warp-per-row CSR tails.  Matrices that are applied together share one long-row set,
// and the first of them marks a long row with column -1 in ELL slot 0.
#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "prim.cuh"

namespace gk {

namespace {

constexpr int kCap = 64;   // widths are chosen below this; longer rows always go to the tails

__global__ void k_rowlens(const int *__restrict__ rowptr, long long rows, int *__restrict__ len) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < rows) len[r] = rowptr[r + 1] - rowptr[r];
}

__global__ void k_hist(const int *__restrict__ len, long long rows, unsigned long long *__restrict__ hist) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    int l = len[r];
    atomicAdd(&hist[l < kCap ? l : kCap], 1ull);
    if (l >= kCap) atomicAdd(&hist[kCap + 1], (unsigned long long)l);
}

__global__ void k_long_flags(const int *const *__restrict__ lens, const int *__restrict__ widths, int nm,
                             long long rows, long long *__restrict__ flag) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    int lg = 0;
    for (int i = 0; i < nm; ++i) lg |= lens[i][r] > widths[i];
    flag[r] = lg;
}

__global__ void k_long_list(const long long *__restrict__ flag, const long long *__restrict__ pos, long long rows,
                            int *__restrict__ list) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < rows && flag[r]) list[pos[r]] = (int)r;
}

template <typename VT>
__global__ void k_ell_fill(const int *__restrict__ rowptr, const int *__restrict__ col, const double *__restrict__ val,
                           double scale, long long rows, long long ld, int W, const long long *__restrict__ is_long,
                           bool mark, int *__restrict__ ecol, VT *__restrict__ evals) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ld) return;
    if (r >= rows) {
        for (int j = 0; j < W; ++j) { ecol[(long long)j * ld + r] = 0; evals[(long long)j * ld + r] = VT(0); }
        return;
    }
    int j = 0;
    if (!is_long[r]) {
        for (int e = rowptr[r]; e < rowptr[r + 1]; ++e, ++j) {
            ecol[(long long)j * ld + r] = col[e];
            evals[(long long)j * ld + r] = (VT)(scale * val[e]);
        }
    }
    for (; j < W; ++j) {
        ecol[(long long)j * ld + r] = (j == 0 && mark && is_long[r]) ? -1 : (int)r;
        evals[(long long)j * ld + r] = VT(0);
    }
}

__global__ void k_tail_lens(const int *__restrict__ rowptr, const int *__restrict__ list, long long nl,
                            long long *__restrict__ cnt) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nl) cnt[i] = rowptr[list[i] + 1] - rowptr[list[i]];
}

template <typename VT>
__global__ void k_tail_fill(const int *__restrict__ rowptr, const int *__restrict__ col, const double *__restrict__ val,
                            double scale, const int *__restrict__ list, long long nl, const long long *__restrict__ tp,
                            int *__restrict__ tptr, int *__restrict__ tcol, VT *__restrict__ tval) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > nl) return;
    tptr[i] = (int)tp[i];
    if (i == nl) return;
    int r = list[i];
    long long o = tp[i];
    for (int e = rowptr[r]; e < rowptr[r + 1]; ++e, ++o) {
        tcol[o] = col[e];
        tval[o] = (VT)(scale * val[e]);
    }
}

int choose_width(const std::vector<unsigned long long> &h, long long rows) {
    // bytes ~ rows * W slots + long rows at their length plus a warp's worth of overhead
    const double over = 8.0;
    int best = 1;
    double best_cost = 1e300;
    for (int W = 1; W < kCap; ++W) {
        double cost = (double)rows * W;
        for (int l = W + 1; l < kCap; ++l) cost += (double)h[l] * (l + over);
        cost += (double)h[kCap + 1] + over * (double)h[kCap];
        if (cost < best_cost) { best_cost = cost; best = W; }
    }
    return best;
}

template <typename VT>
void fill_one(const CsrR &a, double scale, long long rows, long long ld, int W, const long long *is_long, bool mark,
              const int *list, long long nl, const long long *tp, long long tnnz, Hyb<VT> &h, cudaStream_t s) {
    h.rows = rows;
    h.ld = ld;
    h.width = W;
    h.ell_col.alloc((size_t)(ld * W));
    h.ell_val.alloc((size_t)(ld * W));
    k_ell_fill<VT><<<grid_for(ld, 256), 256, 0, s>>>(a.rowptr.p, a.col.p, a.val.p, scale, rows, ld, W, is_long, mark,
                                                      h.ell_col.p, h.ell_val.p);
    GK_LAUNCH_CHECK();
    h.n_long = nl;
    h.tail_nnz = tnnz;
    h.tail_ptr.alloc((size_t)nl + 1);
    h.tail_col.alloc((size_t)(tnnz > 0 ? tnnz : 1));
    h.tail_val.alloc((size_t)(tnnz > 0 ? tnnz : 1));
    k_tail_fill<VT><<<grid_for(nl + 1, 256), 256, 0, s>>>(a.rowptr.p, a.col.p, a.val.p, scale, list, nl, tp,
                                                           h.tail_ptr.p, h.tail_col.p, h.tail_val.p);
    GK_LAUNCH_CHECK();
}

// Build the formats of a set of matrices that share rows and one long-row set.
void build_set(const std::vector<const CsrR *> &ms, const std::vector<double> &scales, long long rows,
               const std::vector<Hyb<double> *> &out, const std::vector<Hyb<float> *> &outf, cudaStream_t s) {
    int nm = (int)ms.size();
    std::vector<DBuf<int>> lens(nm);
    std::vector<int> widths(nm);
    for (int i = 0; i < nm; ++i) {
        lens[i].alloc((size_t)rows);
        k_rowlens<<<grid_for(rows, 256), 256, 0, s>>>(ms[i]->rowptr.p, rows, lens[i].p);
        GK_LAUNCH_CHECK();
        DBuf<unsigned long long> hist(kCap + 2);
        GK_CUDA(cudaMemsetAsync(hist.p, 0, sizeof(unsigned long long) * (kCap + 2), s));
        k_hist<<<grid_for(rows, 256), 256, 0, s>>>(lens[i].p, rows, hist.p);
        GK_LAUNCH_CHECK();
        std::vector<unsigned long long> h(kCap + 2);
        GK_CUDA(cudaMemcpyAsync(h.data(), hist.p, sizeof(unsigned long long) * (kCap + 2), cudaMemcpyDeviceToHost, s));
        GK_CUDA(cudaStreamSynchronize(s));
        widths[i] = choose_width(h, rows);
    }
    std::vector<const int *> lp(nm);
    for (int i = 0; i < nm; ++i) lp[i] = lens[i].p;
    DBuf<const int *> dlens((size_t)nm);
    DBuf<int> dw((size_t)nm);
    GK_CUDA(cudaMemcpyAsync(dlens.p, lp.data(), sizeof(const int *) * nm, cudaMemcpyHostToDevice, s));
    GK_CUDA(cudaMemcpyAsync(dw.p, widths.data(), sizeof(int) * nm, cudaMemcpyHostToDevice, s));
    DBuf<long long> flag((size_t)rows), pos((size_t)rows + 1);
    k_long_flags<<<grid_for(rows, 256), 256, 0, s>>>(dlens.p, dw.p, nm, rows, flag.p);
    GK_LAUNCH_CHECK();
    long long nl = scan_ll(flag.p, pos.p, rows, true, true, s);
    DBuf<int> list((size_t)(nl > 0 ? nl : 1));
    k_long_list<<<grid_for(rows, 256), 256, 0, s>>>(flag.p, pos.p, rows, list.p);
    GK_LAUNCH_CHECK();
    long long ld = (rows + 31) / 32 * 32;
    for (int i = 0; i < nm; ++i) {
        DBuf<long long> cnt((size_t)(nl > 0 ? nl : 1)), tp((size_t)nl + 1);
        if (nl > 0) {
            k_tail_lens<<<grid_for(nl, 256), 256, 0, s>>>(ms[i]->rowptr.p, list.p, nl, cnt.p);
            GK_LAUNCH_CHECK();
        }
        long long tnnz = scan_ll(cnt.p, tp.p, nl, true, true, s);
        if (out[i]) fill_one<double>(*ms[i], scales[i], rows, ld, widths[i], flag.p, i == 0, list.p, nl, tp.p, tnnz,
                                     *out[i], s);
        if (outf[i]) fill_one<float>(*ms[i], scales[i], rows, ld, widths[i], flag.p, i == 0, list.p, nl, tp.p, tnnz,
                                     *outf[i], s);
        GK_CUDA(cudaStreamSynchronize(s));
    }
    for (int i = 0; i < nm; ++i) {
        if (out[i]) { out[i]->long_rows.alloc((size_t)(nl > 0 ? nl : 1)); }
        if (outf[i]) { outf[i]->long_rows.alloc((size_t)(nl > 0 ? nl : 1)); }
        if (nl > 0) {
            if (out[i])
                GK_CUDA(cudaMemcpyAsync(out[i]->long_rows.p, list.p, sizeof(int) * nl, cudaMemcpyDeviceToDevice, s));
            if (outf[i])
                GK_CUDA(cudaMemcpyAsync(outf[i]->long_rows.p, list.p, sizeof(int) * nl, cudaMemcpyDeviceToDevice, s));
        }
    }
    GK_CUDA(cudaStreamSynchronize(s));
}

// Rows that keep Q1 out of slot 0: more than one Q1 entry, or its column missing from the
// row's [Q0 + E Q1] entries with no free slot to add it (long rows keep Q1 in the tails and are
// skipped).  The column can be missing where q0 + E q1 cancels and was dropped as a numerical
// zero; that leaves a free slot.
__global__ void k_q1_fold_check(const int *__restrict__ q0_rowptr, const int *__restrict__ q1_rowptr,
                                const int *__restrict__ q1_col, const int *__restrict__ ell_col, long long ld, int W,
                                long long rows, int *__restrict__ bad) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const int n1 = q1_rowptr[r + 1] - q1_rowptr[r];
    if (n1 == 0 || ell_col[r] < 0) return;
    if (n1 > 1) {
        atomicOr(bad, 1);
        return;
    }
    const int c1 = q1_col[q1_rowptr[r]];
    const int len = q0_rowptr[r + 1] - q0_rowptr[r];
    for (int j = 0; j < len; ++j)
        if (ell_col[(long long)j * ld + r] == c1) return;
    if (len >= W) atomicOr(bad, 1);
}

// Move the entry at Q1's column to slot 0 of each short row (adding it with value 0 in the
// first free slot when it was dropped) and record Q1's value there.
template <typename VT>
__global__ void k_q1_fold(const int *__restrict__ q0_rowptr, const int *__restrict__ q1_rowptr,
                          const int *__restrict__ q1_col, const double *__restrict__ q1_val, long long ld,
                          long long rows, int *__restrict__ ell_col, VT *__restrict__ ell_val, VT *__restrict__ q1v) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ld) return;
    q1v[r] = VT(0);
    if (r >= rows || ell_col[r] < 0) return;
    const int n1 = q1_rowptr[r + 1] - q1_rowptr[r];
    if (n1 == 0) return;
    const int c1 = q1_col[q1_rowptr[r]];
    const int len = q0_rowptr[r + 1] - q0_rowptr[r];
    int found = -1;
    for (int j = 0; j < len && found < 0; ++j)
        if (ell_col[(long long)j * ld + r] == c1) found = j;
    if (found < 0) {   // the free slot `len` exists (checked by k_q1_fold_check)
        found = len;
        ell_col[(long long)len * ld + r] = c1;
        ell_val[(long long)len * ld + r] = VT(0);
    }
    const long long p = (long long)found * ld + r;
    const int tc = ell_col[r];
    const VT tv = ell_val[r];
    ell_col[r] = ell_col[p];
    ell_val[r] = ell_val[p];
    ell_col[p] = tc;
    ell_val[p] = tv;
    q1v[r] = (VT)q1_val[q1_rowptr[r]];
}

// Compact columns of one row: each slot's column as a delta from the row (s = 0) or from its
// S/J partner (s = 1), whichever fits in kC16Max; a long row or a row with a column that fits
// neither way gets kC16Esc in slot 0, and the latter is flagged for the escape list.  Rows past
// `rows` (padding up to ld) get zeros.
__global__ void k_c16(const int *__restrict__ ell_col, long long ld, int W, long long rows, long long pairs,
                      short *__restrict__ c16, long long *__restrict__ esc) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ld) return;
    if (r >= rows) {
        for (int j = 0; j < W; ++j) c16[(long long)j * ld + r] = 0;
        return;
    }
    const long long pr = c16_partner(r, pairs);
    bool ok = ell_col[r] >= 0;
    for (int j = 0; j < W && ok; ++j) {
        const long long p = (long long)j * ld + r;
        const long long col = ell_col[p];
        const long long d0 = col - r, d1 = col - pr;
        if (d0 >= -kC16Max && d0 <= kC16Max) c16[p] = (short)(2 * d0);
        else if (d1 >= -kC16Max && d1 <= kC16Max) c16[p] = (short)(2 * d1 + 1);
        else ok = false;
    }
    if (!ok) c16[r] = (short)kC16Esc;
    esc[r] = !ok && ell_col[r] >= 0;
}

}  // namespace

template <typename VT>
void drop_c16(Hyb<VT> &h) {
    h.ell_c16.release();
    h.c16_esc.release();
    h.n_esc = 0;
}

template <typename VT>
bool build_c16(Hyb<VT> &h, long long pairs, cudaStream_t s) {
    drop_c16(h);
    h.c16_pairs = pairs;
    if (h.width < 1 || h.rows < 1) return false;
    h.ell_c16.alloc((size_t)(h.ld * h.width));
    DBuf<long long> flag((size_t)h.rows), pos((size_t)h.rows + 1);
    k_c16<<<grid_for(h.ld, 256), 256, 0, s>>>(h.ell_col.p, h.ld, h.width, h.rows, pairs, h.ell_c16.p, flag.p);
    GK_LAUNCH_CHECK();
    const long long n = scan_ll(flag.p, pos.p, h.rows, true, true, s);
    if (n * 8 > h.rows - h.n_long) {
        drop_c16(h);
        return false;
    }
    h.n_esc = n;
    h.c16_esc.alloc((size_t)(n > 0 ? n : 1));
    if (n > 0) {
        k_long_list<<<grid_for(h.rows, 256), 256, 0, s>>>(flag.p, pos.p, h.rows, h.c16_esc.p);
        GK_LAUNCH_CHECK();
    }
    GK_CUDA(cudaStreamSynchronize(s));
    return true;
}

template void drop_c16<double>(Hyb<double> &);
template void drop_c16<float>(Hyb<float> &);
template bool build_c16<double>(Hyb<double> &, long long, cudaStream_t);
template bool build_c16<float>(Hyb<float> &, long long, cudaStream_t);

bool fold_q1(const CsrR &q0e, const CsrR &q1, long long rows, Hyb<double> &h0, Hyb<float> *h0f, DBuf<double> &q1v,
             DBuf<float> &q1vf, cudaStream_t s) {
    q1v.release();
    q1vf.release();
    if (q1.nnz == 0 || h0.width < 1) return false;
    DBuf<int> bad(1);
    GK_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
    k_q1_fold_check<<<grid_for(rows, 256), 256, 0, s>>>(q0e.rowptr.p, q1.rowptr.p, q1.col.p, h0.ell_col.p, h0.ld,
                                                          h0.width, rows, bad.p);
    GK_LAUNCH_CHECK();
    int hbad = 0;
    GK_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    if (hbad) return false;
    q1v.alloc((size_t)h0.ld);
    k_q1_fold<double><<<grid_for(h0.ld, 256), 256, 0, s>>>(q0e.rowptr.p, q1.rowptr.p, q1.col.p, q1.val.p, h0.ld, rows,
                                                            h0.ell_col.p, h0.ell_val.p, q1v.p);
    GK_LAUNCH_CHECK();
    if (h0f) {
        q1vf.alloc((size_t)h0f->ld);
        k_q1_fold<float><<<grid_for(h0f->ld, 256), 256, 0, s>>>(q0e.rowptr.p, q1.rowptr.p, q1.col.p, q1.val.p,
                                                                 h0f->ld, rows, h0f->ell_col.p, h0f->ell_val.p,
                                                                 q1vf.p);
        GK_LAUNCH_CHECK();
    }
    GK_CUDA(cudaStreamSynchronize(s));
    return true;
}

void build_hyb_pair(const CsrR &a0, const CsrR &a1, long long rows, Hyb<double> &h0, Hyb<double> &h1, Hyb<float> *h0f,
                    Hyb<float> *h1f, cudaStream_t s) {
    build_set({&a0, &a1}, {1.0, 1.0}, rows, {&h0, &h1}, {h0f, h1f}, s);
}

void build_hyb_single(const CsrR &a, long long rows, Hyb<double> &h, Hyb<float> *hf, double scale, cudaStream_t s) {
    build_set({&a}, {scale}, rows, {&h}, {hf}, s);
}

void build_hyb_multi(const std::vector<const CsrR *> &ms, const std::vector<double> &scales, long long rows,
                     const std::vector<Hyb<double> *> &out, const std::vector<Hyb<float> *> &outf, cudaStream_t s) {
    build_set(ms, scales, rows, out, outf, s);
}

}  // namespace gk
