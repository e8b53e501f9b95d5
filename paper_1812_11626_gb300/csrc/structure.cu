// Enumeration of the nonzero structure constants f_mns and d_mns (Eq. 5) from their closed
// forms (Sec. IV step 2.2 states that the nonzero set is known analytically and has
// 5N^3-9N^2-2N+6 and 6N^3-N(21N+7)/2+1 ordered elements).  The nonzero set is the union of
//   triangles  {S/J of (pq), (qr), (pr)}, p < q < r  (f: odd number of J, d: even),
//   pair + D   {S_ab, J_ab, D^l} (f) and {S_ab, S_ab, D^l}, {J_ab, J_ab, D^l} (d),
//   diagonal   {D^l, D^l, D^n}, n >= l (d only);
// each set is walked and every candidate is evaluated with structure_value().
#include "internal.cuh"

namespace gk {

namespace {

struct Sink {
    int *m, *n, *s;
    double *val;
    long long cap;
    unsigned long long *pos;   // running output position (enumeration) or count
};

// all orderings of three generators; `same` marks duplicates so equal orderings are not repeated
__device__ inline void emit_orderings(int which, const Basis &B, const El &x, const El &y, const El &z, bool write,
                                      Sink &sk, unsigned long long &local) {
    const El e[3] = {x, y, z};
    const int perm[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {1, 0, 2}, {0, 2, 1}, {2, 1, 0}};
    long long idx[3] = {B.encode(x), B.encode(y), B.encode(z)};
    for (int p = 0; p < 6; ++p) {
        // skip orderings that repeat an earlier one (when two generators coincide)
        bool dup = false;
        for (int q = 0; q < p && !dup; ++q) {
            bool same = true;
            for (int k = 0; k < 3; ++k) same = same && idx[perm[p][k]] == idx[perm[q][k]];
            dup = same;
        }
        if (dup) continue;
        double v = structure_value(which, e[perm[p][0]], e[perm[p][1]], e[perm[p][2]]);
        if (v == 0.0) continue;
        if (write) {
            unsigned long long o = atomicAdd(sk.pos, 1ull);
            if ((long long)o < sk.cap) {
                sk.m[o] = (int)idx[perm[p][0]];
                sk.n[o] = (int)idx[perm[p][1]];
                sk.s[o] = (int)idx[perm[p][2]];
                sk.val[o] = v;
            }
        } else {
            ++local;
        }
    }
}

// one thread per pair (p, q): triangles with r > q
__global__ void k_triangles(int N, int which, bool write, Sink sk) {
    Basis B(N);
    long long pi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (pi >= B.P2) return;
    int p, q;
    B.unpair(pi, p, q);
    unsigned long long local = 0;
    for (int r = q + 1; r < N; ++r)
        for (int t = 0; t < 8; ++t) {
            El x{(t >> 2) & 1, p, q}, y{(t >> 1) & 1, q, r}, z{t & 1, p, r};
            if (write) emit_orderings(which, B, x, y, z, true, sk, local);
            else if (structure_value(which, x, y, z) != 0.0) local += 6;   // all six orderings share the support
        }
    if (!write) atomicAdd(sk.pos, local);
}

// one thread per pair (a, b): partners D^l
__global__ void k_pair_d(int N, int which, bool write, Sink sk) {
    Basis B(N);
    long long pi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (pi >= B.P2) return;
    int a, b;
    B.unpair(pi, a, b);
    unsigned long long local = 0;
    for (int l = 1; l < N; ++l) {
        El Dl{2, l, -1};
        if (which == 0) {
            El S{0, a, b}, J{1, a, b};
            if (write) emit_orderings(0, B, S, J, Dl, true, sk, local);
            else if (structure_value(0, S, J, Dl) != 0.0) local += 6;
        } else {
            for (int t = 0; t < 2; ++t) {
                El P{t, a, b};
                if (write) emit_orderings(1, B, P, P, Dl, true, sk, local);
                else if (structure_value(1, P, P, Dl) != 0.0) local += 3;
            }
        }
    }
    if (!write) atomicAdd(sk.pos, local);
}

// one thread per l: {D^l, D^l, D^n}, n >= l (d only)
__global__ void k_ddd(int N, bool write, Sink sk) {
    Basis B(N);
    int l = blockIdx.x * blockDim.x + threadIdx.x + 1;
    if (l >= N) return;
    unsigned long long local = 0;
    El L{2, l, -1};
    for (int n = l; n < N; ++n) {
        El M{2, n, -1};
        if (write) emit_orderings(1, B, L, L, M, true, sk, local);
        else if (structure_value(1, L, L, M) != 0.0) local += (n == l ? 1 : 3);
    }
    if (!write) atomicAdd(sk.pos, local);
}

long long run(int N, int which, bool write, Sink sk, cudaStream_t s) {
    Basis B(N);
    DBuf<unsigned long long> pos(1);
    GK_CUDA(cudaMemsetAsync(pos.p, 0, sizeof(unsigned long long), s));
    sk.pos = pos.p;
    if (N >= 3) {
        k_triangles<<<grid_for(B.P2, 128), 128, 0, s>>>(N, which, write, sk);
        GK_LAUNCH_CHECK();
    }
    k_pair_d<<<grid_for(B.P2, 128), 128, 0, s>>>(N, which, write, sk);
    GK_LAUNCH_CHECK();
    if (which == 1) {
        k_ddd<<<grid_for(N, 128), 128, 0, s>>>(N, write, sk);
        GK_LAUNCH_CHECK();
    }
    unsigned long long h = 0;
    GK_CUDA(cudaMemcpyAsync(&h, pos.p, sizeof h, cudaMemcpyDeviceToHost, s));
    GK_CUDA(cudaStreamSynchronize(s));
    return (long long)h;
}

}  // namespace

long long structure_count(int N, int which, cudaStream_t s) {
    Sink sk{nullptr, nullptr, nullptr, nullptr, 0, nullptr};
    return run(N, which, false, sk, s);
}

long long structure_enumerate(int N, int which, long long cap, int *m, int *n, int *sidx, double *val,
                              cudaStream_t s) {
    Sink sk{m, n, sidx, val, cap, nullptr};
    return run(N, which, true, sk, s);
}

}  // namespace gk
