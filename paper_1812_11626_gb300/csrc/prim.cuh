// Device primitives used by the assembly: exclusive scan, stable LSD radix sort of
// 64-bit keys, and (key, value) reduction into CSR.
#pragma once

#include "common.cuh"

namespace gk {

// out[i] = sum_{j<i} in[j] for i < n, and out[n] = total when out has n + 1 slots
// (`with_total`).  Returns the total (synchronises the stream to read it) when `want_total`.
long long scan_ll(const long long *in, long long *out, long long n, bool with_total, bool want_total,
                  cudaStream_t s);
long long scan_u32_to_ll(const unsigned *in, long long *out, long long n, bool want_total, cudaStream_t s);

// Stable sort of (key, idx) pairs by the low `key_bits` bits of key, in place (the buffers
// are swapped internally; the result is always left in keys/idx).
void radix_sort(DBuf<uint64_t> &keys, DBuf<uint32_t> &idx, long long n, int key_bits, cudaStream_t s);

// COO (key = row * ncols + col, value) -> CSR, summing duplicates in the stable sorted order
// and dropping entries whose |sum| <= drop (drop < 0: keep everything, including zeros).
void coo_to_csr_real(DBuf<uint64_t> &keys, DBuf<double> &vals, long long n, long long nrows, long long ncols,
                     double drop, CsrR &out, cudaStream_t s);
void coo_to_csr_cplx(DBuf<uint64_t> &keys, DBuf<double2> &vals, long long n, long long nrows, long long ncols,
                     double drop, CsrC &out, cudaStream_t s);

// max |val| over n entries (synchronises)
double max_abs(const double *val, long long n, cudaStream_t s);

int bits_for(unsigned long long x);

}  // namespace gk
