// Records taken at every measurement (Appendix A): the state of the PT
// random walk ("history_betas": the ladder slot, i.e. the value of k, of
// every system copy) and the sums of A and B over blocks of maxit
// consecutive measurements, whose averages are what the paper writes out.
//
// Both live in device ring buffers indexed by the measurement number m, a
// device counter, so the record step can sit in a captured sweep graph:
//   hist  uint8 [hist_len][n_samples][n_rep][n_slots walkers]   slot of walker
//   blkA  int64 [blk_len][n_samples][n_rep][n_slots]             by slot
//   blkB  likewise
// Measurement m writes hist entry m % hist_len and adds into block entry
// (m / maxit) % blk_len (the block's first measurement overwrites it).
#include <cstring>
#include <vector>

#include "qisg_internal.cuh"

namespace qisg {
namespace {

// One block strides over the chain slots; it reads m once and, after its
// barrier, thread 0 advances the counter (no other block reads it).
__global__ void record_kernel(const int32_t *__restrict__ walker, const unsigned long long *__restrict__ U,
                              int by_slot, int64_t n_cs, int n_slots, int64_t N, unsigned long long *d_meas,
                              uint8_t *hist, int hist_len, long long *blkA, long long *blkB, int maxit,
                              int blk_len) {
  const unsigned long long m = *d_meas;
  const bool first = maxit > 0 && m % (unsigned long long)maxit == 0;
  const int64_t hrow = hist ? (int64_t)(m % (unsigned long long)hist_len) * n_cs : 0;
  const int64_t brow = blkA ? (int64_t)((m / (unsigned long long)maxit) % (unsigned long long)blk_len) * n_cs : 0;
  for (int64_t i = threadIdx.x; i < n_cs; i += blockDim.x) {
    const int64_t row = i / n_slots;
    const int s = (int)(i - row * n_slots);
    const int w = walker[i];
    if (hist) hist[hrow + row * n_slots + w] = (uint8_t)s;
    if (blkA) {
      const int64_t e = by_slot ? i : row * n_slots + w;
      const long long A = 2 * N - 2 * (long long)U[2 * e];
      const long long B = N - 2 * (long long)U[2 * e + 1];
      blkA[brow + i] = (first ? 0ll : blkA[brow + i]) + A;
      blkB[brow + i] = (first ? 0ll : blkB[brow + i]) + B;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *d_meas = m + 1ull;
}

}  // namespace

int record_measurement(qisg_handle *h) {
  const int64_t n_cs = h->n_samples * h->n_rep * h->n_slots;
  record_kernel<<<1, 1024, 0, h->stream>>>(h->d_walker, h->d_U, h->layout == QISG_LAYOUT_SAMPLES, n_cs,
                                           h->n_slots, h->N, h->d_meas, h->d_hist, h->hist_len, h->d_blkA,
                                           h->d_blkB, h->maxit, h->blk_len);
  h->launches++;
  return cuda_check(cudaGetLastError(), "record measurement");
}

}  // namespace qisg

using namespace qisg;

namespace {

// Copy ring entries first .. first+n-1 (entry e at row e % len) to host.
template <typename T>
int copy_ring(qisg_handle *h, const T *ring, int len, int64_t first, int64_t n, int64_t n_cs, T *out) {
  for (int64_t e = first; e < first + n; ++e) {
    const int rc = cuda_check(cudaMemcpyAsync(out + (e - first) * n_cs, ring + (e % len) * n_cs,
                                              (size_t)n_cs * sizeof(T), cudaMemcpyDeviceToHost, h->stream),
                              "copy record");
    if (rc) return rc;
  }
  return handle_sync(h);
}

// Complete blocks kept in the ring: [lo, hi).
void kept_blocks(const qisg_handle *h, int64_t *lo, int64_t *hi) {
  const int64_t cur = h->n_meas / h->maxit;                 // block in progress (or about to start)
  const int64_t partial = (h->n_meas % h->maxit) ? 1 : 0;   // it already overwrote its ring entry
  const int64_t base = (h->rec_base + h->maxit - 1) / h->maxit;   // first block recorded in full
  *hi = cur;
  *lo = cur - h->blk_len + partial;
  if (*lo < base) *lo = base;
}

}  // namespace

extern "C" {

int qisg_walk_history(qisg_handle *h, int64_t first, int64_t n, uint8_t *slot_of) {
  if (!h || (!slot_of && n > 0) || first < 0 || n < 0) return fail(QISG_EINVAL, "bad arguments");
  if (h->hist_len == 0) return fail(QISG_ESTATE, "no walk history kept (history_len = 0)");
  if (first + n > h->n_meas || first < h->n_meas - h->hist_len || first < h->rec_base)
    return fail(QISG_ESTATE, "measurements outside the kept history");
  if (n == 0) return QISG_OK;
  return copy_ring(h, h->d_hist, h->hist_len, first, n, h->n_samples * h->n_rep * h->n_slots, slot_of);
}

int qisg_block_sums(qisg_handle *h, int64_t first, int64_t n, int64_t *sumA, int64_t *sumB) {
  if (!h || ((!sumA || !sumB) && n > 0) || first < 0 || n < 0) return fail(QISG_EINVAL, "bad arguments");
  if (h->maxit == 0) return fail(QISG_ESTATE, "no block sums kept (maxit = 0)");
  int64_t lo = 0, hi = 0;
  kept_blocks(h, &lo, &hi);
  if (first < lo || first + n > hi) return fail(QISG_ESTATE, "blocks not complete or no longer kept");
  if (n == 0) return QISG_OK;
  const int64_t n_cs = h->n_samples * h->n_rep * h->n_slots;
  int rc = copy_ring(h, reinterpret_cast<const int64_t *>(h->d_blkA), h->blk_len, first, n, n_cs, sumA);
  if (!rc) rc = copy_ring(h, reinterpret_cast<const int64_t *>(h->d_blkB), h->blk_len, first, n, n_cs, sumB);
  return rc;
}

int qisg_block_means(qisg_handle *h, int64_t first, int64_t n, double *e_s, double *e_t) {
  if (!h || ((!e_s || !e_t) && n > 0) || n < 0) return fail(QISG_EINVAL, "bad arguments");
  const int64_t n_cs = h->n_samples * h->n_rep * h->n_slots;
  std::vector<int64_t> A((size_t)(n * n_cs)), B(A.size());
  int rc = qisg_block_sums(h, first, n, A.data(), B.data());
  if (rc) return rc;
  const double N = (double)h->N, den = (double)h->maxit * (double)h->n_samples * (double)h->n_rep;
  for (int64_t b = 0; b < n; ++b)
    for (int s = 0; s < h->n_slots; ++s) {
      double sa = 0.0, sb = 0.0;
      for (int64_t a = 0; a < h->n_samples; ++a)
        for (int r = 0; r < h->n_rep; ++r) {
          const size_t i = (size_t)(b * n_cs + (a * h->n_rep + r) * h->n_slots + s);
          sa += (double)A[i];
          sb += (double)B[i];
        }
      e_s[b * h->n_slots + s] = sa / (den * 2.0 * N);
      e_t[b * h->n_slots + s] = sb / (den * N);
    }
  return QISG_OK;
}

}  // extern "C"
