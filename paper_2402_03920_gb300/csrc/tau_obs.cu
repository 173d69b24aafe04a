// Imaginary-time observables of the configurations now at each ladder slot
// (Appendix E.1, the quantities of the overlap_tau and corr_euclidea
// programs, computed online on the resident configurations instead of from
// files).  For one configuration S and a lag tau (tau_1 + tau taken modulo
// L_tau):
//   q~_x(tau_1, tau) = S_{x, tau_1} S_{x, tau_1 + tau},
//   Q~(tau_1, tau)   = sum_x q~_x(tau_1, tau),
// and over tau_1 = 0 .. L_tau-1 the sums
//   S1(tau) = sum Q~                  (L^2 L_tau times the site average of C_x(tau))
//   S2(tau) = sum Q~^2, S4(tau) = sum Q~^4    (L_tau Q_2(tau), L_tau Q_4(tau))
//   SF(tau) = sum ( |sum_x e^{i 2 pi x_1 / L} q~_x|^2 + |sum_x e^{i 2 pi x_2 / L} q~_x|^2 )
//                                     (2 L_tau F(tau))
// per (sample, replica, slot); averages over measurements and replicas are
// the caller's.
//
// A block takes one configuration: its spins (staged as int8 by walker)
// become two bitmaps per tau-plane in shared memory, one 32-bit word per
// row (fixed x_2, bit x_1) and one per column (fixed x_1, bit x_2), so a row
// or column sum of q~ is L - 2 popc(word(tau_1) ^ word(tau_1 + tau)).  A
// thread owns lags tau and walks tau_1 in order; the Fourier sums take the
// rows and columns in order x = 0 .. L-1 with the host's cos / sin table, in
// FP64 without contraction, so the result does not depend on the schedule.
#include <algorithm>
#include <cmath>
#include <vector>

#include "qisg_internal.cuh"

namespace qisg {
namespace {

constexpr int kTauBlock = 256;
constexpr size_t kTauSmemMax = 227 * 1024;

__global__ void __launch_bounds__(kTauBlock) tau_obs_kernel(const int8_t *__restrict__ S,
                                                            const int32_t *__restrict__ walker, int64_t a0,
                                                            int n_rep, int n_slots, int L, int Lt,
                                                            const double *__restrict__ cs,
                                                            const double *__restrict__ sn, long long *S1,
                                                            long long *S2, long long *S4, double *SF) {
  extern __shared__ uint32_t plane_words[];
  uint32_t *rows = plane_words;                       // [Lt][L]: row x2, bit x1
  uint32_t *cols = plane_words + (size_t)Lt * L;      // [Lt][L]: column x1, bit x2
  const int64_t c = blockIdx.x;                       // configuration (ai, r, s) of this chunk
  const int s = (int)(c % n_slots);
  const int64_t ar = c / n_slots;                     // ai * n_rep + r
  const int64_t ai = ar / n_rep;
  const int r = (int)(ar - ai * n_rep);
  const int w = walker[((a0 + ai) * n_rep + r) * n_slots + s];
  const int64_t N = (int64_t)L * L * Lt;
  const int8_t *src = S + (ar * n_slots + w) * N;
  for (int i = threadIdx.x; i < Lt * L; i += blockDim.x) {
    const int tau = i / L, k = i - tau * L;
    uint32_t row = 0, col = 0;
    for (int j = 0; j < L; ++j) {
      row |= (uint32_t)(src[(int64_t)j + (int64_t)L * k + (int64_t)L * L * tau] < 0) << j;   // x1 = j, x2 = k
      col |= (uint32_t)(src[(int64_t)k + (int64_t)L * j + (int64_t)L * L * tau] < 0) << j;   // x1 = k, x2 = j
    }
    rows[i] = row;
    cols[i] = col;
  }
  __syncthreads();
  for (int tau = threadIdx.x; tau < Lt; tau += blockDim.x) {
    long long s1 = 0, s2 = 0, s4 = 0;
    double sf = 0.0;
    for (int t1 = 0; t1 < Lt; ++t1) {
      const int t2 = t1 + tau < Lt ? t1 + tau : t1 + tau - Lt;
      const uint32_t *r1 = rows + (size_t)t1 * L, *r2 = rows + (size_t)t2 * L;
      const uint32_t *c1 = cols + (size_t)t1 * L, *c2 = cols + (size_t)t2 * L;
      long long q = 0;
      double re1 = 0.0, im1 = 0.0, re2 = 0.0, im2 = 0.0;
      for (int x = 0; x < L; ++x) {
        const int R = L - 2 * __popc(r1[x] ^ r2[x]);   // sum over x1 of q~ at x2 = x
        const int C = L - 2 * __popc(c1[x] ^ c2[x]);   // sum over x2 of q~ at x1 = x
        q += R;
        re1 = __dadd_rn(re1, __dmul_rn(cs[x], (double)C));
        im1 = __dadd_rn(im1, __dmul_rn(sn[x], (double)C));
        re2 = __dadd_rn(re2, __dmul_rn(cs[x], (double)R));
        im2 = __dadd_rn(im2, __dmul_rn(sn[x], (double)R));
      }
      const long long q2 = q * q;
      s1 += q;
      s2 += q2;
      s4 += q2 * q2;
      const double f1 = __dadd_rn(__dmul_rn(re1, re1), __dmul_rn(im1, im1));
      const double f2 = __dadd_rn(__dmul_rn(re2, re2), __dmul_rn(im2, im2));
      sf = __dadd_rn(sf, __dadd_rn(f1, f2));
    }
    const int64_t o = c * Lt + tau;
    S1[o] = s1;
    S2[o] = s2;
    S4[o] = s4;
    SF[o] = sf;
  }
}

}  // namespace
}  // namespace qisg

using namespace qisg;

extern "C" int qisg_tau_observables(qisg_handle *h, int64_t a_lo, int64_t n_a, int64_t *S1, int64_t *S2,
                                    int64_t *S4, double *SF) {
  if (!h || ((!S1 || !S2 || !S4 || !SF) && n_a > 0)) return fail(QISG_EINVAL, "NULL argument");
  if (a_lo < 0 || n_a < 0 || a_lo + n_a > h->n_samples) return fail(QISG_EINVAL, "sample range");
  if (h->L > 32) return fail(QISG_EINVAL, "tau observables take L <= 32");
  const size_t smem = (size_t)2 * h->Lt * h->L * 4;
  if (smem > kTauSmemMax) return fail(QISG_EINVAL, "tau observables: 2 L L_tau words exceed shared memory");
  if (n_a == 0) return QISG_OK;
  int rc = handle_sync(h);
  if (rc) return rc;
  // cos / sin of 2 pi x / L, x = 0 .. L-1 (host libm, FP64)
  std::vector<double> tab((size_t)2 * h->L);
  for (int x = 0; x < h->L; ++x) {
    tab[(size_t)x] = std::cos(2.0 * M_PI * x / h->L);
    tab[(size_t)h->L + x] = std::sin(2.0 * M_PI * x / h->L);
  }
  const int64_t per_a = (int64_t)h->n_rep * h->n_slots * h->N;
  const int64_t cfg_a = (int64_t)h->n_rep * h->n_slots;
  const int64_t chunk = std::min(n_a, std::max<int64_t>(1, ((int64_t)256 << 20) / per_a));
  int8_t *stage = nullptr;
  double *d_tab = nullptr;
  long long *d_out = nullptr;   // S1, S2, S4 of a chunk, then SF
  const size_t n_out = (size_t)(chunk * cfg_a * h->Lt);
  rc = cuda_check(cudaMalloc(&stage, (size_t)(chunk * per_a)), "cudaMalloc");
  if (!rc) rc = cuda_check(cudaMalloc(&d_tab, tab.size() * 8), "cudaMalloc");
  if (!rc) rc = cuda_check(cudaMalloc(&d_out, n_out * 4 * 8), "cudaMalloc");
  if (!rc) rc = cuda_check(cudaMemcpyAsync(d_tab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, h->stream),
                           "copy table");
  if (!rc && smem > 48 * 1024)
    rc = cuda_check(cudaFuncSetAttribute(tau_obs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                    "shared memory");
  for (int64_t a0 = 0; a0 < n_a && !rc; a0 += chunk) {
    const int64_t na = std::min(chunk, n_a - a0), nc = na * cfg_a, no = nc * h->Lt;
    rc = h->layout == QISG_LAYOUT_LANES   ? lanes_stage_spins(h, a_lo + a0, na, stage)
         : h->layout == QISG_LAYOUT_SITES ? sites_stage_spins(h, a_lo + a0, na, stage)
                                          : samples_stage_spins(h, a_lo + a0, na, stage);
    if (rc) break;
    tau_obs_kernel<<<(unsigned)nc, kTauBlock, smem, h->stream>>>(
        stage, h->d_walker, a_lo + a0, h->n_rep, h->n_slots, h->L, h->Lt, d_tab, d_tab + h->L, d_out,
        d_out + n_out, d_out + 2 * n_out, reinterpret_cast<double *>(d_out + 3 * n_out));
    h->launches++;
    rc = cuda_check(cudaGetLastError(), "tau observables");
    const int64_t o = a0 * cfg_a * h->Lt;
    if (!rc) rc = cuda_check(cudaMemcpyAsync(S1 + o, d_out, (size_t)no * 8, cudaMemcpyDeviceToHost, h->stream), "copy");
    if (!rc)
      rc = cuda_check(cudaMemcpyAsync(S2 + o, d_out + n_out, (size_t)no * 8, cudaMemcpyDeviceToHost, h->stream), "copy");
    if (!rc)
      rc = cuda_check(cudaMemcpyAsync(S4 + o, d_out + 2 * n_out, (size_t)no * 8, cudaMemcpyDeviceToHost, h->stream),
                      "copy");
    if (!rc)
      rc = cuda_check(cudaMemcpyAsync(SF + o, d_out + 3 * n_out, (size_t)no * 8, cudaMemcpyDeviceToHost, h->stream),
                      "copy");
    if (!rc) rc = handle_sync(h);
  }
  if (stage) cudaFree(stage);
  if (d_tab) cudaFree(d_tab);
  if (d_out) cudaFree(d_out);
  return rc;
}
