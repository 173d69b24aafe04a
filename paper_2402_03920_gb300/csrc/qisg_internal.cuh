// Internal declarations shared by the translation units of libqisg.
//
// Paper: "The QISG suite" (MCQSG code).  The model is Eq. (2)-(3) of Sec. 1
// with one (k, k_tau) pair per ladder slot; the update is Sec. 2.1's
// red/blue Metropolis with precomputed Metropolis factors followed by a
// parallel-tempering pass; random numbers are Philox4x32-10 (Sec. 2.1.1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/qisg.h"

namespace qisg {

// Philox counter domains: one per kind of draw.
enum : uint32_t { DOM_J = 1, DOM_INIT = 2, DOM_SWEEP = 3, DOM_PT = 4 };

constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

// Philox4x32-10 (Salmon et al., SC'11), the generator of Sec. 2.1.1.
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t lo0 = kPhiloxM0 * c.x, hi0 = __umulhi(kPhiloxM0, c.x);
    const uint32_t lo1 = kPhiloxM1 * c.z, hi1 = __umulhi(kPhiloxM1, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += kPhiloxW0;
    k.y += kPhiloxW1;
  }
  return c;
}

__device__ __forceinline__ uint32_t pick4(const uint4 &v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// b^e by right-to-left binary powering with round-to-nearest multiplies
// (no contraction), so host and device agree bit for bit.
__device__ __forceinline__ double pow_rn(double b, unsigned long long e) {
  double r = 1.0;
  while (e) {
    if (e & 1ull) r = __dmul_rn(r, b);
    b = __dmul_rn(b, b);
    e >>= 1;
  }
  return r;
}

// Sites of one colour: j in [0, N/2) -> site.  Each (y, tau) row holds L/2
// sites of each colour (L even).
struct SiteXYT {
  int x, y, tau;
};
__device__ __forceinline__ SiteXYT site_of_colour(int64_t j, int L, int colour) {
  const int half_L = L >> 1;
  const int64_t row = j / half_L;
  SiteXYT s;
  s.y = (int)(row % L);
  s.tau = (int)(row / L);
  s.x = 2 * (int)(j - row * half_L) + ((s.y + s.tau + colour) & 1);
  return s;
}

}  // namespace qisg

// ----------------------------------------------------------------------------
// The handle.
// ----------------------------------------------------------------------------
struct qisg_handle {
  // problem
  int L = 0, Lt = 0;
  int64_t N = 0;
  int n_slots = 0, n_rep = 0;
  int64_t n_samples = 0;
  uint64_t seed = 0;
  int pt_every = 1, measure_every = 0;
  int layout = QISG_LAYOUT_LANES, W = 64, per_sample_launch = 0;
  cudaStream_t stream = nullptr;
  size_t mem_budget = 0;
  uint64_t t = 0;          // sweeps done (host mirror of *d_t)
  int64_t n_meas = 0;      // measurements done (host mirror)
  int64_t launches = 0;
  int device = 0;
  int n_sm = 0;

  // host tables (FP64, built once)
  std::vector<double> k, kt;
  std::vector<uint32_t> T;      // [n_slots][5][3]
  std::vector<double> bases;    // [4][n_slots]: alpha+, alpha-, beta+, beta- of pair s

  // LANES geometry: rpw replicas per word, n_groups words per site per sample
  int rpw = 0, n_groups = 0;
  // SAMPLES geometry: n_b words of W samples, n_q groups of 4 replicas
  int64_t n_b = 0;
  int n_q = 0;
  int64_t n_a_pad = 0;          // samples including padding lanes

  // device memory
  void *spins = nullptr;
  size_t spins_bytes = 0;
  void *J = nullptr;
  size_t J_bytes = 0;
  uint32_t *d_T = nullptr;
  double *d_bases = nullptr;
  int32_t *d_walker = nullptr;      // [a_pad][r][s]
  unsigned long long *d_U = nullptr;  // LANES: [a][r][w][2] by walker; SAMPLES: [a_pad][r][s][2] by slot
  long long *d_sumA = nullptr, *d_sumB = nullptr, *d_sumq = nullptr, *d_sumq2 = nullptr;
  long long *d_q = nullptr;         // overlap scratch [a][s][pair]
  long long *d_out = nullptr;       // output staging [2][a][r][s]
  unsigned long long *d_t = nullptr;  // sweep counter
  void *d_acc = nullptr;            // SAMPLES: PT accept masks [b][r][s]
  int *d_err = nullptr;
  size_t device_bytes = 0;

  // launch timing (qisg_profile)
  bool prof = false;
  std::vector<cudaEvent_t> prof_ev[4];   // start/stop pairs per kernel kind
  int64_t prof_launched[4] = {0, 0, 0, 0};

  int n_pairs() const { return n_rep * (n_rep - 1) / 2; }
};

namespace qisg {

// error plumbing (qisg_api.cu)
int fail(int code, const std::string &msg);
int cuda_check(cudaError_t e, const char *what);

// LANES kernels (lanes.cu)
int lanes_init(qisg_handle *h);
int lanes_half_sweep(qisg_handle *h, int colour, int count_only);
int lanes_pt(qisg_handle *h, int explicit_pass);
int lanes_measure(qisg_handle *h, int force_to_q);
int lanes_energies_by_slot(qisg_handle *h);
int lanes_get_spins(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *S);
int lanes_set_spins(qisg_handle *h, const int8_t *S);
int lanes_get_couplings(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *J);
int lanes_set_couplings(qisg_handle *h, const int8_t *J);

// SAMPLES kernels (samples.cu)
int samples_init(qisg_handle *h);
int samples_half_sweep(qisg_handle *h, int colour, int count_only);
int samples_pt(qisg_handle *h, int explicit_pass);
int samples_measure(qisg_handle *h, int force_to_q);
int samples_energies_by_slot(qisg_handle *h);
int samples_get_spins(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *S);
int samples_set_spins(qisg_handle *h, const int8_t *S, const int32_t *walker_at);
int samples_get_couplings(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *J);
int samples_set_couplings(qisg_handle *h, const int8_t *J);

// common small kernels (qisg_api.cu)
int advance_counter(qisg_handle *h);

// Launch timing: call prof_begin(h, kind) before and prof_end(h, kind, tok)
// after a kernel launch on h->stream.
int prof_begin(qisg_handle *h, int kind);
void prof_end(qisg_handle *h, int kind, int tok);

}  // namespace qisg
