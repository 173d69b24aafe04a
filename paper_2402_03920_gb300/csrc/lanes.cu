// LANES packing: one word (32 or 64 bits) holds the replica x walker systems
// of one disorder sample; lane = (r - g*rpw) * n_slots + w for the word group
// g = r / rpw.  Every lane is a different system at a different ladder slot,
// so each lane draws its own number and looks up its own Metropolis
// threshold.  PT exchanges slot labels only (Sec. 2.1: "there is no need to
// swap the spin systems, since it is sufficient to swap the k values").
//
// Device arrays (a = sample, N = L*L*L_tau):
//   spins  Word [a][g][site]           bit = 1 <=> spin -1
//   J      uint8 [a][x + L*y]          bit0: J(+x) = -1, bit1: J(+y) = -1
//   U      u64 [a][r][w][2]            unsatisfied spatial / tau bonds of walker w
#include <algorithm>
#include <cstring>

#include "lanes_core.cuh"
#include "qisg_internal.cuh"

namespace qisg {
namespace {

constexpr int kBlock = 256;
static_assert(kBlock <= kLanesMaxThreads, "the LANES class-code buffer holds kLanesMaxThreads threads");

template <typename Word>
struct LanesArgs {
  Word *spins;
  const uint8_t *J;
  const int32_t *walker;
  const uint32_t *T;
  unsigned long long *U;
  const unsigned long long *d_t;
  uint2 key;
  int64_t N, half_N;
  FastDiv half_plane_div;
  int L, Lt, plane, half_plane, n_slots, n_rep, rpw, n_groups, sites_per_block;
  int tau_ap;
};

template <typename Word>
__device__ __forceinline__ Word all_ones_if(bool b) {
  return b ? ~Word(0) : Word(0);
}

template <typename Word>
__device__ __forceinline__ uint32_t bit_at(Word w, int lane) {
  return (uint32_t)(w >> lane) & 1u;
}

// One half sweep (colour 0 = red, 1 = blue) of samples a0 + blockIdx.y:
// block x is the tile of colour sites [x * tile_sites, (x+1) * tile_sites),
// one thread per site (lanes_core.cuh).  Block 0 of the red pass clears the
// sample's bond counters, which the blue pass fills.
template <typename Word, bool BLUE, int NREP, int NGC>
__global__ void __launch_bounds__(kBlock) lanes_half_sweep_kernel(LanesArgs<Word> p, int colour,
                                                                  int count_only, int64_t a0, int tile_sites) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t a = a0 + blockIdx.y;
  LanesSample<Word> S;
  S.spins = p.spins + a * p.n_groups * p.N;
  S.T = p.T;
  S.walker = p.walker + a * p.n_rep * p.n_slots;
  S.U = p.U + a * p.n_rep * p.n_slots * 2;
  S.J = p.J + a * p.plane;
  S.key = p.key;
  S.ctr_w = (DOM_SWEEP << 28) | (uint32_t)(a >> 6);
  S.t = (uint32_t)*p.d_t;
  S.hpd = p.half_plane_div;
  S.L = p.L;
  S.Lt = p.Lt;
  S.plane = p.plane;
  S.half_plane = p.half_plane;
  S.N = (int)p.N;
  S.n_slots = p.n_slots;
  S.n_rep = p.n_rep;
  S.rpw = p.rpw;
  S.n_groups = p.n_groups;
  S.tau_ap = p.tau_ap;
  const int64_t j0 = (int64_t)blockIdx.x * tile_sites;
  const int n = (int)(p.half_N - j0 < tile_sites ? p.half_N - j0 : tile_sites);
  lanes_tile<Word, false, BLUE, NREP, NGC>(S, colour, (int)j0, n, count_only, colour == 0 && blockIdx.x == 0, smem_raw);
}

// Overlaps of the configurations at slot s (Appendix E.1): count the sites
// where the replicas r1 < r2 differ; q = N - 2 * count.  Grid (chunks,
// n_slots, n_a); accumulates counts into qcnt[a][s][pair].
template <typename Word>
__global__ void __launch_bounds__(kBlock) lanes_overlap_kernel(const Word *spins, const int32_t *walker,
                                                               long long *qcnt, int64_t a0, int64_t N,
                                                               int n_rep, int n_slots, int rpw,
                                                               int n_groups) {
  extern __shared__ long long q_s[];  // [n_pairs]
  const int n_pairs = n_rep * (n_rep - 1) / 2;
  const int s = blockIdx.y;
  const int64_t a = a0 + blockIdx.z;
  for (int i = threadIdx.x; i < n_pairs; i += blockDim.x) q_s[i] = 0;
  __syncthreads();
  const int32_t *wa = walker + a * n_rep * n_slots;
  const Word *base = spins + a * n_groups * N;
  for (int64_t site = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; site < N;
       site += (int64_t)gridDim.x * blockDim.x) {
    int p = 0;
    for (int r1 = 0; r1 < n_rep; ++r1) {
      const int g1 = r1 / rpw;
      const int l1 = (r1 - g1 * rpw) * n_slots + wa[r1 * n_slots + s];
      const uint32_t b1 = (uint32_t)(base[g1 * N + site] >> l1) & 1u;
      for (int r2 = r1 + 1; r2 < n_rep; ++r2, ++p) {
        const int g2 = r2 / rpw;
        const int l2 = (r2 - g2 * rpw) * n_slots + wa[r2 * n_slots + s];
        const uint32_t b2 = (uint32_t)(base[g2 * N + site] >> l2) & 1u;
        const uint32_t d = b1 ^ b2;
        // warp reduce then one shared atomic per warp
        const unsigned act = __activemask();
        const uint32_t cnt = __popc(__ballot_sync(act, d));
        if ((int)(threadIdx.x & 31) == __ffs(act) - 1 && cnt)
          atomicAdd(reinterpret_cast<unsigned long long *>(&q_s[p]), (unsigned long long)cnt);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n_pairs; i += blockDim.x)
    if (q_s[i])
      atomicAdd(reinterpret_cast<unsigned long long *>(&qcnt[(a * n_slots + s) * n_pairs + i]),
                (unsigned long long)q_s[i]);
}

// Measurement finalisation: sums by slot of A, B, q, q^2; turns the
// difference counts into q and clears them.  One thread per (a, s).
__global__ void lanes_finalize_kernel(const int32_t *walker, const unsigned long long *U,
                                      long long *qcnt, long long *sumA, long long *sumB,
                                      long long *sumq, long long *sumq2, int64_t n_a, int n_rep,
                                      int n_slots, int64_t N, int to_q_only) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n_a * n_slots) return;
  const int64_t a = c / n_slots;
  const int s = (int)(c % n_slots);
  const int n_pairs = n_rep * (n_rep - 1) / 2;
  if (to_q_only) {
    for (int p = 0; p < n_pairs; ++p) {
      long long *qc = &qcnt[(a * n_slots + s) * n_pairs + p];
      *qc = N - 2 * *qc;
    }
    return;
  }
  for (int r = 0; r < n_rep; ++r) {
    const int w = walker[(a * n_rep + r) * n_slots + s];
    const unsigned long long *u = U + ((a * n_rep + r) * n_slots + w) * 2;
    sumA[(a * n_rep + r) * n_slots + s] += 2 * N - 2 * (long long)u[0];
    sumB[(a * n_rep + r) * n_slots + s] += N - 2 * (long long)u[1];
  }
  for (int p = 0; p < n_pairs; ++p) {
    long long *qc = &qcnt[(a * n_slots + s) * n_pairs + p];
    const long long q = N - 2 * *qc;
    sumq[(a * n_slots + s) * n_pairs + p] += q;
    sumq2[(a * n_slots + s) * n_pairs + p] += q * q;
    *qc = 0;
  }
}

__global__ void lanes_by_slot_kernel(const int32_t *walker, const unsigned long long *U,
                                     long long *out, int64_t n_a, int n_rep, int n_slots,
                                     int64_t N) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t total = n_a * n_rep * n_slots;
  if (c >= total) return;
  const int64_t ar = c / n_slots;
  const int w = walker[c];
  const unsigned long long *u = U + (ar * n_slots + w) * 2;
  out[c] = 2 * N - 2 * (long long)u[0];
  out[total + c] = N - 2 * (long long)u[1];
}

// Start state: J and spins from Philox domains DOM_J and DOM_INIT.
__global__ void lanes_init_J_kernel(uint8_t *J, int64_t n_a, int L, uint2 key) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t plane = (int64_t)L * L;
  if (c >= n_a * plane) return;
  const int64_t a = c / plane;
  const uint32_t i2 = (uint32_t)(c % plane);
  uint8_t v = 0;
  for (uint32_t dir = 0; dir < 2; ++dir) {
    const uint4 x = philox(make_uint4(i2, dir, (uint32_t)a, DOM_J << 28), key);
    if (!(x.x & 1u)) v |= (uint8_t)(1u << dir);  // J = -1 <=> bit set
  }
  J[c] = v;
}

template <typename Word>
__global__ void lanes_init_spins_kernel(Word *spins, int64_t n_a, int64_t N, int n_rep, int n_slots,
                                        int rpw, int n_groups, uint2 key) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n_a * n_groups * N) return;
  const int64_t site = c % N;
  const int64_t ag = c / N;
  const int g = (int)(ag % n_groups);
  const int64_t a = ag / n_groups;
  Word v = 0;
  const int r_lo = g * rpw, r_hi = min(n_rep, r_lo + rpw);
  for (int r = r_lo; r < r_hi; ++r)
    for (int w = 0; w < n_slots; ++w) {
      const uint4 x = philox(make_uint4((uint32_t)site, (uint32_t)w, (uint32_t)a,
                                        (DOM_INIT << 28) | (uint32_t)r),
                             key);
      if (!(x.x & 1u)) v |= Word(1) << ((r - r_lo) * n_slots + w);  // spin -1
    }
  spins[c] = v;
}

// int8 +-1 spins [ai][r][w][site] of samples a_lo .. a_lo+n_a-1 from the
// lattice: a thread per spin.
template <typename Word>
__global__ void lanes_extract_kernel(const Word *spins, int8_t *out, int64_t a_lo, int64_t n_a, int64_t N, int n_rep,
                                     int n_slots, int rpw, int n_groups) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n_a * n_rep * n_slots * N) return;
  const int64_t site = c % N, rw = c / N;
  const int w = (int)(rw % n_slots);
  const int64_t ar = rw / n_slots;
  const int r = (int)(ar % n_rep);
  const int64_t ai = ar / n_rep;
  const int g = r / rpw, lane = (r - g * rpw) * n_slots + w;
  const Word v = spins[((a_lo + ai) * n_groups + g) * N + site];
  out[c] = ((v >> lane) & 1u) ? -1 : 1;
}

// The lattice words of samples a0 .. a0+n_a-1 from int8 +-1 spins staged as
// [ai][r][w][site]: a thread per (sample, word group, site) word.
template <typename Word>
__global__ void lanes_pack_kernel(Word *spins, const int8_t *stage, int64_t a0, int64_t n_a, int64_t N, int n_rep,
                                  int n_slots, int rpw, int n_groups) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n_a * n_groups * N) return;
  const int64_t site = c % N, ag = c / N;
  const int g = (int)(ag % n_groups);
  const int64_t ai = ag / n_groups;
  const int r_lo = g * rpw, r_hi = min(n_rep, r_lo + rpw);
  Word v = 0;
  for (int r = r_lo; r < r_hi; ++r)
    for (int w = 0; w < n_slots; ++w)
      if (stage[((ai * n_rep + r) * n_slots + w) * N + site] == -1) v |= Word(1) << ((r - r_lo) * n_slots + w);
  spins[((a0 + ai) * n_groups + g) * N + site] = v;
}

template <typename Word>
LanesArgs<Word> make_args(qisg_handle *h) {
  LanesArgs<Word> p;
  p.spins = reinterpret_cast<Word *>(h->spins);
  p.J = reinterpret_cast<const uint8_t *>(h->J);
  p.walker = h->d_walker;
  p.T = h->d_T;
  p.U = h->d_U;
  p.d_t = h->d_t;
  p.key = make_uint2((uint32_t)h->seed, (uint32_t)(h->seed >> 32));
  p.N = h->N;
  p.half_N = h->N / 2;
  p.L = h->L;
  p.Lt = h->Lt;
  p.plane = h->L * h->L;
  p.half_plane = p.plane / 2;
  p.half_plane_div = FastDiv((uint32_t)p.half_plane);
  p.n_slots = h->n_slots;
  p.n_rep = h->n_rep;
  p.rpw = h->rpw;
  p.n_groups = h->n_groups;
  p.sites_per_block = kBlock / h->n_slots;
  p.tau_ap = h->tau_ap;
  return p;
}

template <typename Word>
int half_sweep_t(qisg_handle *h, int colour, int count_only) {
  LanesArgs<Word> p = make_args<Word>(h);
  const size_t smem = lanes_tile_smem(p.plane, h->n_slots, h->n_rep);
  // tiles of rows x 256 sites (rows <= 16, the counters' limit), as long as
  // the grid keeps about four blocks per SM
  const int64_t n_launch_samples = h->per_sample_launch ? 1 : h->n_samples;
  int rows = 16;
  while (rows > 1 && ((p.half_N + 256LL * rows - 1) / (256LL * rows)) * n_launch_samples < 4LL * h->n_sm) rows >>= 1;
  const int tile_sites = 256 * rows;
  const int64_t blocks = (p.half_N + tile_sites - 1) / tile_sites;
  if (blocks > 0x7FFFFFFF) return fail(QISG_EINVAL, "lattice too large for one launch");
  if (smem > 227 * 1024) return fail(QISG_EINVAL, "LANES plane tables exceed shared memory");
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(lanes_half_sweep_kernel<Word, false, 0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(lanes_half_sweep_kernel<Word, true, 0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(lanes_half_sweep_kernel<Word, false, 4, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(lanes_half_sweep_kernel<Word, true, 4, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(lanes_half_sweep_kernel<Word, false, 4, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(lanes_half_sweep_kernel<Word, true, 4, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr_set = true;
  }
  for (int64_t a0 = 0; a0 < h->n_samples; a0 += (h->per_sample_launch ? 1 : 65535)) {
    const int64_t na = h->per_sample_launch ? 1 : std::min<int64_t>(65535, h->n_samples - a0);
    const int tok = prof_begin(h, sweep_kind(colour));
    const dim3 grid((unsigned)blocks, (unsigned)na);
    // compile-time replica count (loops unrolled) and word-group count (fewer
    // registers) for the common cases
    if (h->n_rep == 4 && h->n_groups == 1) {
      if (colour == 1)
        lanes_half_sweep_kernel<Word, true, 4, 1><<<grid, kBlock, smem, h->stream>>>(p, 1, count_only, a0, tile_sites);
      else
        lanes_half_sweep_kernel<Word, false, 4, 1><<<grid, kBlock, smem, h->stream>>>(p, 0, count_only, a0, tile_sites);
    } else if (h->n_rep == 4) {
      if (colour == 1)
        lanes_half_sweep_kernel<Word, true, 4, 0><<<grid, kBlock, smem, h->stream>>>(p, 1, count_only, a0, tile_sites);
      else
        lanes_half_sweep_kernel<Word, false, 4, 0><<<grid, kBlock, smem, h->stream>>>(p, 0, count_only, a0, tile_sites);
    } else {
      if (colour == 1)
        lanes_half_sweep_kernel<Word, true, 0, 0><<<grid, kBlock, smem, h->stream>>>(p, 1, count_only, a0, tile_sites);
      else
        lanes_half_sweep_kernel<Word, false, 0, 0><<<grid, kBlock, smem, h->stream>>>(p, 0, count_only, a0, tile_sites);
    }
    prof_end(h, sweep_kind(colour), tok);
    h->launches++;
  }
  return cuda_check(cudaGetLastError(), "lanes half sweep");
}

template <typename Word>
int measure_t(qisg_handle *h, int force_to_q) {
  const int n_pairs = h->n_pairs();
  if (n_pairs > 0) {
    const int64_t chunks = std::min<int64_t>((h->N + kBlock - 1) / kBlock, 64);
    const size_t smem = (size_t)n_pairs * 8;
    for (int64_t a0 = 0; a0 < h->n_samples; a0 += 65535) {
      const int64_t na = std::min<int64_t>(65535, h->n_samples - a0);
      const int tok = prof_begin(h, QISG_KERNEL_MEASURE);
      lanes_overlap_kernel<Word><<<dim3((unsigned)chunks, (unsigned)h->n_slots, (unsigned)na), kBlock,
                                   smem, h->stream>>>(reinterpret_cast<const Word *>(h->spins),
                                                      h->d_walker, h->d_q, a0, h->N, h->n_rep,
                                                      h->n_slots, h->rpw, h->n_groups);
      prof_end(h, QISG_KERNEL_MEASURE, tok);
      h->launches++;
    }
  }
  const int64_t n = h->n_samples * h->n_slots;
  lanes_finalize_kernel<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(
      h->d_walker, h->d_U, h->d_q, h->d_sumA, h->d_sumB, h->d_sumq, h->d_sumq2, h->n_samples,
      h->n_rep, h->n_slots, h->N, force_to_q);
  h->launches++;
  return cuda_check(cudaGetLastError(), "lanes measure");
}


}  // namespace

int lanes_init_couplings(qisg_handle *h) {
  const uint2 key = make_uint2((uint32_t)h->seed, (uint32_t)(h->seed >> 32));
  const int64_t nJ = h->n_samples * h->L * h->L;
  lanes_init_J_kernel<<<(unsigned)((nJ + 255) / 256), 256, 0, h->stream>>>(
      reinterpret_cast<uint8_t *>(h->J), h->n_samples, h->L, key);
  h->launches++;
  return cuda_check(cudaGetLastError(), "init couplings");
}

int lanes_finalize(qisg_handle *h, int force_to_q) {
  const int64_t n = h->n_samples * h->n_slots;
  lanes_finalize_kernel<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(
      h->d_walker, h->d_U, h->d_q, h->d_sumA, h->d_sumB, h->d_sumq, h->d_sumq2, h->n_samples,
      h->n_rep, h->n_slots, h->N, force_to_q);
  h->launches++;
  return cuda_check(cudaGetLastError(), "finalize measurement");
}

int lanes_init(qisg_handle *h) {
  const uint2 key = make_uint2((uint32_t)h->seed, (uint32_t)(h->seed >> 32));
  int rc = lanes_init_couplings(h);
  if (rc) return rc;
  const int64_t nS = h->n_samples * h->n_groups * h->N;
  if ((nS + 255) / 256 > 0x7FFFFFFF) return fail(QISG_EINVAL, "lattice too large");
  if (h->W == 64)
    lanes_init_spins_kernel<unsigned long long><<<(unsigned)((nS + 255) / 256), 256, 0, h->stream>>>(
        reinterpret_cast<unsigned long long *>(h->spins), h->n_samples, h->N, h->n_rep, h->n_slots,
        h->rpw, h->n_groups, key);
  else
    lanes_init_spins_kernel<unsigned int><<<(unsigned)((nS + 255) / 256), 256, 0, h->stream>>>(
        reinterpret_cast<unsigned int *>(h->spins), h->n_samples, h->N, h->n_rep, h->n_slots,
        h->rpw, h->n_groups, key);
  h->launches += 1;
  return cuda_check(cudaGetLastError(), "lanes init");
}

int lanes_half_sweep(qisg_handle *h, int colour, int count_only) {
  return h->W == 64 ? half_sweep_t<unsigned long long>(h, colour, count_only)
                    : half_sweep_t<unsigned int>(h, colour, count_only);
}

int lanes_pt(qisg_handle *h, int explicit_pass) {
  if (h->per_sample_launch) {
    for (int64_t a = 0; a < h->n_samples; ++a) {
      const int rc = pt_pass(h, explicit_pass, a, 1);
      if (rc) return rc;
    }
    return QISG_OK;
  }
  return pt_pass(h, explicit_pass, 0, h->n_samples);
}

int lanes_measure(qisg_handle *h, int force_to_q) {
  return h->W == 64 ? measure_t<unsigned long long>(h, force_to_q)
                    : measure_t<unsigned int>(h, force_to_q);
}

int lanes_energies_by_slot(qisg_handle *h) {
  const int64_t n = h->n_samples * h->n_rep * h->n_slots;
  lanes_by_slot_kernel<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(
      h->d_walker, h->d_U, h->d_out, h->n_samples, h->n_rep, h->n_slots, h->N);
  h->launches++;
  return cuda_check(cudaGetLastError(), "lanes energies");
}

// Samples per staging chunk of the spin transfers (at most 256 MB of int8).
int64_t spin_chunk(const qisg_handle *h) {
  const int64_t per_a = (int64_t)h->n_rep * h->n_slots * h->N;
  return std::max<int64_t>(1, ((int64_t)256 << 20) / per_a);
}

template <typename Word>
int get_spins_t(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *S) {
  const int64_t per_a = (int64_t)h->n_rep * h->n_slots * h->N, chunk = std::min(n_a, spin_chunk(h));
  if (n_a == 0) return QISG_OK;
  int8_t *stage = nullptr;
  int rc = cuda_check(cudaMalloc(&stage, (size_t)(chunk * per_a)), "cudaMalloc");
  for (int64_t a0 = 0; a0 < n_a && !rc; a0 += chunk) {
    const int64_t na = std::min(chunk, n_a - a0), n = na * per_a;
    lanes_extract_kernel<Word><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(
        reinterpret_cast<const Word *>(h->spins), stage, a_lo + a0, na, h->N, h->n_rep, h->n_slots, h->rpw,
        h->n_groups);
    h->launches++;
    rc = cuda_check(cudaGetLastError(), "unpack spins");
    if (!rc)
      rc = cuda_check(cudaMemcpyAsync(S + a0 * per_a, stage, (size_t)n, cudaMemcpyDeviceToHost, h->stream), "copy");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(h->stream), "sync");
  }
  if (stage) cudaFree(stage);
  return rc;
}

template <typename Word>
int set_spins_t(qisg_handle *h, const int8_t *S) {
  const int64_t per_a = (int64_t)h->n_rep * h->n_slots * h->N, chunk = std::min(h->n_samples, spin_chunk(h));
  int8_t *stage = nullptr;
  int rc = cuda_check(cudaMalloc(&stage, (size_t)(chunk * per_a)), "cudaMalloc");
  for (int64_t a0 = 0; a0 < h->n_samples && !rc; a0 += chunk) {
    const int64_t na = std::min(chunk, h->n_samples - a0), n = na * h->n_groups * h->N;
    rc = cuda_check(cudaMemcpyAsync(stage, S + a0 * per_a, (size_t)(na * per_a), cudaMemcpyHostToDevice, h->stream),
                    "copy spins");
    if (rc) break;
    lanes_pack_kernel<Word><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(
        reinterpret_cast<Word *>(h->spins), stage, a0, na, h->N, h->n_rep, h->n_slots, h->rpw, h->n_groups);
    h->launches++;
    rc = cuda_check(cudaGetLastError(), "pack spins");
  }
  if (!rc) rc = cuda_check(cudaStreamSynchronize(h->stream), "sync");
  if (stage) cudaFree(stage);
  return rc;
}

int lanes_stage_spins(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *d) {
  const int64_t n = n_a * h->n_rep * h->n_slots * h->N;
  if (n == 0) return QISG_OK;
  if (h->W == 64)
    lanes_extract_kernel<unsigned long long><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(
        reinterpret_cast<const unsigned long long *>(h->spins), d, a_lo, n_a, h->N, h->n_rep, h->n_slots, h->rpw,
        h->n_groups);
  else
    lanes_extract_kernel<unsigned int><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(
        reinterpret_cast<const unsigned int *>(h->spins), d, a_lo, n_a, h->N, h->n_rep, h->n_slots, h->rpw,
        h->n_groups);
  h->launches++;
  return cuda_check(cudaGetLastError(), "unpack spins");
}

int lanes_get_spins(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *S) {
  return h->W == 64 ? get_spins_t<unsigned long long>(h, a_lo, n_a, S) : get_spins_t<unsigned int>(h, a_lo, n_a, S);
}

int lanes_set_spins(qisg_handle *h, const int8_t *S) {
  return h->W == 64 ? set_spins_t<unsigned long long>(h, S) : set_spins_t<unsigned int>(h, S);
}

int lanes_get_couplings(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *J) {
  const int64_t plane = (int64_t)h->L * h->L;
  std::vector<uint8_t> buf(plane * n_a);
  int rc = cuda_check(cudaMemcpyAsync(buf.data(), (const uint8_t *)h->J + a_lo * plane, buf.size(),
                                      cudaMemcpyDeviceToHost, h->stream),
                      "copy J");
  if (rc) return rc;
  rc = cuda_check(cudaStreamSynchronize(h->stream), "sync");
  if (rc) return rc;
  for (int64_t i = 0; i < plane * n_a; ++i) {
    J[2 * i] = (buf[i] & 1u) ? -1 : 1;
    J[2 * i + 1] = (buf[i] & 2u) ? -1 : 1;
  }
  return QISG_OK;
}

int lanes_set_couplings(qisg_handle *h, const int8_t *J) {
  const int64_t plane = (int64_t)h->L * h->L;
  std::vector<uint8_t> buf(plane * h->n_samples);
  for (int64_t i = 0; i < plane * h->n_samples; ++i)
    buf[i] = (uint8_t)((J[2 * i] == -1 ? 1u : 0u) | (J[2 * i + 1] == -1 ? 2u : 0u));
  int rc = cuda_check(cudaMemcpyAsync(h->J, buf.data(), buf.size(), cudaMemcpyHostToDevice, h->stream),
                      "copy J");
  if (rc) return rc;
  return cuda_check(cudaStreamSynchronize(h->stream), "sync");
}

}  // namespace qisg
