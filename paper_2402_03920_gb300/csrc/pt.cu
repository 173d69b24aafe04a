// Parallel-tempering pass (Sec. 2.1), one warp per chain (a, r).
//
// Lane s holds the energies of the configuration at slot s and draws the
// Philox word of pair (s, s+1); the pass over pairs s = 0, 1, ... is then a
// short uniform loop over warp shuffles: the configuration carried up from
// pair s-1 meets the original occupant of slot s+1, and the decision fixes
// the final occupant of slot s.
//
//   LANES  : energies are counted by walker; the pass reorders walker_at.
//   SAMPLES: energies are counted by slot; the pass reorders walker_at and
//            the slot energies.  A block is the 8 chains of one (sample
//            block b, replica r, 8-lane octet); their accepted pairs are
//            OR-ed into the lane masks acc[b][r][s] (bit l: sample b*W+l
//            exchanged pair (s, s+1)), from which the permute kernel moves
//            the spin bits.
#include "qisg_internal.cuh"

namespace qisg {
namespace {

// LANES: one warp per chain, chains in (a, r) order.
template <bool WIDE>
__global__ void pt_lanes_kernel(int32_t *walker, unsigned long long *U, const PTConst *ptc, const double *sq,
                                const unsigned long long *d_t, uint2 key, int64_t a0, int64_t n_chains,
                                int n_rep, int n_slots, int explicit_pass) {
  const int64_t chain = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (chain >= n_chains) return;   // whole warp
  const int64_t a = a0 + chain / n_rep;
  const int r = (int)(chain % n_rep);
  const uint32_t t = (uint32_t)(explicit_pass ? *d_t - 1ull : *d_t);
  pt_chain<false, false, WIDE>(walker + (a * n_rep + r) * n_slots, U + (a * n_rep + r) * n_slots * 2, ptc, sq, key,
                               t, a, r, n_slots);
}

// SAMPLES: block = 8 warps = samples b*W + 8*o + v (v = warp) of replica r;
// the block then ORs the 8 accept bitmasks into the lane masks acc[b][r][s]
// (cleared by the red pass of the sweep), one thread per pair.
template <typename Word, bool WIDE>
__global__ void __launch_bounds__(256) pt_samples_kernel(int32_t *walker, unsigned long long *U, Word *accw,
                                                         const PTConst *ptc, const double *sq,
                                                         const unsigned long long *d_t, uint2 key,
                                                         int64_t n_samples, int n_rep, int n_slots,
                                                         int explicit_pass, unsigned long long *adv) {
  pdl_begin();
  constexpr int W = (int)sizeof(Word) * 8, octs = W / 8;
  __shared__ uint32_t bits[8];
  const uint32_t bid = blockIdx.x;
  const int o = (int)(bid % octs);
  const uint32_t rest = bid / octs;
  const uint32_t b = rest / (uint32_t)n_rep;
  const int r = (int)(rest - b * (uint32_t)n_rep);
  const int v = threadIdx.x >> 5;
  const int64_t a = (int64_t)b * W + 8 * o + v;
  uint32_t acc = 0;
  if (a < n_samples) {
    const uint32_t t = (uint32_t)(adv ? adv[1] : explicit_pass ? *d_t - 1ull : *d_t);
    acc = pt_chain<true, false, WIDE>(walker + (a * n_rep + r) * n_slots, U + (a * n_rep + r) * n_slots * 2, ptc,
                                      sq, key, t, a, r, n_slots);
  }
  if ((threadIdx.x & 31) == 0) bits[v] = acc;
  __syncthreads();
  const int s = threadIdx.x;   // thread s gathers pair s of the 8 chains
  if (s + 1 < n_slots) {
    Word m = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) m |= (Word)((bits[u] >> s) & 1u) << (8 * o + u);
    if (m) {
      Word *out = accw + ((int64_t)b * n_rep + r) * n_slots;
      if (sizeof(Word) == 8)
        atomicOr(reinterpret_cast<unsigned long long *>(&out[s]), (unsigned long long)m);
      else
        atomicOr(reinterpret_cast<unsigned int *>(&out[s]), (unsigned int)m);
    }
  }
  // advance: the pass read t from adv[1] (the blue pass's copy); no block
  // reads adv[0], so block 0 sets it to t + 1 for the next sweep
  if (adv && blockIdx.x == 0 && threadIdx.x == 0) adv[0] = adv[1] + 1ull;
}

template <typename Word, bool WIDE>
void launch_pt_samples(qisg_handle *h, uint2 key, int explicit_pass, unsigned long long *adv) {
  const unsigned blocks = (unsigned)(h->n_b * h->n_rep * (h->W / 8));
  launch_kernel(h->pdl, pt_samples_kernel<Word, WIDE>, dim3(blocks), dim3(256), 0, h->stream, h->d_walker, h->d_U,
                reinterpret_cast<Word *>(h->d_acc), reinterpret_cast<const PTConst *>(h->d_ptc), h->d_sq, h->d_t, key,
                h->n_samples, h->n_rep, h->n_slots, explicit_pass, adv);
}

}  // namespace

int pt_pass(qisg_handle *h, int explicit_pass, int64_t a0, int64_t n_a, unsigned long long *adv, bool force_wide) {
  const uint2 key = make_uint2((uint32_t)h->seed, (uint32_t)(h->seed >> 32));
  const bool wide = force_wide || 2 * h->N >= (int64_t(1) << 30);   // energy differences beyond 31 bits
  const int tok = prof_begin(h, QISG_KERNEL_PT);
  if (h->layout == QISG_LAYOUT_SAMPLES) {
    if (h->W == 64) {
      if (wide) launch_pt_samples<unsigned long long, true>(h, key, explicit_pass, adv);
      else launch_pt_samples<unsigned long long, false>(h, key, explicit_pass, adv);
    } else {
      if (wide) launch_pt_samples<unsigned int, true>(h, key, explicit_pass, adv);
      else launch_pt_samples<unsigned int, false>(h, key, explicit_pass, adv);
    }
  } else {
    const int64_t n_chains = n_a * h->n_rep;
    constexpr int kWarps = 4;
    const unsigned blocks = (unsigned)((n_chains + kWarps - 1) / kWarps);
    const PTConst *ptc = reinterpret_cast<const PTConst *>(h->d_ptc);
    if (wide)
      pt_lanes_kernel<true><<<blocks, 32 * kWarps, 0, h->stream>>>(h->d_walker, h->d_U, ptc, h->d_sq, h->d_t, key, a0,
                                                                   n_chains, h->n_rep, h->n_slots, explicit_pass);
    else
      pt_lanes_kernel<false><<<blocks, 32 * kWarps, 0, h->stream>>>(h->d_walker, h->d_U, ptc, h->d_sq, h->d_t, key,
                                                                    a0, n_chains, h->n_rep, h->n_slots, explicit_pass);
  }
  prof_end(h, QISG_KERNEL_PT, tok);
  h->launches++;
  return cuda_check(cudaGetLastError(), "pt pass");
}

}  // namespace qisg
