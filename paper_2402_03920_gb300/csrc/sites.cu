// SITES packing: the paper's own multi-site coding with its daemon-bit
// Metropolis rule (Sec. 2.1 and 2.1.1, Appendices B and C), for equal
// couplings k_tau = k.  A 32-bit word holds 32 imaginary-time sites of ONE
// system: with M = L_tau / 32, site (x, y, tau) is bit tau / M of word-site
// x + L y + L^2 (tau mod M).  M is even, so all bits of a word have the
// colour (x + y + tau) mod 2 of their word-site, and the six neighbours of a
// word are whole words: four spatial ones at the same tau, and the words at
// tau +- 1, rotated by one bit where the word stream wraps (tau mod M = M-1
// upwards, 0 downwards), with the antiperiodic sign on the bit that crosses
// tau = L_tau - 1 -> 0.
//
// The update of a word: u = number of unsatisfied bonds of each bit (6 bond
// masks, a bit-sliced 6-input counter), d = the bit's daemon level, and the
// bit flips iff u + d >= 3 (a flip costs 4k(3 - u); P(d >= n) = e^{-4kn}).
// d >= n is "the first n of the daemon words b4, b8, b12 have the bit set",
// so the flip mask is
//   f = [u >= 3] | b4 & ([u = 2] | b8 & ([u = 1] | b12 & [u = 0])).
// Each daemon word comes from one Philox4x32-10 call (the upper halves of
// four 64-bit "50/50" words) and one xoroshiro128++ state step of the same
// 128 bits (the lower halves); byte i of the word is n* of 64-bit word i,
// the bin of the word in the cumulative table of the walker's slot.  n* is
// found from an index of the top kDaemonLutBits bits, staged in shared
// memory: the words with a given prefix fall in the bins [n_min, n_min +
// span], so n* = n_min + #{q in [n_min, n_min + span): cumulative(q) <= word}.
// With span <= 1 the entry holds the upper half of the one cut point and
// n* = n_min + [upper half of the word > it]; with span >= 2 the upper
// halves of the span cut points are compared one by one.  Only when an
// upper half equals a cut point's does the lower half matter (a running
// product of the XORs of the upper halves then becomes 0): the whole daemon
// word is redone with the full 64-bit words, and the xoroshiro step is only
// computed there.  The bytes are assembled by multiply-adds with run-time
// factors, which keeps that work off the logic pipe.
//
// Device arrays (systems walker-major; PT exchanges slot labels only):
//   spins  u32 [a][r][w][L^2 M]       bit = 1 <=> spin -1
//   J      uint8 [a][x + L*y]          bit0: J(+x) = -1, bit1: J(+y) = -1
//   U      u64 [a][r][w][2]            unsatisfied spatial / tau bonds of walker w
//   cum    u64 [n_slots][256]          cumulative(0..254) of Sec. 2.1.1; [255] = 2^64-1
//   lut    uint2 [n_slots][2^kDaemonLutBits]
//                                      {n_min, | 2^31 when span >= 2; upper half of
//                                       cumulative(n_min) when span = 1, else 2^32 - 1}
//   span   uint8 [n_slots][2^kDaemonLutBits] (after lut)   span of each prefix
#include <algorithm>
#include <cmath>
#include <cstring>

#include "qisg_internal.cuh"

namespace qisg {
namespace {

constexpr int kBlock = 256;

struct SitesArgs {
  uint32_t *spins;
  const uint8_t *J;
  const int32_t *walker;
  const unsigned long long *cum;
  const uint2 *lut;
  const uint8_t *span;
  unsigned long long *U;
  const unsigned long long *d_t;
  uint2 key;
  uint32_t m8, m16, m24;       // 2^8, 2^16, 2^24 at run time (byte assembly by multiply-adds)
  FastDiv half_plane_div, half_L_div;
  int L, M, plane, half_plane, n_words, half_words;
  int n_slots, n_rep;
  int blocks_per_sys, words_per_thread;
  int tau_ap;
};

// xoroshiro128++ state step (Blackman and Vigna, 2019) on the 128 bits of a
// Philox output, state (x | y << 32, z | w << 32); returns the new state's
// four 32-bit quarters in the same order.
__device__ __forceinline__ uint4 xoroshiro_step(uint4 x) {
  const unsigned long long s0 = (unsigned long long)x.x | ((unsigned long long)x.y << 32);
  const unsigned long long s1 = (unsigned long long)x.z | ((unsigned long long)x.w << 32);
  const unsigned long long tt = s1 ^ s0;
  const unsigned long long n0 = ((s0 << 49) | (s0 >> 15)) ^ tt ^ (tt << 21);
  const unsigned long long n1 = (tt << 28) | (tt >> 36);
  return make_uint4((uint32_t)n0, (uint32_t)(n0 >> 32), (uint32_t)n1, (uint32_t)(n1 >> 32));
}

// Philox4x32-10 with 32 x 32 -> 64-bit products (the same function as
// philox(): each round's high and low halves come from one wide multiply).
__device__ __forceinline__ uint4 philox_wide(uint4 c, uint2 k) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const unsigned long long p0 = (unsigned long long)kPhiloxM0 * c.x;
    const unsigned long long p1 = (unsigned long long)kPhiloxM1 * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k.x, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k.y, (uint32_t)p0);
    k.x += kPhiloxW0;
    k.y += kPhiloxW1;
  }
  return c;
}

// Exact n* of 64-bit word i of a daemon word (the rare path): the lower
// half from the xoroshiro step of the Philox output x, then the count of
// the cut points at or below the word among the prefix's candidates.
static __device__ __noinline__ uint32_t nstar_exact(uint4 x, int i, const uint2 *lut, const uint8_t *span,
                                                    const unsigned long long *cum) {
  const uint4 lo = xoroshiro_step(x);
  const uint32_t hi = pick4(x, i), l = pick4(lo, i);
  const unsigned long long R = ((unsigned long long)hi << 32) | l;
  const uint32_t h = hi >> (32 - kDaemonLutBits);
  uint32_t n = lut[h].x & 0xFFu;
  const uint32_t end = n + span[h];
  for (uint32_t q = n; q < end; ++q) n += (R >= cum[q]) ? 1u : 0u;
  return n;
}

// n* of a 64-bit word from its upper half hi (entry e: e.x = n_min, bit 31
// set when the cell holds two or more cut points; e.y = upper half of the
// one cut point, else all ones).  *prod collects hi ^ (cut's upper half):
// it becomes 0 when they tie (the lower halves then decide; a zero product
// without a tie only sends the word to the exact path).
__device__ __forceinline__ uint32_t nstar_hi(uint32_t hi, const uint2 *lut, const uint32_t *cut_hi,
                                             const uint8_t *span, uint32_t *prod) {
  const uint32_t h = hi >> (32 - kDaemonLutBits);
  const uint2 e = lut[h];
  uint32_t n = e.x + (hi > e.y ? 1u : 0u);
  *prod *= hi ^ e.y;
  if ((int)e.x < 0) {   // two or more cut points: compare their upper halves
    const uint32_t n0 = e.x & 0xFFu, end = n0 + span[h];
    n = n0;
    for (uint32_t q = n0; q < end; ++q) {
      const uint32_t c = cut_hi[q];
      n += hi > c ? 1u : 0u;
      *prod *= hi ^ c;
    }
  }
  return n;
}

// Daemon word `which` (0: b4, 1: b8, 2: b12) of word-site ws of system
// (a, r, slot s) in sweep t: byte i is n* of the 64-bit word whose upper
// half is Philox output i.
__device__ __forceinline__ uint32_t daemon_word(uint32_t ws, uint32_t t, uint32_t c2, uint32_t c3, uint2 key,
                                                const uint2 *lut, const uint32_t *cut_hi, const uint8_t *span,
                                                const unsigned long long *cum, uint32_t m8, uint32_t m16,
                                                uint32_t m24) {
  const uint4 x = philox_wide(make_uint4(ws, t, c2, c3), key);
  uint32_t prod = 1;
  const uint32_t b = nstar_hi(x.x, lut, cut_hi, span, &prod) + nstar_hi(x.y, lut, cut_hi, span, &prod) * m8 +
                     nstar_hi(x.z, lut, cut_hi, span, &prod) * m16 + nstar_hi(x.w, lut, cut_hi, span, &prod) * m24;
  if (prod != 0) return b;
  return nstar_exact(x, 0, lut, span, cum) | (nstar_exact(x, 1, lut, span, cum) << 8) |
         (nstar_exact(x, 2, lut, span, cum) << 16) | (nstar_exact(x, 3, lut, span, cum) << 24);
}

__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) { return (a & b) | (c & (a | b)); }

// One half sweep (colour 0 = red, 1 = blue).  Block x serves system
// x / blocks_per_sys (sys = (a n_rep + r) n_slots + w) and the colour words
// [chunk * 256 * wpt, (chunk + 1) * 256 * wpt) of it, thread i taking words
// chunk * 256 * wpt + i + 256 j.  The blue pass counts, per system, the
// unsatisfied bonds of its words after the update: every bond has exactly
// one blue end, so this is each bond once.  Chunk 0 of the red pass clears
// the system's counters.  count_only: no update (energies of the stored
// state).
template <bool BLUE>
__global__ void __launch_bounds__(kBlock) sites_half_sweep_kernel(SitesArgs p, int count_only) {
  __shared__ unsigned long long cum_s[256];
  __shared__ uint32_t cut_hi_s[256];
  __shared__ __align__(16) uint8_t span_s[1 << kDaemonLutBits];
  extern __shared__ __align__(16) uint2 lut_s[];   // [2^kDaemonLutBits]
  __shared__ unsigned long long red_s[2][kBlock / 32];
  const int64_t sys = blockIdx.x / p.blocks_per_sys;
  const int chunk = (int)(blockIdx.x - sys * p.blocks_per_sys);
  const int w = (int)(sys % p.n_slots);
  const int64_t ar = sys / p.n_slots;   // a * n_rep + r
  const int r = (int)(ar % p.n_rep);
  const int64_t a = ar / p.n_rep;
  const int colour = BLUE ? 1 : 0;
  if (!BLUE && chunk == 0 && threadIdx.x < 2) p.U[sys * 2 + threadIdx.x] = 0;
  if (!BLUE && count_only) return;
  // slot of walker w: lane l of every warp reads walker_at[a][r][l]
  const int lane = threadIdx.x & 31;
  const int32_t wl = lane < p.n_slots ? __ldg(p.walker + ar * p.n_slots + lane) : -1;
  const int s = max(__ffs(__ballot_sync(0xFFFFFFFFu, wl == w)) - 1, 0);   // rows are permutations
  // stage the slot's tables
  {
    const unsigned long long *cg = p.cum + (size_t)s * 256;
    for (int i = threadIdx.x; i < 256; i += kBlock) {
      const unsigned long long v = __ldg(cg + i);
      cum_s[i] = v;
      cut_hi_s[i] = (uint32_t)(v >> 32);
    }
    const uint4 *lg = reinterpret_cast<const uint4 *>(p.lut + ((size_t)s << kDaemonLutBits));
    uint4 *ls = reinterpret_cast<uint4 *>(lut_s);
    for (int i = threadIdx.x; i < (1 << kDaemonLutBits) / 2; i += kBlock) ls[i] = __ldg(lg + i);
    const uint4 *sg = reinterpret_cast<const uint4 *>(p.span + ((size_t)s << kDaemonLutBits));
    uint4 *ss = reinterpret_cast<uint4 *>(span_s);
    for (int i = threadIdx.x; i < (1 << kDaemonLutBits) / 16; i += kBlock) ss[i] = __ldg(sg + i);
  }
  __syncthreads();
  uint32_t *S = p.spins + sys * p.n_words;
  const uint8_t *J = p.J + a * p.plane;
  const uint32_t t = (uint32_t)*p.d_t;
  const uint32_t c2 = (uint32_t)s | ((uint32_t)r << 16);
  const uint32_t c3 = (DOM_DAEMON << 28) | (uint32_t)a;
  const uint32_t ap_up = p.tau_ap ? 0x80000000u : 0u, ap_dn = p.tau_ap ? 1u : 0u;
  unsigned long long us_cnt = 0, ut_cnt = 0;
  const int base = chunk * kBlock * p.words_per_thread + threadIdx.x;
  for (int j = 0; j < p.words_per_thread; ++j) {
    const int idx = base + j * kBlock;
    if (idx >= p.half_words) break;
    // idx -> (tau', y, x) of the colour's words
    const uint32_t tq = p.half_plane_div.div((uint32_t)idx);
    const uint32_t rem = (uint32_t)idx - tq * (uint32_t)p.half_plane;
    const uint32_t y = p.half_L_div.div(rem);
    const uint32_t xh = rem - y * (uint32_t)(p.L >> 1);
    const uint32_t x = 2 * xh + ((y + tq + (uint32_t)colour) & 1u);
    const int L = p.L;
    const int ws = (int)(x + (uint32_t)L * y + (uint32_t)p.plane * tq);
    const int xp = (x == (uint32_t)(L - 1)) ? ws - (L - 1) : ws + 1;
    const int xm = (x == 0) ? ws + (L - 1) : ws - 1;
    const int yp = (y == (uint32_t)(L - 1)) ? ws - (L - 1) * L : ws + L;
    const int ym = (y == 0) ? ws + (L - 1) * L : ws - L;
    const bool top = tq == (uint32_t)(p.M - 1), bottom = tq == 0;
    const int tp = top ? ws - (p.M - 1) * p.plane : ws + p.plane;
    const int tm = bottom ? ws + (p.M - 1) * p.plane : ws - p.plane;
    const uint32_t c = S[ws];
    uint32_t nup = S[tp], ndn = S[tm];
    if (top) nup = __funnelshift_r(nup, nup, 1) ^ ap_up;   // bit j <- bit j+1 of tau' = 0
    if (bottom) ndn = __funnelshift_l(ndn, ndn, 1) ^ ap_dn;   // bit j <- bit j-1 of tau' = M-1
    const int i2 = (int)(x + (uint32_t)L * y);
    const uint32_t jc = __ldg(J + i2);
    const uint32_t jxm = __ldg(J + (x == 0 ? i2 + L - 1 : i2 - 1));
    const uint32_t jym = __ldg(J + (y == 0 ? i2 + (L - 1) * L : i2 - L));
    // unsatisfied bond masks: J S S' = -1 <=> bit(S) ^ bit(S') ^ bit(J) = 1
    uint32_t e1 = c ^ S[xp] ^ (0u - (jc & 1u));
    uint32_t e2 = c ^ S[xm] ^ (0u - (jxm & 1u));
    uint32_t e3 = c ^ S[yp] ^ (0u - ((jc >> 1) & 1u));
    uint32_t e4 = c ^ S[ym] ^ (0u - ((jym >> 1) & 1u));
    uint32_t e5 = c ^ nup;
    uint32_t e6 = c ^ ndn;
    uint32_t f = 0;
    if (!count_only) {
      // u = u0 + 2 u1 + 4 u2, bit-sliced over the 32 sites
      const uint32_t s1 = e1 ^ e2 ^ e3, k1 = maj3(e1, e2, e3);
      const uint32_t s2 = e4 ^ e5 ^ e6, k2 = maj3(e4, e5, e6);
      const uint32_t u0 = s1 ^ s2, h = s1 & s2;
      const uint32_t u1 = k1 ^ k2 ^ h, u2 = maj3(k1, k2, h);
      const uint32_t ge3 = u2 | (u1 & u0);
      const uint32_t eq2 = ~u2 & u1 & ~u0, eq1 = ~u2 & ~u1 & u0, eq0 = ~(u2 | u1 | u0);
      // b4, b8, b12 in a rolled loop (one copy of the lookup code)
      uint32_t b4 = 0, b8 = 0, b12 = 0;
#pragma unroll 1
      for (uint32_t which = 0; which < 3; ++which) {
        const uint32_t dw = daemon_word((uint32_t)ws, t, c2, c3 | (which << 24), p.key, lut_s, cut_hi_s, span_s, cum_s,
                                        p.m8, p.m16, p.m24);
        b4 = b8;
        b8 = b12;
        b12 = dw;
      }
      f = ge3 | (b4 & (eq2 | (b8 & (eq1 | (b12 & eq0)))));
      S[ws] = c ^ f;
    }
    if (BLUE) {
      us_cnt += __popc(e1 ^ f) + __popc(e2 ^ f) + __popc(e3 ^ f) + __popc(e4 ^ f);
      ut_cnt += __popc(e5 ^ f) + __popc(e6 ^ f);
    }
  }
  if (BLUE) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      us_cnt += __shfl_xor_sync(0xFFFFFFFFu, us_cnt, o);
      ut_cnt += __shfl_xor_sync(0xFFFFFFFFu, ut_cnt, o);
    }
    if (lane == 0) {
      red_s[0][threadIdx.x >> 5] = us_cnt;
      red_s[1][threadIdx.x >> 5] = ut_cnt;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
      unsigned long long v = 0;
      for (int i = 0; i < kBlock / 32; ++i) v += red_s[threadIdx.x][i];
      if (v) atomicAdd(p.U + sys * 2 + threadIdx.x, v);
    }
  }
}

// Overlaps of the configurations at slot s (Appendix E.1): count the sites
// where the replicas r1 < r2 differ (popcount of the XOR of their words);
// q = N - 2 * count.  Grid (chunks, n_slots, n_a).
__global__ void __launch_bounds__(kBlock) sites_overlap_kernel(const uint32_t *spins, const int32_t *walker,
                                                               long long *qcnt, int64_t a0, int n_words,
                                                               int n_rep, int n_slots) {
  extern __shared__ long long q_s[];  // [n_pairs]
  const int n_pairs = n_rep * (n_rep - 1) / 2;
  const int s = blockIdx.y;
  const int64_t a = a0 + blockIdx.z;
  for (int i = threadIdx.x; i < n_pairs; i += blockDim.x) q_s[i] = 0;
  __syncthreads();
  const int32_t *wa = walker + a * n_rep * n_slots;
  int p = 0;
  for (int r1 = 0; r1 < n_rep; ++r1) {
    const uint32_t *S1 = spins + ((a * n_rep + r1) * n_slots + wa[r1 * n_slots + s]) * (int64_t)n_words;
    for (int r2 = r1 + 1; r2 < n_rep; ++r2, ++p) {
      const uint32_t *S2 = spins + ((a * n_rep + r2) * n_slots + wa[r2 * n_slots + s]) * (int64_t)n_words;
      unsigned cnt = 0;
      for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_words; i += gridDim.x * blockDim.x)
        cnt += __popc(S1[i] ^ S2[i]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
      if ((threadIdx.x & 31) == 0 && cnt)
        atomicAdd(reinterpret_cast<unsigned long long *>(&q_s[p]), (unsigned long long)cnt);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n_pairs; i += blockDim.x)
    if (q_s[i])
      atomicAdd(reinterpret_cast<unsigned long long *>(&qcnt[(a * n_slots + s) * n_pairs + i]),
                (unsigned long long)q_s[i]);
}

// Start spins from Philox domain DOM_INIT: one thread per word, 32 draws.
__global__ void sites_init_spins_kernel(uint32_t *spins, int64_t n_sys, int n_words, int L, int M, int n_rep,
                                        int n_slots, uint2 key) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n_sys * n_words) return;
  const int ws = (int)(c % n_words);
  const int64_t sys = c / n_words;
  const int w = (int)(sys % n_slots);
  const int64_t ar = sys / n_slots;
  const int r = (int)(ar % n_rep);
  const int64_t a = ar / n_rep;
  const int plane = L * L;
  const int tq = ws / plane, i2 = ws - tq * plane;
  uint32_t v = 0;
  for (int j = 0; j < 32; ++j) {
    const uint32_t site = (uint32_t)(i2 + plane * (tq + j * M));
    const uint4 x = philox(make_uint4(site, (uint32_t)w, (uint32_t)a, (DOM_INIT << 28) | (uint32_t)r), key);
    if (!(x.x & 1u)) v |= 1u << j;   // spin -1
  }
  spins[c] = v;
}

// int8 +-1 spins [sys][site] of systems sys0 .. sys0+n_sys-1 from the
// lattice (site (x, y, tau) is bit tau / M of word x + L y + L^2 (tau mod M)).
__global__ void sites_extract_kernel(const uint32_t *spins, int8_t *out, int64_t sys0, int64_t n_sys, int plane,
                                     int M, int n_words, int64_t N) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n_sys * N) return;
  const int64_t sys = c / N, site = c - sys * N;
  const int tau = (int)(site / plane), i2 = (int)(site - (int64_t)tau * plane);
  const uint32_t v = spins[(sys0 + sys) * n_words + i2 + plane * (tau % M)];
  out[c] = ((v >> (tau / M)) & 1u) ? -1 : 1;
}

// The words of systems sys0 .. sys0+n_sys-1 from int8 +-1 spins staged as
// [sys][site]: a thread per word, 32 spins along tau.
__global__ void sites_pack_kernel(uint32_t *spins, const int8_t *stage, int64_t sys0, int64_t n_sys, int plane, int M,
                                  int n_words, int64_t N) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n_sys * n_words) return;
  const int64_t sys = c / n_words;
  const int ws = (int)(c - sys * n_words), tq = ws / plane, i2 = ws - tq * plane;
  uint32_t v = 0;
  for (int j = 0; j < 32; ++j)
    if (stage[sys * N + i2 + (int64_t)plane * (tq + j * M)] == -1) v |= 1u << j;
  spins[(sys0 + sys) * n_words + ws] = v;
}

SitesArgs make_args(qisg_handle *h) {
  SitesArgs p;
  p.spins = reinterpret_cast<uint32_t *>(h->spins);
  p.J = reinterpret_cast<const uint8_t *>(h->J);
  p.walker = h->d_walker;
  p.cum = h->d_dcum;
  p.lut = h->d_dlut;
  p.span = reinterpret_cast<const uint8_t *>(h->d_dlut + ((size_t)h->n_slots << kDaemonLutBits));
  p.U = h->d_U;
  p.d_t = h->d_t;
  p.key = make_uint2((uint32_t)h->seed, (uint32_t)(h->seed >> 32));
  p.m8 = 1u << 8;
  p.m16 = 1u << 16;
  p.m24 = 1u << 24;
  p.L = h->L;
  p.M = h->Lt / 32;
  p.plane = h->L * h->L;
  p.half_plane = p.plane / 2;
  p.n_words = p.plane * p.M;
  p.half_words = p.n_words / 2;
  p.half_plane_div = FastDiv((uint32_t)p.half_plane);
  p.half_L_div = FastDiv((uint32_t)(h->L / 2));
  p.n_slots = h->n_slots;
  p.n_rep = h->n_rep;
  p.tau_ap = h->tau_ap;
  // words per thread: up to 8, while the grid keeps 8 blocks per SM
  const int64_t n_sys = h->n_samples * h->n_rep * h->n_slots;
  int wpt = h->sweep_tile[0] > 0 ? h->sweep_tile[0] : 8;
  while (wpt > 1 && n_sys * ((p.half_words + kBlock * wpt - 1) / (kBlock * wpt)) < 8LL * h->n_sm) wpt >>= 1;
  p.words_per_thread = wpt;
  p.blocks_per_sys = (p.half_words + kBlock * wpt - 1) / (kBlock * wpt);
  return p;
}

// Fixed-point numbers in [0, 2) with 126 fractional bits.
using u128 = unsigned __int128;
constexpr int kFrac = 126;
const u128 kOne = (u128)1 << kFrac;

// floor(a b / 2^126) for a, b < 2^127, through 64-bit limbs.
u128 mulq(u128 a, u128 b) {
  const uint64_t a0 = (uint64_t)a, a1 = (uint64_t)(a >> 64), b0 = (uint64_t)b, b1 = (uint64_t)(b >> 64);
  const u128 p00 = (u128)a0 * b0, p01 = (u128)a0 * b1, p10 = (u128)a1 * b0, p11 = (u128)a1 * b1;
  const u128 mid = (p00 >> 64) + (uint64_t)p01 + (uint64_t)p10;
  const u128 hi = p11 + (p01 >> 64) + (p10 >> 64) + (mid >> 64);   // bits 128..255
  const u128 lo = (mid << 64) | (uint64_t)p00;                       // bits 0..127
  return (hi << (128 - kFrac)) | (lo >> kFrac);
}

// e^{-x} for 0 <= x <= 64 in fixed point: x = y 2^m with y < 1/16 (exact),
// e^{-y} by its Taylor series (terms to y^30/30!), then m squarings.
u128 exp_neg(double x) {
  int m = 0;
  while (x / std::ldexp(1.0, m) >= 1.0 / 16) ++m;
  const double y = x / std::ldexp(1.0, m);   // exact: a power-of-two scaling
  int ex = 0;
  const double fr = std::frexp(y, &ex);     // y = fr 2^ex, fr in [0.5, 1)
  const uint64_t mant = (uint64_t)std::ldexp(fr, 53);
  const int sh = kFrac + ex - 53;
  const u128 yq = y == 0.0 ? 0 : (sh >= 0 ? (u128)mant << sh : (u128)(mant >> (-sh)));
  u128 term = kOne, pos = kOne, neg = 0;
  for (int i = 1; i <= 30; ++i) {
    term = mulq(term, yq) / (u128)i;
    if (i & 1) neg += term;
    else pos += term;
  }
  u128 r = pos - neg;
  for (int i = 0; i < m; ++i) r = mulq(r, r);
  return r;
}

}  // namespace

// cumulative(0..254) of Sec. 2.1.1 for coupling k (0 <= k <= 16):
// floor(2^64 sum_{m <= n} p^pop(m) (1-p)^(8-pop(m))), p = e^{-4k}, in
// fixed point with 126 fractional bits (the paper uses 128-bit floats).
void daemon_cumulative(double k, uint64_t *cum) {
  const u128 p = exp_neg(4.0 * k);
  const u128 q = kOne - p;
  u128 pw[9], qw[9];
  pw[0] = qw[0] = kOne;
  for (int c = 1; c <= 8; ++c) {
    pw[c] = mulq(pw[c - 1], p);
    qw[c] = mulq(qw[c - 1], q);
  }
  u128 acc = 0;
  for (int n = 0; n < 255; ++n) {
    const int c = __builtin_popcount((unsigned)n);
    acc += mulq(pw[c], qw[8 - c]);
    cum[n] = (uint64_t)(acc >> (kFrac - 64));
  }
}

// Prefix index of one cumulative table: entry h covers the words
// [h 2^(64-bits), (h+1) 2^(64-bits)), whose n* lie in [n_min, n_max];
// entry = n_min | (n_max - n_min) << 8.
void daemon_lut(const uint64_t *cum, int bits, uint16_t *lut, uint32_t *cut_hi = nullptr) {
  auto ns = [&](uint64_t R) {
    uint32_t c = 0;
    while (c < 255 && cum[c] <= R) ++c;   // cum is non-decreasing
    return c;
  };
  for (uint64_t h = 0; h < (1ull << bits); ++h) {
    const uint64_t lo = h << (64 - bits), hi = lo + ((~0ull) >> bits);
    const uint32_t a = ns(lo), b = ns(hi);
    lut[h] = (uint16_t)(a | ((b - a) << 8));
    // upper half of the one cut point inside the cell, else all ones
    if (cut_hi) cut_hi[h] = (b - a == 1) ? (uint32_t)(cum[a] >> 32) : 0xFFFFFFFFu;
  }
}

int sites_build_tables(qisg_handle *h) {
  const int n = h->n_slots, nl = 1 << kDaemonLutBits;
  std::vector<unsigned long long> cum((size_t)n * 256);
  std::vector<uint2> lut((size_t)n * nl);
  std::vector<uint8_t> span((size_t)n * nl);
  std::vector<uint16_t> l16((size_t)nl);
  std::vector<uint32_t> chi((size_t)nl);
  for (int s = 0; s < n; ++s) {
    uint64_t c[256];
    daemon_cumulative(h->k[s], c);
    c[255] = ~0ull;
    for (int i = 0; i < 256; ++i) cum[(size_t)s * 256 + i] = c[i];
    daemon_lut(c, kDaemonLutBits, l16.data(), chi.data());
    for (int i = 0; i < nl; ++i) {
      const uint32_t nmin = l16[(size_t)i] & 0xFFu, sp = l16[(size_t)i] >> 8;
      lut[(size_t)s * nl + i] = make_uint2(nmin | (sp >= 2 ? 0x80000000u : 0u), chi[(size_t)i]);
      span[(size_t)s * nl + i] = (uint8_t)sp;
    }
  }
  int rc = cuda_check(cudaMemcpyAsync(h->d_dcum, cum.data(), cum.size() * 8, cudaMemcpyHostToDevice, h->stream),
                      "copy cumulative tables");
  if (!rc)
    rc = cuda_check(cudaMemcpyAsync(h->d_dlut, lut.data(), lut.size() * 8, cudaMemcpyHostToDevice, h->stream),
                    "copy prefix index");
  if (!rc)
    rc = cuda_check(cudaMemcpyAsync(h->d_dlut + lut.size(), span.data(), span.size(), cudaMemcpyHostToDevice,
                                    h->stream),
                    "copy prefix spans");
  // the host vectors must outlive the copies
  if (!rc) rc = cuda_check(cudaStreamSynchronize(h->stream), "sync");
  return rc;
}

int sites_init(qisg_handle *h) {
  int rc = sites_build_tables(h);
  if (rc) return rc;
  const uint2 key = make_uint2((uint32_t)h->seed, (uint32_t)(h->seed >> 32));
  rc = lanes_init_couplings(h);
  if (rc) return rc;
  const int n_words = h->L * h->L * (h->Lt / 32);
  const int64_t n_sys = h->n_samples * h->n_rep * h->n_slots;
  const int64_t nS = n_sys * n_words;
  if ((nS + 255) / 256 > 0x7FFFFFFF) return fail(QISG_EINVAL, "lattice too large");
  sites_init_spins_kernel<<<(unsigned)((nS + 255) / 256), 256, 0, h->stream>>>(
      reinterpret_cast<uint32_t *>(h->spins), n_sys, n_words, h->L, h->Lt / 32, h->n_rep, h->n_slots, key);
  h->launches++;
  return cuda_check(cudaGetLastError(), "sites init");
}

int sites_half_sweep(qisg_handle *h, int colour, int count_only) {
  const SitesArgs p = make_args(h);
  const int64_t n_sys = h->n_samples * h->n_rep * h->n_slots;
  const int64_t blocks = n_sys * p.blocks_per_sys;
  if (blocks > 0x7FFFFFFF) return fail(QISG_EINVAL, "lattice too large for one launch");
  constexpr size_t smem = sizeof(uint2) << kDaemonLutBits;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(sites_half_sweep_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(sites_half_sweep_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  const int tok = prof_begin(h, sweep_kind(colour));
  if (colour == 1)
    sites_half_sweep_kernel<true><<<(unsigned)blocks, kBlock, smem, h->stream>>>(p, count_only);
  else
    sites_half_sweep_kernel<false><<<(unsigned)blocks, kBlock, smem, h->stream>>>(p, count_only);
  prof_end(h, sweep_kind(colour), tok);
  h->launches++;
  return cuda_check(cudaGetLastError(), "sites half sweep");
}

int sites_measure(qisg_handle *h, int force_to_q) {
  const int n_pairs = h->n_pairs();
  if (n_pairs > 0) {
    const int n_words = h->L * h->L * (h->Lt / 32);
    const int64_t chunks = std::min<int64_t>((n_words + kBlock - 1) / kBlock, 64);
    const size_t smem = (size_t)n_pairs * 8;
    for (int64_t a0 = 0; a0 < h->n_samples; a0 += 65535) {
      const int64_t na = std::min<int64_t>(65535, h->n_samples - a0);
      const int tok = prof_begin(h, QISG_KERNEL_MEASURE);
      sites_overlap_kernel<<<dim3((unsigned)chunks, (unsigned)h->n_slots, (unsigned)na), kBlock, smem,
                             h->stream>>>(reinterpret_cast<const uint32_t *>(h->spins), h->d_walker, h->d_q, a0,
                                          n_words, h->n_rep, h->n_slots);
      prof_end(h, QISG_KERNEL_MEASURE, tok);
      h->launches++;
    }
    int rc = cuda_check(cudaGetLastError(), "sites overlaps");
    if (rc) return rc;
  }
  return lanes_finalize(h, force_to_q);
}

int sites_stage_spins(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *d) {
  const int M = h->Lt / 32, plane = h->L * h->L, n_words = plane * M;
  const int64_t n_sys = n_a * h->n_rep * h->n_slots, n = n_sys * h->N;
  if (n == 0) return QISG_OK;
  sites_extract_kernel<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(
      reinterpret_cast<const uint32_t *>(h->spins), d, a_lo * h->n_rep * h->n_slots, n_sys, plane, M, n_words, h->N);
  h->launches++;
  return cuda_check(cudaGetLastError(), "unpack spins");
}

int sites_get_spins(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *S) {
  const int M = h->Lt / 32, plane = h->L * h->L, n_words = plane * M;
  const int64_t per_sys = h->N, n_sys = n_a * h->n_rep * h->n_slots, sys_lo = a_lo * h->n_rep * h->n_slots;
  if (n_sys == 0) return QISG_OK;
  const int64_t chunk = std::min<int64_t>(n_sys, std::max<int64_t>(1, ((int64_t)256 << 20) / per_sys));
  int8_t *stage = nullptr;
  int rc = cuda_check(cudaMalloc(&stage, (size_t)(chunk * per_sys)), "cudaMalloc");
  for (int64_t s0 = 0; s0 < n_sys && !rc; s0 += chunk) {
    const int64_t ns = std::min(chunk, n_sys - s0), n = ns * per_sys;
    sites_extract_kernel<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(
        reinterpret_cast<const uint32_t *>(h->spins), stage, sys_lo + s0, ns, plane, M, n_words, h->N);
    h->launches++;
    rc = cuda_check(cudaGetLastError(), "unpack spins");
    if (!rc)
      rc = cuda_check(cudaMemcpyAsync(S + s0 * per_sys, stage, (size_t)n, cudaMemcpyDeviceToHost, h->stream), "copy");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(h->stream), "sync");
  }
  if (stage) cudaFree(stage);
  return rc;
}

int sites_set_spins(qisg_handle *h, const int8_t *S) {
  const int M = h->Lt / 32, plane = h->L * h->L, n_words = plane * M;
  const int64_t per_sys = h->N, n_sys = h->n_samples * h->n_rep * h->n_slots;
  const int64_t chunk = std::min<int64_t>(n_sys, std::max<int64_t>(1, ((int64_t)256 << 20) / per_sys));
  int8_t *stage = nullptr;
  int rc = cuda_check(cudaMalloc(&stage, (size_t)(chunk * per_sys)), "cudaMalloc");
  for (int64_t s0 = 0; s0 < n_sys && !rc; s0 += chunk) {
    const int64_t ns = std::min(chunk, n_sys - s0), n = ns * n_words;
    rc = cuda_check(cudaMemcpyAsync(stage, S + s0 * per_sys, (size_t)(ns * per_sys), cudaMemcpyHostToDevice,
                                    h->stream),
                    "copy spins");
    if (rc) break;
    sites_pack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(reinterpret_cast<uint32_t *>(h->spins),
                                                                          stage, s0, ns, plane, M, n_words, h->N);
    h->launches++;
    rc = cuda_check(cudaGetLastError(), "pack spins");
  }
  if (!rc) rc = cuda_check(cudaStreamSynchronize(h->stream), "sync");
  if (stage) cudaFree(stage);
  return rc;
}

}  // namespace qisg

extern "C" int qisg_daemon_tables(double k, int lut_bits, uint64_t *cum, uint16_t *lut) {
  if (!cum || !(k >= 0.0) || !(k <= 16.0)) return qisg::fail(QISG_EINVAL, "need 0 <= k <= 16 and a table");
  if (lut && (lut_bits < 1 || lut_bits > 16)) return qisg::fail(QISG_EINVAL, "lut_bits must be in 1..16");
  qisg::daemon_cumulative(k, cum);
  if (lut) qisg::daemon_lut(cum, lut_bits, lut);
  return QISG_OK;
}
