// SAMPLES packing: a word of W = 32 or 64 bits holds W disorder samples
// (lane l = sample a - b*W of sample block b) at one (replica, slot).  This
// is Ito-Kanada's multi-sample multispin coding (Sec. 2.1.1): all lanes of a
// word see the same ladder slot, so they share one Metropolis table row and
// one draw R (the draw is keyed on the 64-sample block a >> 6).  The local
// energy class (u_s, u_t) of every lane is computed with bit-sliced adders;
// a mux tree over the class bits selects the per-class reject flags.
//
// Because a word is one slot, a PT exchange between slots s and s+1 of a
// sample (Sec. 2.1) moves that sample's bits between the two slot words; the
// walker labels are tracked alongside so results are reported by walker.
//
// Device arrays (N = L*L*L_tau, n_q = ceil(n_rep / 4), r = 4q + j):
//   spins  Word [b][s][q][site][4]    bit = 1 <=> spin -1
//   J      Word [b][x + L*y][2]       bit = 1 <=> J = -1
//   U      u64 [a][r][s][2]           unsatisfied spatial / tau bonds, by slot
//   acc    Word [b][r][s]             PT accept masks of the last pass
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "qisg_internal.cuh"

namespace qisg {
namespace {

constexpr int kBlock = 256;          // 64 quads of 4 replicas
constexpr int kQuads = kBlock / 4;
constexpr int kMaxSlotsPermute = 32;

template <typename Word>
struct SamplesArgs {
  Word *spins;
  const Word *J;
  const uint32_t *T;
  unsigned long long *U;
  const unsigned long long *d_t;
  uint2 key;
  int64_t N, half_N;
  int L, Lt, plane, half_plane, n_slots, n_rep, n_q, W;
  int seg_sites;         // G: sites of one colour each quad walks along tau (the most of any thread)
  int n_seg;             // segments per column
  int seg_base, seg_rem; // W = 32 replica-quad kernel: segment g of a column holds seg_base + (g < seg_rem)
                         // sites (n_seg segments covering the L_tau / 2 sites of the colour)
  int seg_blocks;        // > 0: blocks per segment, each block one segment of 128 columns (plane a
                         // multiple of 128), so a block's walks have one length; 0: a block takes
                         // 128 consecutive (segment, column) pairs and seg_rem = 0
  int blocks_per_set;    // blocks per (b, s, q) word set
  uint32_t one;          // 1 as a runtime value (accept_flag)
  unsigned long long *t_copy;   // blue pass, fused mode: copy t here for the PT pass
  int tau_ap;                   // antiperiodic along tau: the wrap tau bond flips sign
  // division by the invariants of the index decomposition (32-bit indices)
  FastDiv fd_bps, fd_nq, fd_ns, fd_plane, fd_L, fd_sb;
  // cleared by the red pass (nothing reads them until the blue pass / PT):
  unsigned long long *zero_U;   // bond counters, n_zero_U words
  int64_t n_zero_U;
  Word *zero_acc;               // PT lane masks, n_zero_acc words
  int64_t n_zero_acc;
};

// Accept constants per slot for the classes (u_t = 0: u_s = 0..4),
// (u_t = 1: u_s = 0, 1), (u_t = 2: u_s = 0, 1); the classes u_t >= 1,
// u_s >= 2 always accept.  A class with table entry T accepts a draw R iff
// R < T', T' = T for a finite entry (T = 0: never) and T' = 2^32 for the
// always-accept sentinel.  The slot holds C = 2^64 - T' (mod 2^64): R + C
// stays below 2^64 iff R < T', and then its high word is 0xFFFFFFFF (R + C
// >= 2^64 - 2^32), else 0.  So one 64-bit multiply-add, R * 1 + C, gives the
// class's accept mask in its high word, on the integer multiply-add pipe
// (leaving the logic pipe to the bit-sliced arithmetic).
struct SlotThresholds {
  unsigned long long v[kMaxSlotsPT][9];
};

// one is the runtime value 1 (a kernel parameter, so the compiler keeps the
// multiply-add rather than splitting it into two additions)
__device__ __forceinline__ uint32_t accept_flag(uint32_t R, unsigned long long C, uint32_t one) {
  unsigned long long v;
  asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(v) : "r"(R), "r"(one), "l"(C));
  return (uint32_t)(v >> 32);
}

// Accept mask of one 32-bit word: a mux tree over the class planes (u_s in
// us2 us1 us0, u_t in ut1 ut0) of the per-class accept masks.
__device__ __forceinline__ uint32_t accept_mask(uint32_t R, const unsigned long long *C, uint32_t us0, uint32_t us1,
                                                uint32_t us2, uint32_t ut0, uint32_t ut1, uint32_t one) {
#define QISG_A(c) accept_flag(R, C[c], one)
  const uint32_t row0 = mux(us2, QISG_A(4), mux(us1, mux(us0, QISG_A(3), QISG_A(2)), mux(us0, QISG_A(1), QISG_A(0))));
  const uint32_t high = us1 | us2;
  const uint32_t row1 = high | mux(us0, QISG_A(6), QISG_A(5));
  const uint32_t row2 = high | mux(us0, QISG_A(8), QISG_A(7));
#undef QISG_A
  return mux(ut1, row2, mux(ut0, row1, row0));
}

// Per-replica-class sum of the block's counters: thread (quad, j) holds
// counter c of replica j; the 64 quads' counters of each replica are summed
// by a tree in shared memory (vertical adds, W lanes per operation) and lane
// l of replica j's total is added to out[j * W + l].
template <typename Word, int K>
__device__ __forceinline__ void quad_sum_counters(const VCount<Word, K> &c, Word *buf, int *out) {
  constexpr int W = (int)sizeof(Word) * 8;
  constexpr int NQ = kQuads, LOG = 6;   // 64 quads per block
  constexpr int KF = K + LOG;
  static_assert((1 << LOG) == NQ, "quads per block");
  const int j = threadIdx.x & 3, quad = threadIdx.x >> 2;
#pragma unroll
  for (int i = 0; i < K; ++i) buf[(j * KF + i) * NQ + quad] = c.p[i];
  __syncthreads();
#pragma unroll
  for (int lvl = 0; lvl < LOG; ++lvl) {
    const int half = NQ >> (lvl + 1);
    for (int w = threadIdx.x; w < 4 * half; w += blockDim.x) {
      const int g = w / half, e = w - g * half;
      Word *a = buf + (size_t)g * KF * NQ + e;
      Word carry = 0;
#pragma unroll
      for (int i = 0; i < K + lvl; ++i) {
        const Word x = a[i * NQ], y = a[i * NQ + half];
        a[i * NQ] = x ^ y ^ carry;
        carry = maj3(x, y, carry);
      }
      a[(K + lvl) * NQ] = carry;
    }
    __syncthreads();
  }
  for (int w = threadIdx.x; w < 4 * W; w += blockDim.x) {
    const int g = w / W, l = w - g * W;
    int v = 0;
#pragma unroll
    for (int i = 0; i < KF; ++i) v |= (int)((buf[(g * KF + i) * NQ] >> l) & 1u) << i;
    out[w] = v;
  }
  __syncthreads();   // buf is reused by the caller
}

// Accept mask of one word for class planes (us, ut): the class masks are 32
// bits wide (accept_flag), doubled for 64-bit words.
template <typename Word>
__device__ __forceinline__ Word accept_word(uint32_t R, const unsigned long long *C, Word us0, Word us1, Word us2,
                                            Word ut0, Word ut1, uint32_t one) {
  if constexpr (sizeof(Word) == 4) {
    return accept_mask(R, C, us0, us1, us2, ut0, ut1, one);
  } else {
    auto f = [&](int c) -> Word {
      const uint32_t m = accept_flag(R, C[c], one);
      return ((Word)m << 32) | (Word)m;
    };
    const Word row0 = mux(us2, f(4), mux(us1, mux(us0, f(3), f(2)), mux(us0, f(1), f(0))));
    const Word high = us1 | us2;
    const Word row1 = high | mux(us0, f(6), f(5));
    const Word row2 = high | mux(us0, f(8), f(7));
    return mux(ut1, row2, mux(ut0, row1, row0));
  }
}

// One half sweep, column walk.  Block: one (b, s, q) word set; quad thread j
// owns replica r = 4q + j.  Quad k owns one (x, y) column and a segment of
// G sites of the colour along tau (tau = tau0, tau0 + 2, ...; tau0 = 2 G seg
// + ((colour + x + y) & 1)), so the column's couplings and neighbour offsets
// stay in registers and the word at tau - 1 is the previous step's tau + 1.
// Per group of 4 steps every thread of a quad computes one Philox call (for
// step 4g + j), which serves the four replicas of that site; the results are
// exchanged in shared memory.  The thresholds of the slot come from the
// parameter bank.  G2 = ceil(log2(G / 4)) sizes the per-thread energy
// counters, summed per replica by a tree in shared memory.
template <typename Word, bool BLUE, int G2>
__global__ void __launch_bounds__(kBlock) samples_half_sweep_kernel(SamplesArgs<Word> p,
                                                                    const __grid_constant__ SlotThresholds th,
                                                                    int colour, int count_only) {
  pdl_begin();
  constexpr int W = (int)sizeof(Word) * 8;
  constexpr int KS = G2 + 5;   // u_s sum <= 4 * 4 * 2^G2 per thread
  constexpr int KT = G2 + 4;   // u_t sum <= 2 * 4 * 2^G2 per thread
  __shared__ uint4 rnd[kBlock];   // one Philox call per thread and group of 4 steps
  __shared__ Word buf[BLUE ? 4 * (KS + 6) * kQuads : 1];
  __shared__ int accU[BLUE ? 2 * 4 * W : 1];

  const uint32_t bid = blockIdx.x;
  const uint32_t set = p.fd_bps.div(bid);
  const uint32_t chunk = bid - set * (uint32_t)p.blocks_per_set;
  const uint32_t bs = p.fd_nq.div(set);
  const int q = (int)(set - bs * (uint32_t)p.n_q);
  const uint32_t b = p.fd_ns.div(bs);
  const int s = (int)(bs - b * (uint32_t)p.n_slots);
  const int j = threadIdx.x & 3;
  const int quad = threadIdx.x >> 2;
  const int r = 4 * q + j;
  {   // counters / masks the host asked this pass to clear
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p.n_zero_U; i += stride) p.zero_U[i] = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p.n_zero_acc; i += stride)
      p.zero_acc[i] = 0;
  }
  const unsigned long long *C = th.v[s];

  const int L = p.L, plane = p.plane, G = p.seg_sites;
  const uint32_t Lt = (uint32_t)p.Lt;
  const uint32_t gq = chunk * (uint32_t)kQuads + (uint32_t)quad;
  const bool live = gq < (uint32_t)plane * (uint32_t)p.n_seg;   // uniform per quad
  const uint32_t segu = p.fd_plane.div(gq);
  const int i2 = (int)(gq - segu * (uint32_t)plane);
  const int seg = (int)segu;
  const int y = (int)p.fd_L.div((uint32_t)i2), x = i2 - y * L;
  const uint32_t ixp = (uint32_t)((x + 1 == L ? 0 : x + 1) + L * y), ixm = (uint32_t)((x == 0 ? L - 1 : x - 1) + L * y);
  const uint32_t iyp = (uint32_t)(x + L * (y + 1 == L ? 0 : y + 1)), iym = (uint32_t)(x + L * (y == 0 ? L - 1 : y - 1));
  const Word *Jb = p.J + b * (int64_t)plane * 2;
  Word Jxp = 0, Jxm = 0, Jyp = 0, Jym = 0;
  if (live) {
    Jxp = Jb[2 * i2];
    Jxm = Jb[2 * ixm];
    Jyp = Jb[2 * i2 + 1];
    Jym = Jb[2 * iym + 1];
  }
  const uint32_t tau0 = 2u * (uint32_t)G * (uint32_t)seg + (uint32_t)((colour + x + y) & 1);

  Word *base = p.spins + ((b * p.n_slots + s) * p.n_q + q) * p.N * 4 + j;
  const unsigned long long t = *p.d_t;
  if (p.t_copy && bid == 0 && threadIdx.x == 0) *p.t_copy = t;
  const uint32_t ctr_z = (uint32_t)s | ((uint32_t)(r >> 2) << 16);
  const uint32_t ctr_w = (DOM_SWEEP << 28) | (uint32_t)((b * W) >> 6);

  VCount<Word, KS> cs;
  VCount<Word, KT> ct;
  if (BLUE) {
    cs.zero();
    ct.zero();
  }

  // word at tau0 - 1 (the first step's tau - 1); later steps reuse tau + 1
  Word prev_up = 0;
  if (live) {
    const uint32_t off0 = tau0 * (uint32_t)plane;
    prev_up = base[(size_t)((uint32_t)i2 + (tau0 == 0 ? (Lt - 1) * (uint32_t)plane : off0 - plane)) * 4];
  }
  uint32_t *rw = reinterpret_cast<uint32_t *>(rnd);   // [step i][quad][replica j]
  for (int g4 = 0; 4 * g4 < G; ++g4) {
    // every load of the group's 4 steps is issued before any store: the
    // steps touch disjoint words (centres of this colour, neighbours of the
    // other), which the compiler cannot prove through one base pointer
    Word c[4], up[4], nb[4][4];
    if (live) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int k = 4 * g4 + i;
        if (k < G) {
          const uint32_t tau = tau0 + 2u * (uint32_t)k;
          const uint32_t off = tau * (uint32_t)plane;
          const uint32_t offp = tau + 1 == Lt ? 0u : off + plane;
          c[i] = base[(size_t)((uint32_t)i2 + off) * 4];
          up[i] = base[(size_t)((uint32_t)i2 + offp) * 4];
          nb[i][0] = base[(size_t)(ixp + off) * 4];
          nb[i][1] = base[(size_t)(ixm + off) * 4];
          nb[i][2] = base[(size_t)(iyp + off) * 4];
          nb[i][3] = base[(size_t)(iym + off) * 4];
        } else {
          c[i] = up[i] = nb[i][0] = nb[i][1] = nb[i][2] = nb[i][3] = 0;
        }
      }
      if (4 * g4 + j < G) {
        const uint32_t tj = tau0 + 2u * (uint32_t)(4 * g4 + j);
        const uint4 x = philox(make_uint4((uint32_t)i2 + tj * (uint32_t)plane, (uint32_t)t, ctr_z, ctr_w), p.key);
        *reinterpret_cast<uint4 *>(rw + ((j * kQuads + quad) << 2)) = x;
      }
    }
    __syncwarp();
    if (live) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int k = 4 * g4 + i;
        if (k >= G) break;
        const uint32_t R = rw[((i * kQuads + quad) << 2) + j];
        const uint32_t tau = tau0 + 2u * (uint32_t)k;
        const uint32_t site = (uint32_t)i2 + tau * (uint32_t)plane;
        const Word sc = c[i];
        const Word dn = prev_up;   // tau - 1 is the previous step's tau + 1
        prev_up = up[i];
        const Word b1 = sc ^ nb[i][0] ^ Jxp;
        const Word b2 = sc ^ nb[i][1] ^ Jxm;
        const Word b3 = sc ^ nb[i][2] ^ Jyp;
        const Word b4 = sc ^ nb[i][3] ^ Jym;
        // the antiperiodic wrap bond is unsatisfied when its spins agree
        const Word t1 = sc ^ up[i] ^ ones_if<Word>(p.tau_ap && tau + 1 == Lt);
        const Word t2 = sc ^ dn ^ ones_if<Word>(p.tau_ap && tau == 0);
        // bit-sliced u_s (3 bits) and u_t (2 bits)
        const Word s1 = b1 ^ b2 ^ b3;
        const Word c1 = maj3(b1, b2, b3);
        const Word us0 = s1 ^ b4;
        const Word c2 = s1 & b4;
        const Word us1 = c1 ^ c2;
        const Word us2 = c1 & c2;
        const Word ut0 = t1 ^ t2;
        const Word ut1 = t1 & t2;
        // accept mask: mux tree over (u_t, u_s) of the per-class masks
        const Word flip = count_only ? Word(0) : accept_word<Word>(R, C, us0, us1, us2, ut0, ut1, p.one);
        if (!count_only) base[(size_t)site * 4] = sc ^ flip;
        if (BLUE) {
          // unsatisfied counts after the flip: u -> 4 - u (spatial), 2 - u (tau)
          const Word vs1 = us1 ^ (flip & us0);
          const Word vs2 = mux(flip, ~(us0 | us1 | us2), us2);
          const Word vt1 = mux(flip, ~(ut0 | ut1), ut1);
          cs.add3(us0, vs1, vs2);
          ct.add2(ut0, vt1);
        }
      }
    }
    __syncwarp();
  }

  if (BLUE) {
    quad_sum_counters<Word, KS>(cs, buf, accU);
    quad_sum_counters<Word, KT>(ct, buf, accU + 4 * W);
    for (int i = threadIdx.x; i < 4 * W; i += blockDim.x) {
      const int jj = i / W, lane = i - jj * W;
      const int rr = 4 * q + jj;
      if (rr >= p.n_rep) continue;
      const int64_t a = b * W + lane;
      unsigned long long *u = p.U + ((a * p.n_rep + rr) * p.n_slots + s) * 2;
      if (accU[i]) atomicAdd(u, (unsigned long long)accU[i]);
      if (accU[4 * W + i]) atomicAdd(u + 1, (unsigned long long)accU[4 * W + i]);
    }
  }
}

// ---- W = 32: one thread per (column segment, 4 replicas) ----
//
// The 4 replica words of a site are adjacent ([site][4] x 32 bits), so one
// 16-byte load brings a site's replica quad and one Philox call gives the
// quad's four draws.  A thread walks G sites of the colour along tau in one
// (x, y) column, loading the next site while it updates the current one
// (the steps touch disjoint words: centres of this colour, neighbours of the
// other).  The 9 thresholds that can reject come from the parameter bank,
// uniform over the block.  In the blue pass each thread keeps bit-sliced
// counters per replica; the block then sums them with a tree in shared
// memory (vertical adds, 32 lanes per operation) instead of warp shuffles.
constexpr int kBlock4 = 128;
constexpr int kLog2Block4 = 7;

struct Quad4 {
  uint4 c, up, xp, xm, yp, ym;
};

__device__ __forceinline__ uint32_t q4(const uint4 &v, int j) {
  return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}

// Red pass with the pending PT exchanges folded in (W = 32).  After a PT pass
// (Sec. 2.1) the stored lattice still holds every slot's words as they were
// before the exchanges; the accepted pairs of each (sample block, replica)
// are the lane masks acc[b][r][s].  A thread owns one red site of one
// replica and streams the slot words s = 0, 1, ... of the seven sites it
// needs (the site, its two tau and four spatial neighbours), carrying up the
// word that the sequential pass moves through pair s (masked exchange of
// the carried word with slot s+1's), so slot s's words are final when the
// thread reaches s.  It updates the red site of slot s from them and writes
// it, with its blue partner at tau + 1 (every blue site is the partner of
// exactly one red site, the one below it), to the other lattice buffer; the
// blue pass then works on that buffer in place.  The four replica threads of
// a site share one Philox call per slot, made by one of them per group of
// four slots and exchanged in shared memory.  The kernel is bounded to seven
// blocks of 128 threads per SM (72 registers), so the 32768 red sites x 4
// replicas of an L = 16, L_tau = 256 word set run as one wave on 152 SMs.
template <typename Word>
struct FusedRedArgsT {
  const Word *src;
  Word *dst;
  const Word *J;
  const Word *acc;
  const unsigned long long *d_t;
  unsigned long long *zero_U;
  int64_t n_zero_U;
  uint2 key;
  int64_t N;
  int L, Lt, plane, n_slots, n_q, n_rep, blocks_per_set;
  uint32_t one;
  unsigned *ticket;   // the blue pass's PT ticket counter, reset here (or null)
  int tau_ap;
  FastDiv fd_bps, fd_nq, fd_plane, fd_L;
};
using FusedRedArgs = FusedRedArgsT<uint32_t>;

// Address base + i elements of `bytes` bytes (the runtime element size) by
// one 64-bit multiply-add.
template <typename T>
__device__ __forceinline__ T *addr_scaled(T *base, uint32_t i, uint32_t bytes) {
  unsigned long long a;
  asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(a) : "r"(i), "r"(bytes), "l"(reinterpret_cast<unsigned long long>(base)));
  return reinterpret_cast<T *>(a);
}

// Address base + 4 i computed by one 64-bit multiply-add (four is the
// runtime value 4, so the compiler keeps the multiply-add): measured 1% off
// the L=16, L_tau=256 sweep against the compiler's own address arithmetic.
__device__ __forceinline__ uint32_t *addr_mad(const uint32_t *base, uint32_t i, uint32_t four) {
  unsigned long long a;
  asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(a) : "r"(i), "r"(four), "l"(reinterpret_cast<unsigned long long>(base)));
  return reinterpret_cast<uint32_t *>(a);
}

__global__ void __launch_bounds__(kBlock4, 7) samples_red_fused_kernel(const FusedRedArgs p,
                                                                     const __grid_constant__ SlotThresholds th) {
  pdl_begin();
  __shared__ uint32_t msk[4][kMaxSlotsPT];
  __shared__ unsigned long long thr[kMaxSlotsPT][9];
  __shared__ uint4 rnd[kBlock4];   // per warp: [slot in group][quad][replica]
  const uint32_t bid = blockIdx.x;
  const uint32_t set = p.fd_bps.div(bid);   // (b, q)
  const uint32_t chunk = bid - set * (uint32_t)p.blocks_per_set;
  const uint32_t b = p.fd_nq.div(set);
  const int q = (int)(set - b * (uint32_t)p.n_q);
  const int n = p.n_slots;
  {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p.n_zero_U; i += stride) p.zero_U[i] = 0;
    if (p.ticket && blockIdx.x == 0 && threadIdx.x == 0) *p.ticket = 0u;
  }

  const uint32_t tid = chunk * (uint32_t)kBlock4 + threadIdx.x;
  const int j = (int)(tid & 3u);
  const uint32_t quad = tid >> 2;
  const uint32_t P = (uint32_t)p.plane, Lt = (uint32_t)p.Lt, L = (uint32_t)p.L;
  const bool live = quad < P * (Lt / 2);
  const uint32_t seg = p.fd_plane.div(quad);
  const uint32_t i2 = quad - seg * P;
  const uint32_t y = p.fd_L.div(i2), x = i2 - y * L;
  const uint32_t tau = 2 * seg + ((x + y) & 1u);
  const uint32_t ixp = (x + 1 == L ? 0 : x + 1) + L * y, ixm = (x == 0 ? L - 1 : x - 1) + L * y;
  const uint32_t iyp = x + L * (y + 1 == L ? 0 : y + 1), iym = x + L * (y == 0 ? L - 1 : y - 1);
  const uint32_t off = tau * P;
  // the antiperiodic wrap bond is unsatisfied when its spins agree
  const uint32_t gtp = ones_if<uint32_t>(p.tau_ap && tau + 1 == Lt), gtm = ones_if<uint32_t>(p.tau_ap && tau == 0);
  // the seven sites: centre, tau + 1 (blue partner), tau - 1, x+, x-, y+, y-
  uint32_t z[7];
  z[0] = i2 + off;
  z[1] = i2 + (tau + 1 == Lt ? 0u : off + P);
  z[2] = i2 + (tau == 0 ? (Lt - 1) * P : off - P);
  z[3] = ixp + off;
  z[4] = ixm + off;
  z[5] = iyp + off;
  z[6] = iym + off;
  // word of site zz at slot sl: slot base (uniform over the block) + 4 zz + j
  // (layout [b][s][q][site][4])
  const int64_t base = (((int64_t)b * n * p.n_q + q) * p.N) * 4;
  const int64_t SS = (int64_t)p.n_q * p.N * 4;
  uint32_t zo[7];
  const uint32_t *Jb = p.J + (int64_t)b * P * 2;
  uint32_t Jxp = 0, Jxm = 0, Jyp = 0, Jym = 0;
  const unsigned long long t = *p.d_t;
  const uint32_t ctr_w = (DOM_SWEEP << 28) | ((b * 32u) >> 6);
  uint32_t cw[7], n1[7];   // carried words at the current slot; words of the next slot
#pragma unroll
  for (int k = 0; k < 7; ++k) zo[k] = 4 * z[k] + (uint32_t)j;
  const uint32_t *sb = p.src + base;
  uint32_t *db = p.dst + base;
  if (live) {
    Jxp = Jb[2 * i2];
    Jxm = Jb[2 * ixm];
    Jyp = Jb[2 * i2 + 1];
    Jym = Jb[2 * iym + 1];
#pragma unroll
    for (int k = 0; k < 7; ++k) cw[k] = sb[zo[k]];
    if (n > 1)
#pragma unroll
      for (int k = 0; k < 7; ++k) n1[k] = sb[SS + zo[k]];
  }
  uint32_t *rw = reinterpret_cast<uint32_t *>(rnd) + (threadIdx.x >> 5) * 128;
  const int ql = (int)((threadIdx.x & 31) >> 2);
  int g = 0;
  uint4 r4 = make_uint4(0u, 0u, 0u, 0u);
  // the bases of slots sl + 2 (loads) and sl (stores) advance by the slot
  // stride as the slots are taken in order
  const uint32_t *ps2 = sb + 2 * SS;
  uint32_t *pd = db;
  const uint32_t four = p.one << 2;
  // slot sl = 4 g + i: the words of slot sl after the exchanges of pairs
  // 0 .. sl, the update of the red site and the stores; H1 / H2: slot sl + 1
  // / sl + 2 exists (known at compile time, so the slot has no checks)
  auto update_slot = [&](const int i, const int sl, auto has1, auto has2) {
    constexpr bool H1 = decltype(has1)::value, H2 = decltype(has2)::value;
    uint32_t fw[7];
    if constexpr (H1) {
      uint32_t n2[7];
      if constexpr (H2) {
#pragma unroll
        for (int k = 0; k < 7; ++k) n2[k] = *addr_mad(ps2, zo[k], four);
      }
      const uint32_t m = msk[j][sl];
#pragma unroll
      for (int k = 0; k < 7; ++k) {   // lanes of m exchange pair (sl, sl + 1)
        fw[k] = mux(m, n1[k], cw[k]);
        cw[k] = mux(m, cw[k], n1[k]);
        if constexpr (H2) n1[k] = n2[k];
      }
    } else {
#pragma unroll
      for (int k = 0; k < 7; ++k) fw[k] = cw[k];
    }
    const uint32_t R = rw[((i * 8 + ql) << 2) + j];
    const unsigned long long *C = thr[sl];
    const uint32_t sc = fw[0];
    const uint32_t b1 = sc ^ fw[3] ^ Jxp;
    const uint32_t b2 = sc ^ fw[4] ^ Jxm;
    const uint32_t b3 = sc ^ fw[5] ^ Jyp;
    const uint32_t b4 = sc ^ fw[6] ^ Jym;
    const uint32_t t1 = sc ^ fw[1] ^ gtp;
    const uint32_t t2 = sc ^ fw[2] ^ gtm;
    const uint32_t s1 = b1 ^ b2 ^ b3;
    const uint32_t c1 = maj3(b1, b2, b3);
    const uint32_t us0 = s1 ^ b4;
    const uint32_t c2 = s1 & b4;
    const uint32_t us1 = c1 ^ c2;
    const uint32_t us2 = c1 & c2;
    const uint32_t ut0 = t1 ^ t2;
    const uint32_t ut1 = t1 & t2;
    const uint32_t acc = accept_mask(R, C, us0, us1, us2, ut0, ut1, p.one);
    *addr_mad(pd, zo[0], four) = sc ^ acc;
    *addr_mad(pd, zo[1], four) = fw[1];
    ps2 += SS;
    pd += SS;
  };
  const std::integral_constant<bool, true> yes;
  const std::integral_constant<bool, false> no;
  // groups of four slots that all have two successors; this thread's Philox
  // call of the group (slot 4 g + j), the next group's call made while this
  // group's slots are updated
  if (live && 6 <= n) r4 = philox(make_uint4(z[0], (uint32_t)t, (uint32_t)j | ((uint32_t)q << 16), ctr_w), p.key);
  // the PT masks of the (b, q) set, staged after the first slots' loads and
  // draw are issued, so the two round trips to L2 overlap
  for (int i = threadIdx.x; i < 4 * kMaxSlotsPT; i += blockDim.x) {
    const int jj = i / kMaxSlotsPT, sl = i - jj * kMaxSlotsPT;
    const int rr = 4 * q + jj;
    msk[jj][sl] = (rr < p.n_rep && sl + 1 < n) ? p.acc[((int64_t)b * p.n_rep + rr) * n + sl] : 0u;
  }
  // the slots' threshold constants through shared memory, so that the
  // accept flags take them from ordinary registers: measured 6 fewer
  // logic-pipe and 9 more multiply-add-pipe instructions per word, 2.1% off
  // the L=16, L_tau=256 sweep (the replica-quad red and the blue kernels,
  // which would hold them across their sites, lost by it)
  for (int i = threadIdx.x; i < n * 9; i += blockDim.x) thr[i / 9][i % 9] = th.v[i / 9][i % 9];
  __syncthreads();
  for (; 4 * g + 6 <= n; ++g) {
    if (live) *reinterpret_cast<uint4 *>(rw + ((j * 8 + ql) << 2)) = r4;
    __syncwarp();
    if (live && 4 * (g + 1) + j < n)
      r4 = philox(make_uint4(z[0], (uint32_t)t, (uint32_t)(4 * (g + 1) + j) | ((uint32_t)q << 16), ctr_w), p.key);
    if (live) {
#pragma unroll 2   // two slots' loads in flight: 72 registers, seven blocks per SM
      for (int i = 0; i < 4; ++i) update_slot(i, 4 * g + i, yes, yes);
    }
    __syncwarp();
  }
  // a multiple of four slots leaves one group, always of the same shape:
  // two slots with two successors, one with one, one with none
  if (n % 4 == 0 && 4 * g < n) {
    if (live) {
      if (g == 0)
        r4 = philox(make_uint4(z[0], (uint32_t)t, (uint32_t)(4 * g + j) | ((uint32_t)q << 16), ctr_w), p.key);
      *reinterpret_cast<uint4 *>(rw + ((j * 8 + ql) << 2)) = r4;
    }
    __syncwarp();
    if (live) {
      update_slot(0, 4 * g, yes, yes);
      update_slot(1, 4 * g + 1, yes, yes);
      update_slot(2, 4 * g + 2, yes, no);
      update_slot(3, 4 * g + 3, no, no);
    }
    __syncwarp();
    ++g;
  }
  // the last groups, slot by slot (the first of them has its call made by
  // the loop above when that ran)
  for (bool made = g > 0; 4 * g < n; ++g, made = false) {
    if (live && 4 * g + j < n) {
      if (!made)
        r4 = philox(make_uint4(z[0], (uint32_t)t, (uint32_t)(4 * g + j) | ((uint32_t)q << 16), ctr_w), p.key);
      *reinterpret_cast<uint4 *>(rw + ((j * 8 + ql) << 2)) = r4;
    }
    __syncwarp();
    if (live) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int sl = 4 * g + i;
        if (sl >= n) break;
        // words of slot sl after the exchanges of pairs 0 .. sl
        uint32_t fw[7];
        if (sl + 1 < n) {
          uint32_t n2[7] = {0, 0, 0, 0, 0, 0, 0};
          if (sl + 2 < n) {
            const uint32_t *ps = sb + (int64_t)(sl + 2) * SS;
#pragma unroll
            for (int k = 0; k < 7; ++k) n2[k] = ps[zo[k]];
          }
          const uint32_t m = msk[j][sl];
#pragma unroll
          for (int k = 0; k < 7; ++k) {
            const uint32_t xx = (cw[k] ^ n1[k]) & m;
            fw[k] = cw[k] ^ xx;
            cw[k] = n1[k] ^ xx;
            n1[k] = n2[k];
          }
        } else {
#pragma unroll
          for (int k = 0; k < 7; ++k) fw[k] = cw[k];
        }
        const uint32_t R = rw[((i * 8 + ql) << 2) + j];
        const unsigned long long *C = thr[sl];
        const uint32_t sc = fw[0];
        const uint32_t b1 = sc ^ fw[3] ^ Jxp;
        const uint32_t b2 = sc ^ fw[4] ^ Jxm;
        const uint32_t b3 = sc ^ fw[5] ^ Jyp;
        const uint32_t b4 = sc ^ fw[6] ^ Jym;
        const uint32_t t1 = sc ^ fw[1] ^ gtp;
        const uint32_t t2 = sc ^ fw[2] ^ gtm;
        const uint32_t s1 = b1 ^ b2 ^ b3;
        const uint32_t c1 = maj3(b1, b2, b3);
        const uint32_t us0 = s1 ^ b4;
        const uint32_t c2 = s1 & b4;
        const uint32_t us1 = c1 ^ c2;
        const uint32_t us2 = c1 & c2;
        const uint32_t ut0 = t1 ^ t2;
        const uint32_t ut1 = t1 & t2;
        const uint32_t acc = accept_mask(R, C, us0, us1, us2, ut0, ut1, p.one);
        uint32_t *pd = db + (int64_t)sl * SS;
        pd[zo[0]] = sc ^ acc;
        pd[zo[1]] = fw[1];
      }
    }
    __syncwarp();
  }
}

// The same pass with one thread per red site and RP of its four replicas
// (RP = 4: the site's 16-byte replica quad; RP = 2: two threads per site,
// 8 bytes each, sharing the Philox calls of the quad's draws through a
// shuffle: the even thread draws even slots, the odd thread odd ones).
// Fewer threads and instructions per word than the per-replica form; the
// autotuner picks the form (results are identical).
template <typename Word, int RP, bool CG = false>
__device__ __forceinline__ void ld_rp(Word (&d)[RP], const Word *p) {
  if constexpr (RP * sizeof(Word) == 16) {
    const uint4 v = ld_g<CG>(reinterpret_cast<const uint4 *>(p));
    memcpy(d, &v, 16);
  } else if constexpr (RP * sizeof(Word) == 8) {
    const uint2 v = ld_g<CG>(reinterpret_cast<const uint2 *>(p));
    memcpy(d, &v, 8);
  } else {
    d[0] = ld_g<CG>(p);
  }
}
template <typename Word, int RP>
__device__ __forceinline__ void st_rp(Word *p, const Word (&d)[RP]) {
  if constexpr (RP * sizeof(Word) == 16) {
    uint4 v;
    memcpy(&v, d, 16);
    *reinterpret_cast<uint4 *>(p) = v;
  } else if constexpr (RP * sizeof(Word) == 8) {
    uint2 v;
    memcpy(&v, d, 8);
    *reinterpret_cast<uint2 *>(p) = v;
  } else {
    *p = d[0];
  }
}

// Red pass with the pending PT exchanges (as above) for either word width,
// one thread per red site and RP of its four replicas (TPS = 4 / RP threads
// per site, consecutive lanes).  The site's Philox calls (one per slot, four
// draws) are spread over its threads: thread h makes the call of slot
// TPS g + h and the draws are passed on by shuffles.
// Body of the pass for (virtual) block bid of sweep t; CG: read what other
// blocks of a persistent launch wrote (spins, masks) through L2 only.
template <typename Word, int RP, bool CG>
__device__ __forceinline__ void red_fusedq_body(const FusedRedArgsT<Word> &p, const SlotThresholds &th, uint32_t bid,
                                                unsigned long long t) {
  constexpr int TPS = 4 / RP;
  constexpr int W = (int)sizeof(Word) * 8;
  __shared__ __align__(16) Word msk[kMaxSlotsPT][4];
  const uint32_t set = p.fd_bps.div(bid);   // (b, q)
  const uint32_t chunk = bid - set * (uint32_t)p.blocks_per_set;
  const uint32_t b = p.fd_nq.div(set);
  const int q = (int)(set - b * (uint32_t)p.n_q);
  const int n = p.n_slots;
  __syncthreads();   // msk of the previous (virtual) block is no longer read

  const uint32_t tid = chunk * (uint32_t)kBlock4 + threadIdx.x;
  const int h = (int)(tid % TPS);                 // which replica group of the site
  const uint32_t quad = tid / TPS;                // red site of the (b, q) set
  const uint32_t P = (uint32_t)p.plane, Lt = (uint32_t)p.Lt, L = (uint32_t)p.L;
  const bool live = quad < P * (Lt / 2);          // uniform over a site's threads
  const uint32_t seg = p.fd_plane.div(quad);
  const uint32_t i2 = quad - seg * P;
  const uint32_t y = p.fd_L.div(i2), x = i2 - y * L;
  const uint32_t tau = 2 * seg + ((x + y) & 1u);
  const uint32_t ixp = (x + 1 == L ? 0 : x + 1) + L * y, ixm = (x == 0 ? L - 1 : x - 1) + L * y;
  const uint32_t iyp = x + L * (y + 1 == L ? 0 : y + 1), iym = x + L * (y == 0 ? L - 1 : y - 1);
  const uint32_t off = tau * P;
  // the antiperiodic wrap bond is unsatisfied when its spins agree
  const Word gtp = ones_if<Word>(p.tau_ap && tau + 1 == Lt), gtm = ones_if<Word>(p.tau_ap && tau == 0);
  uint32_t zo[7];   // word offsets of the seven sites' replica groups
  {
    uint32_t z[7];
    z[0] = i2 + off;
    z[1] = i2 + (tau + 1 == Lt ? 0u : off + P);
    z[2] = i2 + (tau == 0 ? (Lt - 1) * P : off - P);
    z[3] = ixp + off;
    z[4] = ixm + off;
    z[5] = iyp + off;
    z[6] = iym + off;
#pragma unroll
    for (int k = 0; k < 7; ++k) zo[k] = 4 * z[k] + (uint32_t)(RP * h);
  }
  const int64_t base = (((int64_t)b * n * p.n_q + q) * p.N) * 4;
  const int64_t SS = (int64_t)p.n_q * p.N * 4;
  const Word *sb = p.src + base;
  Word *db = p.dst + base;
  const Word *Jb = p.J + (int64_t)b * P * 2;
  Word Jxp = 0, Jxm = 0, Jyp = 0, Jym = 0;
  const uint32_t ctr_w = (DOM_SWEEP << 28) | ((b * (uint32_t)W) >> 6);
  const uint32_t site = i2 + off;
  const int lane = (int)(threadIdx.x & 31), lane0 = lane & ~(TPS - 1);
  Word cw[7][RP], n1[7][RP];
  if (live) {
    Jxp = Jb[2 * i2];
    Jxm = Jb[2 * ixm];
    Jyp = Jb[2 * i2 + 1];
    Jym = Jb[2 * iym + 1];
#pragma unroll
    for (int k = 0; k < 7; ++k) ld_rp<Word, RP, CG>(cw[k], sb + zo[k]);
    if (n > 1)
#pragma unroll
      for (int k = 0; k < 7; ++k) ld_rp<Word, RP, CG>(n1[k], sb + SS + zo[k]);
  }
  // the PT masks of the (b, q) set, staged after the first slots' loads are
  // issued, so the two round trips to L2 overlap
  for (int i = threadIdx.x; i < 4 * kMaxSlotsPT; i += blockDim.x) {
    const int sl = i >> 2, jj = i & 3;
    const int rr = 4 * q + jj;
    msk[sl][jj] = (rr < p.n_rep && sl + 1 < n) ? ld_g<CG>(p.acc + ((int64_t)b * p.n_rep + rr) * n + sl) : Word(0);
  }
  __syncthreads();
  uint4 R4 = make_uint4(0, 0, 0, 0);
  const uint32_t wbytes = p.one * (uint32_t)sizeof(Word);   // the runtime element size (addr_scaled)
  // slot sl: its draws, the words of slot sl after the exchanges of pairs
  // 0 .. sl, the update of the red site and the stores; H1 / H2: slot sl + 1
  // / sl + 2 exists (known at compile time, so the slot has no checks)
  auto step = [&](const int sl, auto has1, auto has2) {
    constexpr bool H1 = decltype(has1)::value, H2 = decltype(has2)::value;
    const int i = sl % TPS;   // thread i of the site holds slot sl's call
    if (i == 0) {
      const int sm = sl + h;
      if (live && sm < n) R4 = philox(make_uint4(site, (uint32_t)t, (uint32_t)sm | ((uint32_t)q << 16), ctr_w), p.key);
    }
    uint32_t Rj[RP];
    if constexpr (TPS == 1) {
      Rj[0] = R4.x; Rj[1] = R4.y; Rj[2] = R4.z; Rj[3] = R4.w;
    } else if constexpr (TPS == 2) {
      // the owner passes the partner's two components
      const uint32_t give0 = (i == h) ? (h ? R4.x : R4.z) : 0u;
      const uint32_t give1 = (i == h) ? (h ? R4.y : R4.w) : 0u;
      const uint32_t got0 = __shfl_xor_sync(0xffffffffu, give0, 1);
      const uint32_t got1 = __shfl_xor_sync(0xffffffffu, give1, 1);
      Rj[0] = (i == h) ? (h ? R4.z : R4.x) : got0;
      Rj[1] = (i == h) ? (h ? R4.w : R4.y) : got1;
    } else {
      const uint32_t v0 = __shfl_sync(0xffffffffu, R4.x, lane0 + i);
      const uint32_t v1 = __shfl_sync(0xffffffffu, R4.y, lane0 + i);
      const uint32_t v2 = __shfl_sync(0xffffffffu, R4.z, lane0 + i);
      const uint32_t v3 = __shfl_sync(0xffffffffu, R4.w, lane0 + i);
      Rj[0] = h == 0 ? v0 : h == 1 ? v1 : h == 2 ? v2 : v3;
    }
    if (!live) return;
    Word fw[7][RP];
    if constexpr (H1) {
      Word n2[7][RP];
      if constexpr (H2) {
        const Word *ps = sb + (int64_t)(sl + 2) * SS;
#pragma unroll
        for (int k = 0; k < 7; ++k) ld_rp<Word, RP, CG>(n2[k], addr_scaled(ps, zo[k], wbytes));
      }
      Word m[RP];
#pragma unroll
      for (int jj = 0; jj < RP; ++jj) m[jj] = msk[sl][RP * h + jj];
#pragma unroll
      for (int k = 0; k < 7; ++k)
#pragma unroll
        for (int jj = 0; jj < RP; ++jj) {   // lanes of m exchange pair (sl, sl + 1)
          fw[k][jj] = mux(m[jj], n1[k][jj], cw[k][jj]);
          cw[k][jj] = mux(m[jj], cw[k][jj], n1[k][jj]);
          if constexpr (H2) n1[k][jj] = n2[k][jj];
        }
    } else {
#pragma unroll
      for (int k = 0; k < 7; ++k)
#pragma unroll
        for (int jj = 0; jj < RP; ++jj) fw[k][jj] = cw[k][jj];
    }
    const unsigned long long *C = th.v[sl];
    Word out[RP];
#pragma unroll
    for (int jj = 0; jj < RP; ++jj) {
      const Word sc = fw[0][jj];
      const Word b1 = sc ^ fw[3][jj] ^ Jxp;
      const Word b2 = sc ^ fw[4][jj] ^ Jxm;
      const Word b3 = sc ^ fw[5][jj] ^ Jyp;
      const Word b4 = sc ^ fw[6][jj] ^ Jym;
      const Word t1 = sc ^ fw[1][jj] ^ gtp;
      const Word t2 = sc ^ fw[2][jj] ^ gtm;
      const Word s1 = b1 ^ b2 ^ b3;
      const Word c1 = maj3(b1, b2, b3);
      const Word us0 = s1 ^ b4;
      const Word c2 = s1 & b4;
      const Word us1 = c1 ^ c2;
      const Word us2 = c1 & c2;
      const Word ut0 = t1 ^ t2;
      const Word ut1 = t1 & t2;
      out[jj] = sc ^ accept_word<Word>(Rj[jj], C, us0, us1, us2, ut0, ut1, p.one);
    }
    Word *pd = db + (int64_t)sl * SS;
    st_rp<Word, RP>(addr_scaled(pd, zo[0], wbytes), out);
    st_rp<Word, RP>(addr_scaled(pd, zo[1], wbytes), fw[1]);
  };
  const std::integral_constant<bool, true> yes;
  const std::integral_constant<bool, false> no;
  int sl = 0;
  for (; sl + 2 < n; ++sl) step(sl, yes, yes);   // slots with two successors
  if (sl + 1 < n) step(sl++, yes, no);
  if (sl < n) step(sl, no, no);
}

template <typename Word, int RP>
__global__ void __launch_bounds__(kBlock4) samples_red_fusedq_kernel(const FusedRedArgsT<Word> p,
                                                                      const __grid_constant__ SlotThresholds th) {
  pdl_begin();
  {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p.n_zero_U; i += stride) p.zero_U[i] = 0;
    if (p.ticket && blockIdx.x == 0 && threadIdx.x == 0) *p.ticket = 0u;
  }
  red_fusedq_body<Word, RP, false>(p, th, blockIdx.x, *p.d_t);
}

// Sum the block's per-thread counters (NC counters of K planes in registers)
// and add lane l of counter c into out[c * 32 + l]: tree over the 128
// threads in shared memory, one more plane per level.
template <int K, int NC, typename Word = uint32_t>
__device__ __forceinline__ void block_sum_counters(const VCount<Word, K> *cnt, Word *buf, int *out) {
  constexpr int KF = K + kLog2Block4;
  constexpr int W = (int)sizeof(Word) * 8;
  const int tid = threadIdx.x;
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int i = 0; i < K; ++i) buf[(c * KF + i) * kBlock4 + tid] = cnt[c].p[i];
  __syncthreads();
#pragma unroll
  for (int lvl = 0; lvl < kLog2Block4; ++lvl) {
    const int half = kBlock4 >> (lvl + 1);
    for (int w = tid; w < NC * half; w += kBlock4) {
      const int c = w / half, e = w - c * half;
      Word *a = buf + (size_t)c * KF * kBlock4 + e;
      Word carry = 0;
#pragma unroll
      for (int i = 0; i < K + lvl; ++i) {
        const Word x = a[i * kBlock4], y = a[i * kBlock4 + half];
        a[i * kBlock4] = x ^ y ^ carry;
        carry = maj3(x, y, carry);
      }
      a[(K + lvl) * kBlock4] = carry;
    }
    __syncthreads();
  }
  for (int w = tid; w < NC * W; w += kBlock4) {
    const int c = w / W, l = w - c * W;
    int v = 0;
#pragma unroll
    for (int i = 0; i < KF; ++i) v |= (int)((buf[(c * KF + i) * kBlock4] >> l) & 1u) << i;
    out[w] = v;
  }
  __syncthreads();   // buf is reused by the caller
}

// Body of the pass for (virtual) block bid of sweep t; CG: read the spins
// through L2 only (a persistent launch, where other blocks wrote them).
// KS: counter planes of a thread's u_s sum (at most 4 G, so KS =
// counter_planes(G)); the u_t sum (at most 2 G) takes one plane less.
template <bool BLUE, int KS, bool PF, bool CG>
__device__ __forceinline__ void sweep4_body(const SamplesArgs<uint32_t> &p, const SlotThresholds &th, uint32_t bid,
                                            unsigned long long t, int colour, int count_only) {
  constexpr int KT = KS - 1;
  constexpr int KF = KS + kLog2Block4;
  __shared__ uint32_t buf[BLUE ? 4 * KF * kBlock4 : 1];
  __shared__ int tot[BLUE ? 2 * 4 * 32 : 1];

  // block -> (b, s, q, chunk) and thread -> (segment, column) in 32 bits
  const uint32_t set = p.fd_bps.div(bid);
  const uint32_t chunk = bid - set * (uint32_t)p.blocks_per_set;
  const uint32_t bs = p.fd_nq.div(set);
  const int q = (int)(set - bs * (uint32_t)p.n_q);
  const uint32_t b = p.fd_ns.div(bs);
  const int s = (int)(bs - b * (uint32_t)p.n_slots);
  const unsigned long long *C = th.v[s];
  const int L = p.L, plane = p.plane;
  const uint32_t Lt = (uint32_t)p.Lt, P = (uint32_t)plane;
  // segment segu and column i2 of the thread; segb is the block's segment
  // when a block holds one segment (else 0, with seg_rem = 0), so the walk
  // length G is the same for the whole block
  uint32_t segu, segb, i2u;
  bool live;
  if (p.seg_blocks) {
    segb = p.fd_sb.div(chunk);
    segu = segb;
    i2u = (chunk - segb * (uint32_t)p.seg_blocks) * (uint32_t)kBlock4 + threadIdx.x;
    live = i2u < P;
  } else {
    const uint32_t gq = chunk * (uint32_t)kBlock4 + threadIdx.x;
    live = gq < P * (uint32_t)p.n_seg;
    segu = p.fd_plane.div(gq);
    segb = 0;
    i2u = gq - segu * P;
  }
  const int i2 = (int)i2u;
  const int y = (int)p.fd_L.div((uint32_t)i2), x = i2 - y * L;
  const int ixp = (x + 1 == L ? 0 : x + 1) + L * y, ixm = (x == 0 ? L - 1 : x - 1) + L * y;
  const int iyp = x + L * (y + 1 == L ? 0 : y + 1), iym = x + L * (y == 0 ? L - 1 : y - 1);
  const uint4 *src = reinterpret_cast<const uint4 *>(p.spins) + ((b * p.n_slots + s) * p.n_q + q) * p.N;
  const uint4 *pc = src + i2, *pxp = src + ixp, *pxm = src + ixm, *pyp = src + iyp, *pym = src + iym;
  uint4 *wc = reinterpret_cast<uint4 *>(p.spins) + ((b * p.n_slots + s) * p.n_q + q) * p.N + i2;
  const uint32_t *Jb = p.J + b * (int64_t)plane * 2;
  uint32_t Jxp = 0, Jxm = 0, Jyp = 0, Jym = 0;
  const uint32_t tau0 = 2u * (segu * (uint32_t)p.seg_base + min(segu, (uint32_t)p.seg_rem)) +
                        (uint32_t)((colour + x + y) & 1);
  const int G = p.seg_base + (segb < (uint32_t)p.seg_rem ? 1 : 0);
  const uint32_t ctr_z = (uint32_t)s | ((uint32_t)q << 16);
  const uint32_t ctr_w = (DOM_SWEEP << 28) | (uint32_t)((b * 32) >> 6);

  VCount<uint32_t, KS> cs[4];
  VCount<uint32_t, KT> ct[4];
  if (BLUE)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      cs[j].zero();
      ct[j].zero();
    }

  if (live) {
    Jxp = Jb[2 * i2];
    Jxm = Jb[2 * ixm];
    Jyp = Jb[2 * i2 + 1];
    Jym = Jb[2 * iym + 1];
    uint32_t off = tau0 * P;
    uint4 dn = ld_g<CG>(pc + (size_t)(tau0 == 0 ? (Lt - 1) * P : off - P));
    Quad4 cur;
    cur.c = ld_g<CG>(pc + off);
    cur.up = ld_g<CG>(pc + (size_t)(tau0 + 1 == Lt ? 0u : off + P));
    cur.xp = ld_g<CG>(pxp + off);
    cur.xm = ld_g<CG>(pxm + off);
    cur.yp = ld_g<CG>(pyp + off);
    cur.ym = ld_g<CG>(pym + off);
    uint4 R4 = philox(make_uint4((uint32_t)i2 + off, (uint32_t)t, ctr_z, ctr_w), p.key);
    // the even site's post-flip counts, held until the odd site's are added
    // with them (the prefetching walk of the per-pass launch)
    uint32_t h0[4], h1[4], h2[4], g0[4], g1[4];
    // site k of the walk, its words in cu; with the prefetch the next site's
    // words go to nx while this one is updated, else to cu after it.  PH: 0
    // hold this site's counts, 1 add them with the held ones, 2 add them
    auto site = [&](int k, Quad4 &cu, Quad4 &nx, auto phase) {
      constexpr int PH = decltype(phase)::value;
      const uint32_t tau = tau0 + 2u * (uint32_t)k;
      // the draws of the walk's next site are made while this one is
      // updated, so the Philox chain overlaps independent work
      uint4 R4n = R4;
      if (k + 1 < G) R4n = philox(make_uint4((uint32_t)i2 + off + 2 * P, (uint32_t)t, ctr_z, ctr_w), p.key);
      auto load_next = [&](Quad4 &q) {
        const uint32_t offn = off + 2 * P;
        q.c = ld_g<CG>(pc + offn);
        q.up = ld_g<CG>(pc + (size_t)(tau + 3 == Lt ? 0u : offn + P));
        q.xp = ld_g<CG>(pxp + offn);
        q.xm = ld_g<CG>(pxm + offn);
        q.yp = ld_g<CG>(pyp + offn);
        q.ym = ld_g<CG>(pym + offn);
      };
      if (PF && k + 1 < G) load_next(nx);
      // the antiperiodic wrap bond is unsatisfied when its spins agree
      const uint32_t gtp = ones_if<uint32_t>(p.tau_ap && tau + 1 == Lt), gtm = ones_if<uint32_t>(p.tau_ap && tau == 0);
      uint32_t f[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t sc = q4(cu.c, j);
        const uint32_t b1 = sc ^ q4(cu.xp, j) ^ Jxp;
        const uint32_t b2 = sc ^ q4(cu.xm, j) ^ Jxm;
        const uint32_t b3 = sc ^ q4(cu.yp, j) ^ Jyp;
        const uint32_t b4 = sc ^ q4(cu.ym, j) ^ Jym;
        const uint32_t t1 = sc ^ q4(cu.up, j) ^ gtp;
        const uint32_t t2 = sc ^ q4(dn, j) ^ gtm;
        const uint32_t s1 = b1 ^ b2 ^ b3;
        const uint32_t c1 = maj3(b1, b2, b3);
        const uint32_t us0 = s1 ^ b4;
        const uint32_t c2 = s1 & b4;
        const uint32_t us1 = c1 ^ c2;
        const uint32_t us2 = c1 & c2;
        const uint32_t ut0 = t1 ^ t2;
        const uint32_t ut1 = t1 & t2;
        const uint32_t flip = count_only ? 0u : accept_mask(q4(R4, j), C, us0, us1, us2, ut0, ut1, p.one);
        f[j] = flip;
        if (BLUE) {
          // unsatisfied counts after the flip: u -> 4 - u (spatial), 2 - u (tau)
          const uint32_t vs1 = us1 ^ (flip & us0);
          const uint32_t vs2 = mux(flip, ~(us0 | us1 | us2), us2);
          const uint32_t vt1 = mux(flip, ~(ut0 | ut1), ut1);
          if constexpr (PH == 0) {
            h0[j] = us0;
            h1[j] = vs1;
            h2[j] = vs2;
            g0[j] = ut0;
            g1[j] = vt1;
          } else if constexpr (PH == 1) {
            cs[j].add3x2(h0[j], h1[j], h2[j], us0, vs1, vs2);
            ct[j].add2x2(g0[j], g1[j], ut0, vt1);
          } else {
            cs[j].add3(us0, vs1, vs2);
            ct[j].add2(ut0, vt1);
          }
        }
      }
      if (!count_only) wc[off] = make_uint4(cu.c.x ^ f[0], cu.c.y ^ f[1], cu.c.z ^ f[2], cu.c.w ^ f[3]);
      R4 = R4n;
      dn = cu.up;
      if (!PF && k + 1 < G) load_next(nx);
      off += 2 * P;
    };
    using Hold = std::integral_constant<int, 0>;
    using Pair = std::integral_constant<int, 1>;
    using One = std::integral_constant<int, 2>;
    if constexpr (BLUE && PF && !CG) {
      // two sites per iteration: the current and next sites' words swap
      // registers instead of being copied, and their counts enter the
      // counters together (not in the persistent kernel, whose register
      // bound would make this walk spill)
      Quad4 nxt;
      int k = 0;
      for (; k + 1 < G; k += 2) {
        site(k, cur, nxt, Hold{});
        site(k + 1, nxt, cur, Pair{});
      }
      if (k < G) site(k, cur, nxt, One{});
    } else if constexpr (PF) {
      Quad4 nxt;
#pragma unroll 1
      for (int k = 0; k < G; ++k) {
        site(k, cur, nxt, One{});
        if (k + 1 < G) cur = nxt;
      }
    } else {
#pragma unroll 1
      for (int k = 0; k < G; ++k) site(k, cur, cur, One{});
    }
  }

  if (BLUE) {
    block_sum_counters<KS, 4>(cs, buf, tot);
    block_sum_counters<KT, 4>(ct, buf, tot + 4 * 32);
    {
      const int w = threadIdx.x;   // 128 = 4 replicas x 32 lanes
      const int jj = w >> 5, lane = w & 31;
      const int rr = 4 * q + jj;
      const int64_t a = b * 32 + lane;
      if (rr < p.n_rep) {
        unsigned long long *u = p.U + ((a * p.n_rep + rr) * p.n_slots + s) * 2;
        if (tot[w]) atomicAdd(u, (unsigned long long)tot[w]);
        if (tot[4 * 32 + w]) atomicAdd(u + 1, (unsigned long long)tot[4 * 32 + w]);
      }
    }
  }
}


// The PT pass in the blue pass's last blocks (fused mode, 32-bit words; Sec.
// 2.1's PT update after the sweep).  Instead of a separate PT launch, each
// block of the blue pass takes a ticket once its bond counts are added; the
// last P blocks to take one wait (bounded by wait_ns, error flag on expiry)
// until every block has, then run the chains of the sweep, a warp per chain,
// exactly as the PT kernel does, and the block with the last ticket advances
// the sweep counter.  Only the last P blocks wait, so the blocks not yet
// started always find room on the SMs (P is at most half the grid and half
// the resident blocks).
struct PTFold {
  int P;                         // PT blocks of this launch (0: no PT here)
  unsigned *ticket;              // blocks done; the red pass resets it
  int32_t *walker;
  unsigned long long *U;
  uint32_t *acc;
  const PTConst *ptc;
  const double *sq;
  unsigned long long *d_t;
  int *err;
  long long wait_ns;
  int64_t n_samples;
  int n_rep, n_slots;
};

__device__ __forceinline__ void pt_in_blue_tail(const PTFold &f, uint2 key, unsigned long long t) {
  __shared__ unsigned s_tk;
  __shared__ int s_go;
  __syncthreads();   // every bond-count atomic of this block is issued
  if (threadIdx.x == 0) {
    __threadfence();
    s_tk = atomicAdd(f.ticket, 1u);
  }
  __syncthreads();
  const unsigned nb = gridDim.x, tk = s_tk;
  if (tk + (unsigned)f.P < nb) return;   // not among the last P blocks
  if (threadIdx.x == 0) {
    int go = 1;
    const unsigned long long t0 = gtime();
    while (*(volatile unsigned *)f.ticket < nb) {
      if (*(volatile int *)f.err) {
        go = 0;
        break;
      }
      if (gtime() - t0 > (unsigned long long)f.wait_ns) {
        atomicExch(f.err, 1);
        go = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_go = go;
  }
  __syncthreads();
  if (!s_go) return;
  constexpr int kWarps = kBlock4 / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n_chains = f.n_samples * f.n_rep;
  for (int64_t c = (int64_t)(tk - (nb - (unsigned)f.P)) * kWarps + warp; c < n_chains; c += (int64_t)f.P * kWarps) {
    const int64_t sa = c / f.n_rep;   // c is uniform over the warp
    const int r = (int)(c - sa * f.n_rep);
    const uint32_t acc = pt_chain<true, true, false>(f.walker + c * f.n_slots, f.U + c * f.n_slots * 2, f.ptc, f.sq,
                                                     key, (uint32_t)t, sa, r, f.n_slots);
    if (lane + 1 < f.n_slots && ((acc >> lane) & 1u))
      atomicOr(f.acc + ((sa >> 5) * f.n_rep + r) * f.n_slots + lane, 1u << (sa & 31));
  }
  if (tk == nb - 1 && threadIdx.x == 0) *f.d_t = t + 1;   // every block read t at its start
}

template <bool BLUE, int KS, bool PF, int MINB = 0>
__global__ void __launch_bounds__(kBlock4, MINB) samples_sweep4_kernel(SamplesArgs<uint32_t> p,
                                                                  const __grid_constant__ SlotThresholds th,
                                                                  int colour, int count_only, const PTFold f) {
  pdl_begin();
  {   // counters / masks the host asked this pass to clear (nothing reads them before the next pass)
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p.n_zero_U; i += stride) p.zero_U[i] = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p.n_zero_acc; i += stride)
      p.zero_acc[i] = 0;
  }
  const unsigned long long t = *p.d_t;
  if (p.t_copy && blockIdx.x == 0 && threadIdx.x == 0) *p.t_copy = t;
  sweep4_body<BLUE, KS, PF, false>(p, th, blockIdx.x, t, colour, count_only);
  if (BLUE && f.P > 0) pt_in_blue_tail(f, p.key, t);
}


// Apply the PT pass to the spins: for pair s = 0 .. n_slots-2 in order,
// exchange the bits of accepting lanes between slot words s and s+1.
// With advance set, block 0 also advances the sweep counter (nothing in this
// kernel reads it), saving the separate launch at the end of the sweep.
template <typename Word>
__global__ void __launch_bounds__(kBlock) samples_permute_kernel(Word *spins, const Word *acc, int64_t N,
                                                                 int n_slots, int n_q, int n_rep,
                                                                 int blocks_per_set,
                                                                 unsigned long long *advance) {
  pdl_begin();
  __shared__ Word accs[4 * kMaxSlotsPermute];
  __shared__ int any;
  if (advance && blockIdx.x == 0 && threadIdx.x == 0) *advance += 1ull;
  const int64_t set = blockIdx.x / blocks_per_set;     // (b, q)
  const int chunk = (int)(blockIdx.x - set * blocks_per_set);
  const int q = (int)(set % n_q);
  const int64_t b = set / n_q;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * n_slots; i += blockDim.x) {
    const int jj = i / n_slots, s = i - jj * n_slots;
    const int rr = 4 * q + jj;
    const Word m = (rr < n_rep && s + 1 < n_slots) ? acc[(b * n_rep + rr) * n_slots + s] : Word(0);
    accs[jj * kMaxSlotsPermute + s] = m;
    if (m) any = 1;
  }
  __syncthreads();
  if (!any) return;   // no exchange in this (b, q): nothing moves
  const int64_t idx = (int64_t)chunk * blockDim.x + threadIdx.x;   // (site, j)
  if (idx >= N * 4) return;
  const int jj = (int)(idx & 3);
  const int64_t stride = (int64_t)n_q * N * 4;
  Word *w0 = spins + ((b * n_slots) * n_q + q) * N * 4 + idx;
  Word w[kMaxSlotsPermute];
#pragma unroll
  for (int s = 0; s < kMaxSlotsPermute; ++s)
    if (s < n_slots) w[s] = w0[s * stride];
#pragma unroll
  for (int s = 0; s + 1 < kMaxSlotsPermute; ++s)
    if (s + 1 < n_slots) {
      const Word x = (w[s] ^ w[s + 1]) & accs[jj * kMaxSlotsPermute + s];
      w[s] ^= x;
      w[s + 1] ^= x;
    }
#pragma unroll
  for (int s = 0; s < kMaxSlotsPermute; ++s)
    if (s < n_slots) w0[s * stride] = w[s];
}

// W = 32 form of the same: thread per site, the site's 4 replica words as
// one 16-byte word per slot, NS >= n_slots slot words held in registers.
template <int NS>
__global__ void __launch_bounds__(kBlock4) samples_permute4_kernel(uint4 *spins, const uint32_t *acc, int64_t N,
                                                                    int n_slots, int n_q, int n_rep,
                                                                    int blocks_per_set,
                                                                    unsigned long long *advance) {
  pdl_begin();
  __shared__ uint32_t msk[4][NS];
  if (advance && blockIdx.x == 0 && threadIdx.x == 0) *advance += 1ull;
  const int64_t set = blockIdx.x / blocks_per_set;     // (b, q)
  const int chunk = (int)(blockIdx.x - set * blocks_per_set);
  const int q = (int)(set % n_q);
  const int64_t b = set / n_q;
  for (int i = threadIdx.x; i < 4 * NS; i += blockDim.x) {
    const int jj = i / NS, s = i - jj * NS;
    const int rr = 4 * q + jj;
    msk[jj][s] = (rr < n_rep && s + 1 < n_slots) ? acc[(b * n_rep + rr) * n_slots + s] : 0u;
  }
  __syncthreads();
  const int64_t site = (int64_t)chunk * kBlock4 + threadIdx.x;
  if (site >= N) return;
  const int64_t stride = (int64_t)n_q * N;
  uint4 *w0 = spins + ((b * n_slots) * n_q + q) * N + site;
  uint4 w[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s)
    if (s < n_slots) w[s] = w0[s * stride];
#pragma unroll
  for (int s = 0; s + 1 < NS; ++s)
    if (s + 1 < n_slots) {
      uint32_t x;
      x = (w[s].x ^ w[s + 1].x) & msk[0][s]; w[s].x ^= x; w[s + 1].x ^= x;
      x = (w[s].y ^ w[s + 1].y) & msk[1][s]; w[s].y ^= x; w[s + 1].y ^= x;
      x = (w[s].z ^ w[s + 1].z) & msk[2][s]; w[s].z ^= x; w[s + 1].z ^= x;
      x = (w[s].w ^ w[s + 1].w) & msk[3][s]; w[s].w ^= x; w[s + 1].w ^= x;
    }
#pragma unroll
  for (int s = 0; s < NS; ++s)
    if (s < n_slots) w0[s * stride] = w[s];
}

// Overlaps (Appendix E.1) of every replica pair at one slot, for up to 4
// replicas (one replica quad): a thread reads the quad of G sites of one
// (b, s) once and counts, per pair, the sites where the two configurations
// differ (per lane, bit-sliced); the block sums its threads' counters (tree
// in shared memory, in two batches of three pairs) and adds lane a's counts
// into qcnt[a][s][p].  Pairs p in the order (0,1), (0,2), (0,3), (1,2),
// (1,3), (2,3) restricted to the replicas present.
template <typename Word, int K>
__global__ void __launch_bounds__(kBlock4) samples_overlap4_kernel(const Word *spins, long long *qcnt, int64_t N,
                                                                    int n_slots, int n_rep, int64_t n_samples,
                                                                    int sites_per_thread, int blocks_per_set) {
  pdl_begin();
  constexpr int W = (int)sizeof(Word) * 8;
  constexpr int KF = K + kLog2Block4;
  __shared__ Word buf[3 * KF * kBlock4];
  __shared__ int tot[6 * W];
  const int64_t set = blockIdx.x / blocks_per_set;   // (b, s)
  const int chunk = (int)(blockIdx.x - set * blocks_per_set);
  const int s = (int)(set % n_slots);
  const int64_t b = set / n_slots;
  const Word *w0 = spins + (b * n_slots + s) * N * 4;   // n_q = 1
  VCount<Word, K> c[6];
#pragma unroll
  for (int p = 0; p < 6; ++p) c[p].zero();
  const int64_t start = (int64_t)chunk * kBlock4 * sites_per_thread + threadIdx.x;
  // four sites at a time: per pair, the four difference bits are compressed
  // to a 3-bit count (a full and two half adders) and added at once
  for (int k = 0; k < sites_per_thread; k += 4) {
    Word d[4][6];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t site = start + (int64_t)(k + u) * kBlock4;
      Word r[4] = {0, 0, 0, 0};
      if (k + u < sites_per_thread && site < N) {
        if constexpr (sizeof(Word) == 4) {
          const uint4 v = reinterpret_cast<const uint4 *>(w0)[site];
          r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
        } else {
          const ulonglong2 v0 = reinterpret_cast<const ulonglong2 *>(w0)[2 * site];
          const ulonglong2 v1 = reinterpret_cast<const ulonglong2 *>(w0)[2 * site + 1];
          r[0] = v0.x; r[1] = v0.y; r[2] = v1.x; r[3] = v1.y;
        }
      }
      d[u][0] = r[0] ^ r[1];
      d[u][1] = r[0] ^ r[2];
      d[u][2] = r[0] ^ r[3];
      d[u][3] = r[1] ^ r[2];
      d[u][4] = r[1] ^ r[3];
      d[u][5] = r[2] ^ r[3];
    }
#pragma unroll
    for (int pp = 0; pp < 6; ++pp) {
      const Word s1 = d[0][pp] ^ d[1][pp] ^ d[2][pp];
      const Word c1 = maj3(d[0][pp], d[1][pp], d[2][pp]);
      const Word b0 = s1 ^ d[3][pp];
      const Word c2 = s1 & d[3][pp];
      c[pp].add3(b0, c1 ^ c2, c1 & c2);
    }
  }
  block_sum_counters<K, 3, Word>(c, buf, tot);
  block_sum_counters<K, 3, Word>(c + 3, buf, tot + 3 * W);
  // the pair index of (x, y) among the replicas present
  const int n_pairs = n_rep * (n_rep - 1) / 2;
  for (int w = threadIdx.x; w < 6 * W; w += blockDim.x) {
    const int pp = w / W, lane = (int)(w - pp * W);
    const int x = pp < 3 ? 0 : pp < 5 ? 1 : 2;
    const int y = pp < 3 ? pp + 1 : pp < 5 ? pp - 1 : 3;
    if (y >= n_rep || !tot[w]) continue;
    const int p = x * n_rep - x * (x + 1) / 2 + (y - x - 1);
    const int64_t a = b * W + lane;
    if (a < n_samples) atomicAdd(reinterpret_cast<unsigned long long *>(&qcnt[(a * n_slots + s) * n_pairs + p]),
                                 (unsigned long long)tot[w]);
  }
}

// Measurement sums (Appendix E.1): one thread per (sample, slot) and item,
// items = the replicas' (A, B) then the pairs' q = N - 2 (differing sites);
// to_q_only only converts the counts to q.
__global__ void samples_finalize2_kernel(const unsigned long long *__restrict__ U, long long *__restrict__ qcnt,
                                         long long *__restrict__ sumA, long long *__restrict__ sumB,
                                         long long *__restrict__ sumq, long long *__restrict__ sumq2, int64_t n_a,
                                         int n_rep, int n_slots, int64_t N, int to_q_only) {
  pdl_begin();
  const int n_pairs = n_rep * (n_rep - 1) / 2;
  const int items = n_rep + n_pairs;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n_a * n_slots * items) return;
  const int it = (int)(g % items);
  const int64_t as = g / items;   // a * n_slots + s
  const int64_t a = as / n_slots;
  const int s = (int)(as - a * n_slots);
  if (it < n_rep) {
    if (to_q_only) return;
    const int64_t c = (a * n_rep + it) * n_slots + s;
    sumA[c] += 2 * N - 2 * (long long)U[2 * c];
    sumB[c] += N - 2 * (long long)U[2 * c + 1];
    return;
  }
  long long *qc = &qcnt[as * n_pairs + (it - n_rep)];
  const long long qv = N - 2 * *qc;
  if (to_q_only) {
    *qc = qv;
    return;
  }
  sumq[as * n_pairs + (it - n_rep)] += qv;
  sumq2[as * n_pairs + (it - n_rep)] += qv * qv;
  *qc = 0;
}

// Overlaps (Appendix E.1) at slot s for replica pair p: per-lane number of
// sites where the two configurations differ, accumulated into qcnt[a][s][p].
template <typename Word>
__global__ void __launch_bounds__(kBlock) samples_overlap_kernel(const Word *spins, long long *qcnt,
                                                                 int64_t N, int n_slots, int n_q,
                                                                 int n_rep, int64_t n_samples,
                                                                 int sites_per_thread) {
  pdl_begin();
  constexpr int W = (int)sizeof(Word) * 8;
  __shared__ int acc[W];
  const int n_pairs = n_rep * (n_rep - 1) / 2;
  const int p = blockIdx.y % n_pairs;
  const int s = (blockIdx.y / n_pairs) % n_slots;
  const int64_t b = blockIdx.y / ((int64_t)n_pairs * n_slots);
  int r1 = 0, r2 = 1, k = 0;
  for (int x = 0; x < n_rep; ++x)
    for (int y = x + 1; y < n_rep; ++y, ++k)
      if (k == p) {
        r1 = x;
        r2 = y;
      }
  for (int i = threadIdx.x; i < W; i += blockDim.x) acc[i] = 0;
  __syncthreads();
  const Word *w1 = spins + ((b * n_slots + s) * n_q + (r1 >> 2)) * N * 4 + (r1 & 3);
  const Word *w2 = spins + ((b * n_slots + s) * n_q + (r2 >> 2)) * N * 4 + (r2 & 3);
  VCount<Word, 8> c;
  c.zero();
  const int64_t start = (int64_t)blockIdx.x * blockDim.x * sites_per_thread + threadIdx.x;
  for (int k2 = 0; k2 < sites_per_thread; ++k2) {
    const int64_t site = start + (int64_t)k2 * blockDim.x;
    if (site < N) c.add1(w1[site * 4] ^ w2[site * 4]);
  }
  flush_counter<Word, 8, 1>(c, acc);
  __syncthreads();
  for (int i = threadIdx.x; i < W; i += blockDim.x) {
    const int64_t a = b * W + i;
    if (a < n_samples && acc[i])
      atomicAdd(reinterpret_cast<unsigned long long *>(&qcnt[(a * n_slots + s) * n_pairs + p]),
                (unsigned long long)acc[i]);
  }
}

__global__ void samples_by_slot_kernel(const unsigned long long *U, long long *out, int64_t n, int64_t stride,
                                       int64_t N) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n) return;
  out[c] = 2 * N - 2 * (long long)U[2 * c];
  out[stride + c] = N - 2 * (long long)U[2 * c + 1];
}

template <typename Word>
__global__ void samples_init_J_kernel(Word *J, int64_t n_b, int L, uint2 key) {
  constexpr int W = (int)sizeof(Word) * 8;
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;   // (b, i2, dir)
  const int64_t plane = (int64_t)L * L;
  if (c >= n_b * plane * 2) return;
  const uint32_t dir = (uint32_t)(c & 1);
  const uint32_t i2 = (uint32_t)((c >> 1) % plane);
  const int64_t b = (c >> 1) / plane;
  Word v = 0;
  for (int l = 0; l < W; ++l) {
    const uint4 x = philox(make_uint4(i2, dir, (uint32_t)(b * W + l), DOM_J << 28), key);
    if (!(x.x & 1u)) v |= Word(1) << l;
  }
  J[c] = v;
}

template <typename Word>
__global__ void samples_init_spins_kernel(Word *spins, int64_t total, int64_t N, int n_slots, int n_q,
                                          uint2 key) {
  constexpr int W = (int)sizeof(Word) * 8;
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;   // [b][s][q][site][j]
  if (c >= total) return;
  const int jj = (int)(c & 3);
  const int64_t site = (c >> 2) % N;
  const int64_t bsq = (c >> 2) / N;
  const int q = (int)(bsq % n_q);
  const int s = (int)((bsq / n_q) % n_slots);
  const int64_t b = bsq / ((int64_t)n_q * n_slots);
  const uint32_t r = (uint32_t)(4 * q + jj);
  Word v = 0;
  // walker w starts at slot w: the word of slot s holds walker s
  for (int l = 0; l < W; ++l) {
    const uint4 x = philox(make_uint4((uint32_t)site, (uint32_t)s, (uint32_t)(b * W + l),
                                      (DOM_INIT << 28) | r),
                           key);
    if (!(x.x & 1u)) v |= Word(1) << l;
  }
  spins[c] = v;
}

// Unpack samples a_lo .. a_lo+n_a-1 by walker into int8 +-1.
template <typename Word>
__global__ void samples_extract_kernel(const Word *spins, const int32_t *walker, int8_t *out, int64_t a_lo,
                                       int64_t n_a, int64_t N, int n_slots, int n_q, int n_rep) {
  constexpr int W = (int)sizeof(Word) * 8;
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;   // [ai][r][s][site]
  if (c >= n_a * n_rep * n_slots * N) return;
  const int64_t site = c % N;
  const int s = (int)((c / N) % n_slots);
  const int r = (int)((c / (N * n_slots)) % n_rep);
  const int64_t ai = c / (N * n_slots * n_rep);
  const int64_t a = a_lo + ai;
  const int64_t b = a / W;
  const int lane = (int)(a - b * W);
  const Word v = spins[(((b * n_slots + s) * n_q + (r >> 2)) * N + site) * 4 + (r & 3)];
  const int w = walker[(a * n_rep + r) * n_slots + s];
  out[((ai * n_rep + r) * n_slots + w) * N + site] = ((v >> lane) & 1u) ? -1 : 1;
}

// Pack the int8 +-1 spins of replica r of the samples of word group b
// (staged [a - b W][walker][site], n_a of them) into the lattice: a thread
// per (slot, site) word, lane a - b W, walker from the device labels.
// Pack staged int8 spins into the SAMPLES words: the stage holds n_a
// samples of word group b, each with replicas r0 .. r0 + nr - 1 ([al][rr]
// [slot][site], slot by walker label); a thread packs four consecutive sites
// of one (replica, slot) (N is a multiple of 4: L and L_tau are even).
template <typename Word>
__global__ void samples_pack_kernel(Word *spins, const int8_t *stage, const int32_t *walker, int64_t b, int r0,
                                    int nr, int n_a, int64_t N, int n_slots, int n_q, int n_rep) {
  constexpr int W = (int)sizeof(Word) * 8;
  const int64_t N4 = N / 4;
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;   // [rr][s][site / 4]
  if (c >= (int64_t)nr * n_slots * N4) return;
  const int64_t rs = c / N4;
  const int64_t site = (c - rs * N4) * 4;
  const int rr = (int)(rs / n_slots), s = (int)(rs - (int64_t)rr * n_slots);
  const int r = r0 + rr;
  const int64_t pitch = (int64_t)nr * n_slots * N;   // bytes of one sample in the stage
  Word v0 = 0, v1 = 0, v2 = 0, v3 = 0;
  for (int al = 0; al < n_a; ++al) {
    const int64_t a = b * W + al;
    const int w = walker[(a * n_rep + r) * n_slots + s];
    const char4 x = *reinterpret_cast<const char4 *>(stage + al * pitch + ((int64_t)rr * n_slots + w) * N + site);
    v0 |= Word(x.x == -1) << al;
    v1 |= Word(x.y == -1) << al;
    v2 |= Word(x.z == -1) << al;
    v3 |= Word(x.w == -1) << al;
  }
  Word *o = spins + (((b * n_slots + s) * n_q + (r >> 2)) * N + site) * 4 + (r & 3);
  o[0] = v0;
  o[4] = v1;
  o[8] = v2;
  o[12] = v3;
}

// ---- persistent form: red | blue | PT for a run of sweeps in one launch ----
//
// One cooperative launch runs n sweeps of the 32-bit SAMPLES packing.  Per
// sweep: the fused red pass (the pending PT exchanges applied, the red sites
// updated, the lattice copied into the other buffer; the bond counters
// cleared), a grid barrier, the blue pass in place (bond counters; the PT
// masks cleared, the red pass having read them), a barrier, the PT pass (a
// warp per chain, accepted pairs OR-ed into the masks the next red pass
// applies), a barrier.  Blocks take the passes' blocks in turn (block b does
// b, b + grid, ...), so a pass's work split is the one its own kernel has;
// anything another block wrote earlier in the launch is read through L2.
// The barriers' waits are bounded (error flag -> QISG_ETIMEOUT).
struct PersistArgs {
  FusedRedArgsT<uint32_t> red;    // src/dst set per sweep from buf
  SamplesArgs<uint32_t> blue;     // spins set per sweep
  uint32_t *buf[2];               // the two lattice buffers; buf[0] holds the lattice at launch
  int red_blocks, blue_blocks;
  int32_t *walker;                // [a_pad][r][s]
  unsigned long long *U;          // [a_pad][r][s][2] by slot
  uint32_t *acc;                  // PT lane masks [b][r][s]
  const PTConst *ptc;
  const double *sq;
  uint2 key;
  int64_t n_samples;
  int n_rep, n_slots;
  int64_t n_U, n_acc;             // words the red / blue phase clears
  unsigned long long *d_t;        // sweeps done; advanced by n at the end
  int n_sweeps;
  unsigned *bar;
  int *err;
  long long wait_ns;
};

template <int RP, int KS>
__global__ void __launch_bounds__(kBlock4, 3) samples_persistent_kernel(const PersistArgs a,
                                                                      const __grid_constant__ SlotThresholds th) {
  const unsigned long long t0 = __ldcg(a.d_t);
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  const int warps = (int)((gridDim.x * blockDim.x) >> 5);
  const int gwarp = (int)(gtid >> 5);
  const int lane = threadIdx.x & 31;
  const int64_t n_chains = a.n_samples * a.n_rep;
  for (int sw = 0; sw < a.n_sweeps; ++sw) {
    const unsigned long long t = t0 + (unsigned long long)sw;
    const int cur = sw & 1;
    FusedRedArgsT<uint32_t> rp = a.red;
    rp.src = a.buf[cur];
    rp.dst = a.buf[cur ^ 1];
    for (int64_t i = gtid; i < a.n_U; i += gstride) a.U[i] = 0;
    for (int vb = blockIdx.x; vb < a.red_blocks; vb += gridDim.x) red_fusedq_body<uint32_t, RP, true>(rp, th, vb, t);
    if (!grid_barrier(a.bar, a.err, a.wait_ns)) return;
    for (int64_t i = gtid; i < a.n_acc; i += gstride) a.acc[i] = 0;
    SamplesArgs<uint32_t> bp = a.blue;
    bp.spins = a.buf[cur ^ 1];
    for (int vb = blockIdx.x; vb < a.blue_blocks; vb += gridDim.x)
      sweep4_body<true, KS, true, true>(bp, th, vb, t, 1, 0);
    if (!grid_barrier(a.bar, a.err, a.wait_ns)) return;
    for (int64_t c = gwarp; c < n_chains; c += warps) {   // whole warps: c is uniform over the warp
      const int64_t sa = c / a.n_rep;
      const int r = (int)(c - sa * a.n_rep);
      const uint32_t acc = pt_chain<true, true, false>(a.walker + c * a.n_slots, a.U + c * a.n_slots * 2, a.ptc,
                                                       a.sq, a.key, (uint32_t)t, sa, r, a.n_slots);
      if (lane + 1 < a.n_slots && ((acc >> lane) & 1u))
        atomicOr(a.acc + ((sa >> 5) * a.n_rep + r) * a.n_slots + lane, 1u << (sa & 31));
    }
    if (!grid_barrier(a.bar, a.err, a.wait_ns)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.d_t = t0 + (unsigned long long)a.n_sweeps;
}

template <typename Word>
SamplesArgs<Word> make_args(qisg_handle *h, int colour) {
  SamplesArgs<Word> p;
  p.spins = reinterpret_cast<Word *>(h->spins);
  p.J = reinterpret_cast<const Word *>(h->J);
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
  p.n_slots = h->n_slots;
  p.n_rep = h->n_rep;
  p.n_q = h->n_q;
  p.W = h->W;
  p.zero_U = h->d_U;
  p.n_zero_U = h->n_a_pad * h->n_rep * h->n_slots * 2;
  p.zero_acc = reinterpret_cast<Word *>(h->d_acc);
  p.n_zero_acc = h->n_b * h->n_rep * h->n_slots;
  p.one = 1u;
  // sites per quad along tau: as many as possible (cheaper energy flushes)
  // while the grid keeps about sweep_min_blocks_per_sm blocks per SM; G must
  // divide L_tau / 2
  const int half_col = h->Lt / 2;
  const int64_t sets = h->n_b * h->n_slots * h->n_q;
  const int64_t want_blocks = (int64_t)h->sweep_min_blocks_per_sm * std::max(1, h->n_sm);
  const int tile = h->sweep_tile[colour];
  int G = 4 * std::max(1, tile > 0 ? tile : 64);
  auto blocks_for = [&](int g) {
    const int gg = std::min(g, half_col);
    const int ns = half_col / gg;
    return sets * (((int64_t)p.plane * ns + kQuads - 1) / kQuads);
  };
  if (tile <= 0)
    while (G > 4 && blocks_for(G) < want_blocks) G >>= 1;
  if (G > half_col) G = half_col;
  if (half_col % G) G = half_col;   // one segment per column
  p.seg_sites = G;
  p.n_seg = half_col / G;
  p.seg_base = G;
  p.seg_rem = 0;
  p.seg_blocks = 0;
  p.blocks_per_set = (int)(((int64_t)p.plane * p.n_seg + kQuads - 1) / kQuads);
  p.fd_bps = FastDiv((uint32_t)p.blocks_per_set);
  p.fd_nq = FastDiv((uint32_t)p.n_q);
  p.fd_ns = FastDiv((uint32_t)p.n_slots);
  p.fd_plane = FastDiv((uint32_t)p.plane);
  p.fd_L = FastDiv((uint32_t)p.L);
  p.t_copy = nullptr;
  p.tau_ap = h->tau_ap;
  return p;
}

// Bit planes that hold a sum of at most 4 G per lane (the u_s counter of a
// walk of G sites; the u_t counter takes one less), at least 3.
int counter_planes(int G) {
  int k = 0;
  while ((4 * G) >> k) ++k;
  return std::max(k, 3);
}

template <typename Word, bool BLUE, int G2>
void launch_sweep(bool pdl, const SamplesArgs<Word> &p, const SlotThresholds &th, unsigned blocks, cudaStream_t st,
                  int colour, int count_only) {
  launch_kernel(pdl, samples_half_sweep_kernel<Word, BLUE, G2>, dim3(blocks), dim3(kBlock), 0, st, p, th, colour,
                count_only);
}

template <typename Word, bool BLUE>
void launch_sweep_g(bool pdl, const SamplesArgs<Word> &p, const SlotThresholds &th, unsigned blocks, cudaStream_t st,
                    int colour, int count_only) {
  // counter planes for G sites per thread: G2 = ceil(log2(G / 4))
  int g2 = 0;
  while ((4 << g2) < p.seg_sites) ++g2;
  switch (g2) {
    case 0: launch_sweep<Word, BLUE, 0>(pdl, p, th, blocks, st, colour, count_only); break;
    case 1: launch_sweep<Word, BLUE, 1>(pdl, p, th, blocks, st, colour, count_only); break;
    case 2: launch_sweep<Word, BLUE, 2>(pdl, p, th, blocks, st, colour, count_only); break;
    case 3: launch_sweep<Word, BLUE, 3>(pdl, p, th, blocks, st, colour, count_only); break;
    case 4: launch_sweep<Word, BLUE, 4>(pdl, p, th, blocks, st, colour, count_only); break;
    case 5: launch_sweep<Word, BLUE, 5>(pdl, p, th, blocks, st, colour, count_only); break;
    case 6: launch_sweep<Word, BLUE, 6>(pdl, p, th, blocks, st, colour, count_only); break;
    default: launch_sweep<Word, BLUE, 7>(pdl, p, th, blocks, st, colour, count_only); break;
  }
}

// The 9 classes' accept constants C = 2^64 - T' of every slot, in the form
// accept_flag reads them (T' = T, or 2^32 for the always-accept sentinel).
void fill_thresholds(const qisg_handle *h, SlotThresholds &th) {
  std::memset(&th, 0, sizeof(th));
  static const int cls[9] = {0, 3, 6, 9, 12, 1, 4, 2, 5};   // us * 3 + ut of the 9 classes
  for (int sl = 0; sl < h->n_slots; ++sl)
    for (int c = 0; c < 9; ++c) {
      const uint32_t T = h->T[(size_t)sl * 15 + cls[c]];
      const unsigned long long Tp = T == 0xFFFFFFFFu ? (1ull << 32) : (unsigned long long)T;
      th.v[sl][c] = 0ull - Tp;
    }
}

// Blocks per SM the blue kernel's registers are bounded to: MINB when the
// caller asks (variant 2), three for the prefetching walk up to 7 counter
// planes (168 registers without spills; 7 planes would otherwise take two
// blocks), none beyond (the bound would spill).
template <bool PF, int MINB, int KS>
constexpr int blue_min_blocks() {
  return MINB > 0 ? MINB : (PF && KS <= 7) ? 3 : 0;
}

// Blocks of the W = 32 blue kernel (variant 0 or 2, ks = 3 .. 9 counter
// planes) resident on one SM, cached in the handle.
int blue_blocks_per_sm(qisg_handle *h, int ks, int variant) {
  const int v = variant == 2 ? 1 : 0;
  ks = std::min(std::max(ks, 3), 9);
  int &c = h->blue_occ[v][ks - 3];
  if (c > 0) return c;
  const void *fn = nullptr;
#define QISG_OCC(n)                                                                                   \
  case n:                                                                                             \
    fn = v ? (const void *)samples_sweep4_kernel<true, n, false, 4>                                   \
           : (const void *)samples_sweep4_kernel<true, n, true, blue_min_blocks<true, 0, n>()>;         \
    break;
  switch (ks) { QISG_OCC(3) QISG_OCC(4) QISG_OCC(5) QISG_OCC(6) QISG_OCC(7) QISG_OCC(8) default: QISG_OCC(9) }
#undef QISG_OCC
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlock4, 0) != cudaSuccess || per_sm < 1) {
    (void)cudaGetLastError();
    per_sm = 1;
  }
  return c = per_sm;
}

// Blocks of one (b, s, q) set for n_seg segments per column: a block per
// (segment, 128 columns) when the plane is a multiple of 128 (walk lengths
// may then differ between segments), else 128 consecutive (segment, column)
// pairs per block (segments of one length).
int64_t blocks_per_set4(int plane, int n_seg) {
  return plane % kBlock4 == 0 ? (int64_t)(plane / kBlock4) * n_seg
                              : ((int64_t)plane * n_seg + kBlock4 - 1) / kBlock4;
}

// Segments per column of the blue pass when no tile is pinned: the count
// that minimises (waves of blocks over the resident ones) x (work of one
// block), a block's work being its threads' walks of G sites on average
// (about 490 instructions a site for the four replica words) plus its
// counter tree (about 32 instructions per counter plane and level): the
// pass is latency-bound, so a block takes about the same time whatever the
// blocks beside it on the SM.  Walks of at most max_walk sites; counts that
// leave segments of unequal length are candidates only when a block holds
// one segment.  resident(ks) gives the resident blocks for ks counter
// planes.
template <typename Resident>
int wave_fill_segments(int64_t sets, int plane, int half_col, int max_walk, Resident resident) {
  int best = half_col;
  double best_cost = -1.0;
  for (int ns = std::max(1, (half_col + max_walk - 1) / max_walk); ns <= half_col; ++ns) {
    if (plane % kBlock4 != 0 && half_col % ns != 0) continue;
    const int gmax = (half_col + ns - 1) / ns;
    const int ks = counter_planes(gmax);
    const int64_t R = std::max<int64_t>(1, resident(ks));
    const int64_t blocks = sets * blocks_per_set4(plane, ns);
    const int64_t waves = (blocks + R - 1) / R;
    const double cost = (double)waves * (490.0 * half_col / ns + 32.0 * (2 * ks + 13));
    if (best_cost < 0.0 || cost < best_cost) {
      best_cost = cost;
      best = ns;
    }
  }
  return best;
}

// W = 32 kernel: one thread per column segment.  A pinned tile G gives
// ceil((L_tau / 2) / G) segments of at most G sites (planes that are not a
// multiple of 128: the largest divisor of L_tau / 2 not above G); the
// default gives the
// blue pass the wave-filling count above (resident_blocks: the launch's
// resident blocks, 0 = those of the blue kernel itself; walks of at most
// max_walk sites) and the red pass as many sites per thread as keep about
// half the old kernel's thread count.
SamplesArgs<uint32_t> make_args4(qisg_handle *h, int colour, SlotThresholds &th, int64_t resident_blocks = 0,
                                 int max_walk = 64) {
  SamplesArgs<uint32_t> p = make_args<uint32_t>(h, colour);
  const int half_col = h->Lt / 2;
  const int64_t sets = h->n_b * h->n_slots * h->n_q;
  const int tile = std::min(h->sweep_tile[colour], half_col);
  int n_seg;
  if (tile > 0 && p.plane % kBlock4 == 0) {
    n_seg = (half_col + tile - 1) / tile;
  } else if (tile > 0) {
    int G = tile;
    while (G > 1 && half_col % G) --G;
    n_seg = half_col / G;
  } else if (colour == 1) {
    const int variant = h->sweep_variant[1];
    n_seg = wave_fill_segments(sets, p.plane, half_col, max_walk, [&](int ks) -> int64_t {
      return resident_blocks > 0 ? resident_blocks : (int64_t)blue_blocks_per_sm(h, ks, variant) * std::max(1, h->n_sm);
    });
  } else {
    const int64_t want_threads = (int64_t)h->sweep_min_blocks_per_sm * std::max(1, h->n_sm) * kBlock / 2;
    int G = 64;
    while (G > 1 && sets * p.plane * (int64_t)(half_col / std::min(G, half_col)) < want_threads) G >>= 1;
    if (G > half_col) G = half_col;
    while (G > 1 && half_col % G) --G;
    n_seg = half_col / G;
  }
  p.n_seg = n_seg;
  p.seg_base = half_col / n_seg;
  p.seg_rem = half_col % n_seg;
  p.seg_sites = p.seg_base + (p.seg_rem > 0 ? 1 : 0);
  p.seg_blocks = p.plane % kBlock4 == 0 ? p.plane / kBlock4 : 0;
  p.fd_sb = FastDiv((uint32_t)std::max(1, p.seg_blocks));
  p.blocks_per_set = (int)blocks_per_set4(p.plane, n_seg);
  p.fd_bps = FastDiv((uint32_t)p.blocks_per_set);
  fill_thresholds(h, th);
  return p;
}

// MINB > 0: the kernel's registers are bounded so that MINB blocks fit on an
// SM (variant 2 of the blue pass: more resident warps, no prefetch).
template <bool BLUE, bool PF, int MINB = 0>
void launch_sweep4(bool pdl, const SamplesArgs<uint32_t> &p, const SlotThresholds &th, unsigned blocks, cudaStream_t st,
                   int colour, int count_only, const PTFold &f = PTFold{}) {
  if constexpr (!BLUE) {   // the red pass keeps no counters
    launch_kernel(pdl, samples_sweep4_kernel<false, 3, PF>, dim3(blocks), dim3(kBlock4), 0, st, p, th, colour,
                  count_only, f);
  } else {
    switch (counter_planes(p.seg_sites)) {   // walks of at most 64 sites: 3 .. 9 planes
#define QISG_CASE(n)                                                                                         \
  case n:                                                                                                    \
    launch_kernel(pdl, samples_sweep4_kernel<true, n, PF, blue_min_blocks<PF, MINB, n>()>, dim3(blocks),      \
                  dim3(kBlock4), 0, st, p, th, colour, count_only, f);                                       \
    break;
      QISG_CASE(3) QISG_CASE(4) QISG_CASE(5) QISG_CASE(6) QISG_CASE(7) QISG_CASE(8)
      default:
        launch_kernel(pdl, samples_sweep4_kernel<true, 9, PF, blue_min_blocks<PF, MINB, 9>()>, dim3(blocks),
                      dim3(kBlock4), 0, st, p, th, colour, count_only, f);
        break;
#undef QISG_CASE
    }
  }
}

// Arguments of the fused red pass (and its threads per site, from the red
// tile: 1 -> four, 2 -> two, else one, 0 -> four for lattices with few sites
// per launch; 64-bit words: at most two replicas per thread) and its block
// count.
template <typename Word>
int make_red_args(qisg_handle *h, SlotThresholds &th, FusedRedArgsT<Word> &p, int &tpsite, int64_t &blocks) {
  const SamplesArgs<Word> a = make_args<Word>(h, 0);
  fill_thresholds(h, th);
  p.src = reinterpret_cast<const Word *>(h->spins);
  p.dst = reinterpret_cast<Word *>(h->spins_alt);
  p.J = reinterpret_cast<const Word *>(h->J);
  p.acc = reinterpret_cast<const Word *>(h->d_acc);
  p.d_t = h->d_t;
  p.zero_U = h->d_U;
  p.n_zero_U = a.n_zero_U;
  p.key = a.key;
  p.N = h->N;
  p.L = h->L;
  p.Lt = h->Lt;
  p.plane = a.plane;
  p.n_slots = h->n_slots;
  p.n_q = h->n_q;
  p.n_rep = h->n_rep;
  p.one = 1u;
  p.tau_ap = h->tau_ap;
  p.ticket = h->d_bar ? h->d_bar + 2 : nullptr;
  if (h->sweep_tile[0] == 0) {
    // default: a thread per site and replica unless one thread per site
    // already gives a few waves of full SMs (2048 threads each)
    const int64_t site_threads = h->n_b * h->n_q * (int64_t)a.plane * (h->Lt / 2);
    tpsite = site_threads < (int64_t)4 * 2048 * std::max(1, h->n_sm) ? 4 : 1;
  } else {
    tpsite = h->sweep_tile[0] == 1 ? 4 : h->sweep_tile[0] == 2 ? 2 : 1;
  }
  if (sizeof(Word) == 8 && tpsite == 1) tpsite = 2;
  const int64_t threads_per_set = (int64_t)a.plane * (h->Lt / 2) * tpsite;
  if (threads_per_set + kBlock4 > 0x7FFFFFFF) return fail(QISG_EINVAL, "lattice too large for one launch");
  p.blocks_per_set = (int)((threads_per_set + kBlock4 - 1) / kBlock4);
  p.fd_bps = FastDiv((uint32_t)p.blocks_per_set);
  p.fd_nq = FastDiv((uint32_t)h->n_q);
  p.fd_plane = FastDiv((uint32_t)a.plane);
  p.fd_L = FastDiv((uint32_t)h->L);
  blocks = h->n_b * h->n_q * p.blocks_per_set;
  if (blocks > 0x7FFFFFFF) return fail(QISG_EINVAL, "lattice too large for one launch");
  return QISG_OK;
}

template <typename Word>
int fused_red(qisg_handle *h) {
  SlotThresholds th;
  FusedRedArgsT<Word> p;
  int tpsite = 1;
  int64_t blocks = 0;
  const int rc = make_red_args<Word>(h, th, p, tpsite, blocks);
  if (rc) return rc;
  const int tok = prof_begin(h, QISG_KERNEL_SWEEP);
  if constexpr (sizeof(Word) == 4) {
    const FusedRedArgs &p32 = p;
    if (tpsite == 4)
      launch_kernel(h->pdl, samples_red_fused_kernel, dim3((unsigned)blocks), dim3(kBlock4), 0, h->stream, p32, th);
    else if (tpsite == 2)
      launch_kernel(h->pdl, samples_red_fusedq_kernel<uint32_t, 2>, dim3((unsigned)blocks), dim3(kBlock4), 0, h->stream, p, th);
    else
      launch_kernel(h->pdl, samples_red_fusedq_kernel<uint32_t, 4>, dim3((unsigned)blocks), dim3(kBlock4), 0, h->stream, p, th);
  } else {
    if (tpsite == 4)
      launch_kernel(h->pdl, samples_red_fusedq_kernel<Word, 1>, dim3((unsigned)blocks), dim3(kBlock4), 0, h->stream, p, th);
    else
      launch_kernel(h->pdl, samples_red_fusedq_kernel<Word, 2>, dim3((unsigned)blocks), dim3(kBlock4), 0, h->stream, p, th);
  }
  prof_end(h, QISG_KERNEL_SWEEP, tok);
  h->launches++;
  std::swap(h->spins, h->spins_alt);
  h->perm_pending = false;
  return cuda_check(cudaGetLastError(), "samples red pass");
}

template <typename Word>
int half_sweep_t(qisg_handle *h, int colour, int count_only) {
  if (h->fused && colour == 0 && !count_only) return fused_red<Word>(h);
  // W = 32, blue variants 0 and 2 (and the counting red pass): a thread per
  // (column segment, replica quad), variant 2 with its registers bounded to
  // four blocks per SM; otherwise the column walk, a thread per (column
  // segment, replica)
  if (sizeof(Word) == 4 && !(colour == 1 && h->sweep_variant[1] == 1)) {
    SlotThresholds th;
    SamplesArgs<uint32_t> p = make_args4(h, colour, th);
    if (h->fused && colour == 1) {   // the fused red pass read the masks: clear them here
      p.n_zero_U = 0;
      if (!count_only) p.t_copy = h->d_t + 1;
    } else if (colour == 1) {
      p.n_zero_U = 0;
      p.n_zero_acc = 0;
    }
    const int64_t blocks = h->n_b * h->n_slots * h->n_q * p.blocks_per_set;
    if (blocks > 0x7FFFFFFF || (int64_t)p.blocks_per_set * kBlock4 > 0x7FFFFFFF)
      return fail(QISG_EINVAL, "lattice too large for one launch");
    // the PT pass of this sweep in the blue pass's last blocks, when the
    // chains fit a warp each in at most half the grid and half the resident
    // blocks, energy differences fit 32 bits and the sweep's PT is due
    PTFold f{};
    h->pt_folded = false;
    if (colour == 1 && h->fused && !count_only && h->pt_in_blue && h->pt_every > 0 &&
        (h->t + 1) % (uint64_t)h->pt_every == 0 && 2 * h->N < (int64_t(1) << 30) && h->n_slots <= kMaxSlotsPT) {
      const int64_t chains = h->n_samples * h->n_rep;
      const int64_t P = (chains + kBlock4 / 32 - 1) / (kBlock4 / 32);
      const int64_t resident = (int64_t)blue_blocks_per_sm(h, counter_planes(p.seg_sites), h->sweep_variant[1]) *
                               std::max(1, h->n_sm);
      if (P >= 1 && 2 * P <= blocks && 2 * P <= resident) {
        f.P = (int)P;
        f.ticket = h->d_bar + 2;
        f.walker = h->d_walker;
        f.U = h->d_U;
        f.acc = reinterpret_cast<uint32_t *>(h->d_acc);
        f.ptc = reinterpret_cast<const PTConst *>(h->d_ptc);
        f.sq = h->d_sq;
        f.d_t = h->d_t;
        f.err = h->d_err;
        f.wait_ns = h->wait_ns;
        f.n_samples = h->n_samples;
        f.n_rep = h->n_rep;
        f.n_slots = h->n_slots;
        p.t_copy = nullptr;
        h->pt_folded = true;
      }
    }
    const int tok = prof_begin(h, sweep_kind(colour));
    // the blue pass loads the next site of its walk while it updates the
    // current one (measured: 4% off the production sweep, with the tuner then
    // taking walks of 4 sites)
    if (colour == 1 && h->sweep_variant[1] == 2)
      launch_sweep4<true, false, 4>(h->pdl, p, th, (unsigned)blocks, h->stream, 1, count_only, f);
    else if (colour == 1)
      launch_sweep4<true, true>(h->pdl, p, th, (unsigned)blocks, h->stream, 1, count_only, f);
    else
      launch_sweep4<false, false>(h->pdl, p, th, (unsigned)blocks, h->stream, 0, count_only);
    prof_end(h, sweep_kind(colour), tok);
    h->launches++;
    return cuda_check(cudaGetLastError(), "samples half sweep");
  }
  SamplesArgs<Word> p = make_args<Word>(h, colour);
  SlotThresholds th;
  fill_thresholds(h, th);
  if (colour == 1) {
    p.n_zero_U = 0;
    if (h->fused) {   // masks read by the fused red pass: clear them here
      if (!count_only) p.t_copy = h->d_t + 1;
    } else {
      p.n_zero_acc = 0;
    }
  }
  const int64_t sets = h->n_b * h->n_slots * h->n_q;
  const int64_t blocks = sets * p.blocks_per_set;
  if (blocks > 0x7FFFFFFF || (int64_t)p.blocks_per_set * kQuads > 0x7FFFFFFF)
    return fail(QISG_EINVAL, "lattice too large for one launch");
  const int tok = prof_begin(h, sweep_kind(colour));
  if (colour == 1)
    launch_sweep_g<Word, true>(h->pdl, p, th, (unsigned)blocks, h->stream, 1, count_only);
  else
    launch_sweep<Word, false, 0>(h->pdl, p, th, (unsigned)blocks, h->stream, 0, count_only);
  prof_end(h, sweep_kind(colour), tok);
  h->launches++;
  return cuda_check(cudaGetLastError(), "samples half sweep");
}

template <typename Word>
int clear_masks(qisg_handle *h) {
  return cuda_check(cudaMemsetAsync(h->d_acc, 0, (size_t)h->n_b * h->n_rep * h->n_slots * sizeof(Word), h->stream),
                    "clear PT masks");
}

template <typename Word>
int permute_t(qisg_handle *h, int advance);

// PT pass.  Fused mode (W = 32), sweep pass: the exchanges stay pending in
// the masks for the next red pass, and the PT kernel advances the sweep
// counter.  Otherwise (and for an explicit pass) the lattice is permuted now.
template <typename Word>
int pt_t(qisg_handle *h, int explicit_pass, int advance) {
  int rc = QISG_OK;
  if (explicit_pass || h->perm_pending) {   // masks still set: apply them first
    rc = samples_materialize(h);
    if (!rc) rc = clear_masks<Word>(h);
  }
  if (rc) return rc;
  if (h->fused && !explicit_pass) {
    // the blue pass of this sweep ran the PT chains in its last blocks and
    // advanced the counter
    if (!h->pt_folded) rc = pt_pass(h, 0, 0, h->n_samples, advance ? h->d_t : nullptr);
    h->pt_folded = false;
    if (!rc) h->perm_pending = true;
    return rc;
  }
  rc = pt_pass(h, explicit_pass, 0, h->n_samples, nullptr);
  if (!rc) rc = permute_t<Word>(h, advance);
  if (!rc && h->fused) rc = clear_masks<Word>(h);
  return rc;
}

template <typename Word>
int permute_t(qisg_handle *h, int advance) {
  const int tok = prof_begin(h, QISG_KERNEL_PERMUTE);
  unsigned long long *adv = advance ? h->d_t : nullptr;
  if (sizeof(Word) == 4) {
    const int64_t per_set = (h->N + kBlock4 - 1) / kBlock4;
    const unsigned blocks = (unsigned)(h->n_b * h->n_q * per_set);
    uint4 *sp = reinterpret_cast<uint4 *>(h->spins);
    const uint32_t *ac = reinterpret_cast<const uint32_t *>(h->d_acc);
    if (h->n_slots <= 8)
      launch_kernel(h->pdl, samples_permute4_kernel<8>, dim3(blocks), dim3(kBlock4), 0, h->stream, sp, ac, h->N, h->n_slots, h->n_q, h->n_rep,
                                                                   (int)per_set, adv);
    else if (h->n_slots <= 16)
      launch_kernel(h->pdl, samples_permute4_kernel<16>, dim3(blocks), dim3(kBlock4), 0, h->stream, sp, ac, h->N, h->n_slots, h->n_q, h->n_rep,
                                                                    (int)per_set, adv);
    else
      launch_kernel(h->pdl, samples_permute4_kernel<32>, dim3(blocks), dim3(kBlock4), 0, h->stream, sp, ac, h->N, h->n_slots, h->n_q, h->n_rep,
                                                                    (int)per_set, adv);
  } else {
    const int64_t per_set = (h->N * 4 + kBlock - 1) / kBlock;
    const int64_t blocks = h->n_b * h->n_q * per_set;
    launch_kernel(h->pdl, samples_permute_kernel<Word>, dim3((unsigned)blocks), dim3(kBlock), 0, h->stream,
                  reinterpret_cast<Word *>(h->spins), reinterpret_cast<const Word *>(h->d_acc), h->N, h->n_slots,
                  h->n_q, h->n_rep, (int)per_set, adv);
  }
  prof_end(h, QISG_KERNEL_PERMUTE, tok);
  h->launches++;
  return cuda_check(cudaGetLastError(), "samples permute");
}

template <typename Word>
int measure_t(qisg_handle *h, int force_to_q) {
  int rc0 = samples_materialize(h);
  if (rc0) return rc0;
  const int n_pairs = h->n_pairs();
  if (n_pairs > 0 && h->n_q == 1) {
    constexpr int spt = 16, K = 5;   // 16 sites per thread: counts <= 16 need 5 planes
    const int64_t per_set = (h->N + (int64_t)kBlock4 * spt - 1) / ((int64_t)kBlock4 * spt);
    const int64_t blocks = h->n_b * h->n_slots * per_set;
    if (blocks > 0x7FFFFFFF) return fail(QISG_EINVAL, "lattice too large for one launch");
    const int tok = prof_begin(h, QISG_KERNEL_MEASURE);
    launch_kernel(h->pdl, samples_overlap4_kernel<Word, K>, dim3((unsigned)blocks), dim3(kBlock4), 0, h->stream,
                  reinterpret_cast<const Word *>(h->spins), h->d_q, h->N, h->n_slots, h->n_rep, h->n_samples, spt,
                  (int)per_set);
    prof_end(h, QISG_KERNEL_MEASURE, tok);
    h->launches++;
  } else if (n_pairs > 0) {
    const int spt = 16;
    const int64_t bx = (h->N + (int64_t)kBlock * spt - 1) / ((int64_t)kBlock * spt);
    const int64_t by = h->n_b * h->n_slots * n_pairs;
    if (by > 65535) return fail(QISG_EINVAL, "too many (block, slot, pair) sets for one launch");
    const int tok = prof_begin(h, QISG_KERNEL_MEASURE);
    launch_kernel(h->pdl, samples_overlap_kernel<Word>, dim3((unsigned)bx, (unsigned)by), dim3(kBlock), 0, h->stream,
                  reinterpret_cast<const Word *>(h->spins), h->d_q, h->N, h->n_slots, h->n_q, h->n_rep,
                  h->n_samples, spt);
    prof_end(h, QISG_KERNEL_MEASURE, tok);
    h->launches++;
  }
  const int64_t n = h->n_samples * h->n_slots * (h->n_rep + n_pairs);
  launch_kernel(h->pdl, samples_finalize2_kernel, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, h->stream,
                h->d_U, h->d_q, h->d_sumA, h->d_sumB, h->d_sumq, h->d_sumq2, h->n_samples, h->n_rep,
                h->n_slots, h->N, force_to_q);
  h->launches++;
  return cuda_check(cudaGetLastError(), "samples measure");
}

template <typename Word>
int init_t(qisg_handle *h) {
  const uint2 key = make_uint2((uint32_t)h->seed, (uint32_t)(h->seed >> 32));
  const int64_t nJ = h->n_b * h->L * h->L * 2;
  samples_init_J_kernel<Word><<<(unsigned)((nJ + 255) / 256), 256, 0, h->stream>>>(
      reinterpret_cast<Word *>(h->J), h->n_b, h->L, key);
  const int64_t total = h->n_b * h->n_slots * h->n_q * h->N * 4;
  if ((total + 255) / 256 > 0x7FFFFFFF) return fail(QISG_EINVAL, "lattice too large");
  samples_init_spins_kernel<Word><<<(unsigned)((total + 255) / 256), 256, 0, h->stream>>>(
      reinterpret_cast<Word *>(h->spins), total, h->N, h->n_slots, h->n_q, key);
  h->launches += 2;
  return cuda_check(cudaGetLastError(), "samples init");
}

// Unpacked in chunks of samples (at most 256 MB of int8 staged at a time).
template <typename Word>
int get_spins_t(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *S) {
  if (n_a == 0) return QISG_OK;
  const int64_t per_a = (int64_t)h->n_rep * h->n_slots * h->N;
  const int64_t chunk = std::min(n_a, std::max<int64_t>(1, ((int64_t)256 << 20) / per_a));
  int rc = samples_materialize(h);
  if (rc) return rc;
  int8_t *d = nullptr;
  rc = cuda_check(cudaMalloc(&d, (size_t)(chunk * per_a)), "cudaMalloc");
  if (rc) return rc;
  for (int64_t a0 = 0; a0 < n_a && !rc; a0 += chunk) {
    const int64_t na = std::min(chunk, n_a - a0), n = na * per_a;
    samples_extract_kernel<Word><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(
        reinterpret_cast<const Word *>(h->spins), h->d_walker, d, a_lo + a0, na, h->N, h->n_slots, h->n_q,
        h->n_rep);
    h->launches++;
    rc = cuda_check(cudaGetLastError(), "extract");
    if (!rc) rc = cuda_check(cudaMemcpyAsync(S + a0 * per_a, d, (size_t)n, cudaMemcpyDeviceToHost, h->stream), "copy");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(h->stream), "sync");
  }
  cudaFree(d);
  return rc;
}

// Every byte of the staged state is +1 (0x01) or -1 (0xFF); a thread sets
// *bad when one of its words holds another byte.
__global__ void pm1_check_kernel(const uint32_t *__restrict__ w, int64_t n_words, int *bad) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  uint32_t any = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_words; i += stride) {
    const uint32_t v = w[i];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t b = (v >> (8 * k)) & 0xFFu;
      any |= (uint32_t)(b != 0x01u && b != 0xFFu);
    }
  }
  if (any) atomicOr(bad, 1);
}

template <typename Word>
int set_spins_t(qisg_handle *h, const int8_t *S, const int32_t *walker_at, const int8_t *d_S) {
  constexpr int W = (int)sizeof(Word) * 8;
  if (h->perm_pending) {   // the new state replaces the one the masks refer to
    const int rc = clear_masks<Word>(h);
    if (rc) return rc;
    h->perm_pending = false;
  }
  // the walker labels are on the device already (qisg_set_state uploads
  // them first).  With the state already on the device (d_S) each word
  // group is packed from there; otherwise the spins go up one word group at
  // a time (all its replicas in one copy while that stays within 256 MB of
  // staging, else a few replicas per copy) into a staging buffer and are
  // packed there
  (void)walker_at;
  const int64_t row = (int64_t)h->n_slots * h->N;   // bytes of one (sample, replica)
  if (d_S) {
    int rc = QISG_OK;
    if ((size_t)h->n_q * 4 > (size_t)h->n_rep)
      rc = cuda_check(cudaMemsetAsync(h->spins, 0, (size_t)h->n_b * h->n_slots * h->n_q * h->N * 4 * sizeof(Word),
                                      h->stream),
                      "memset");
    for (int64_t b = 0; b < h->n_b && !rc; ++b) {
      const int n_a = (int)std::min<int64_t>(W, h->n_samples - b * W);
      const int64_t threads = (int64_t)h->n_rep * row / 4;
      samples_pack_kernel<Word><<<(unsigned)((threads + 255) / 256), 256, 0, h->stream>>>(
          reinterpret_cast<Word *>(h->spins), d_S + b * W * h->n_rep * row, h->d_walker, b, 0, h->n_rep, n_a, h->N,
          h->n_slots, h->n_q, h->n_rep);
      h->launches++;
      rc = cuda_check(cudaGetLastError(), "pack spins");
    }
    if (!rc) rc = cuda_check(cudaStreamSynchronize(h->stream), "sync");
    return rc;
  }
  const int nr = (int)std::max<int64_t>(1, std::min<int64_t>(h->n_rep, ((int64_t)256 << 20) / ((int64_t)W * row)));
  int8_t *stage = nullptr;
  int rc = cuda_check(cudaMalloc(&stage, (size_t)W * nr * row), "cudaMalloc");
  if (rc) return rc;
  if ((size_t)h->n_q * 4 > (size_t)h->n_rep) {   // padding replicas of the last quad stay 0
    rc = cuda_check(cudaMemsetAsync(h->spins, 0, (size_t)h->n_b * h->n_slots * h->n_q * h->N * 4 * sizeof(Word),
                                    h->stream),
                    "memset");
  }
  for (int64_t b = 0; b < h->n_b && !rc; ++b) {
    const int n_a = (int)std::min<int64_t>(W, h->n_samples - b * W);
    for (int r0 = 0; r0 < h->n_rep && !rc; r0 += nr) {
      const int k = std::min(nr, h->n_rep - r0);
      rc = cuda_check(cudaMemcpy2DAsync(stage, (size_t)(k * row), S + ((b * W) * h->n_rep + r0) * row,
                                        (size_t)(h->n_rep * row), (size_t)(k * row), (size_t)n_a,
                                        cudaMemcpyHostToDevice, h->stream),
                      "copy spins");
      if (rc) break;
      const int64_t threads = (int64_t)k * row / 4;
      samples_pack_kernel<Word><<<(unsigned)((threads + 255) / 256), 256, 0, h->stream>>>(
          reinterpret_cast<Word *>(h->spins), stage, h->d_walker, b, r0, k, n_a, h->N, h->n_slots, h->n_q, h->n_rep);
      h->launches++;
      rc = cuda_check(cudaGetLastError(), "pack spins");
    }
  }
  if (!rc) rc = cuda_check(cudaStreamSynchronize(h->stream), "sync");
  cudaFree(stage);
  return rc;
}

template <typename Word>
int get_couplings_t(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *J) {
  constexpr int W = (int)sizeof(Word) * 8;
  const int64_t plane = (int64_t)h->L * h->L;
  std::vector<Word> buf((size_t)h->n_b * plane * 2);
  int rc = cuda_check(cudaMemcpyAsync(buf.data(), h->J, buf.size() * sizeof(Word), cudaMemcpyDeviceToHost,
                                      h->stream),
                      "copy J");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(h->stream), "sync");
  if (rc) return rc;
  for (int64_t ai = 0; ai < n_a; ++ai) {
    const int64_t a = a_lo + ai, b = a / W;
    const int lane = (int)(a - b * W);
    for (int64_t i = 0; i < plane; ++i)
      for (int d = 0; d < 2; ++d)
        J[(ai * plane + i) * 2 + d] = ((buf[(size_t)((b * plane + i) * 2 + d)] >> lane) & 1u) ? -1 : 1;
  }
  return QISG_OK;
}

template <typename Word>
int set_couplings_t(qisg_handle *h, const int8_t *J) {
  constexpr int W = (int)sizeof(Word) * 8;
  const int64_t plane = (int64_t)h->L * h->L;
  std::vector<Word> buf((size_t)h->n_b * plane * 2);
  int rc = cuda_check(cudaMemcpyAsync(buf.data(), h->J, buf.size() * sizeof(Word), cudaMemcpyDeviceToHost,
                                      h->stream),
                      "copy J");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(h->stream), "sync");
  if (rc) return rc;
  for (int64_t a = 0; a < h->n_samples; ++a) {
    const int64_t b = a / W;
    const Word bit = Word(1) << (a - b * W);
    for (int64_t i = 0; i < plane; ++i)
      for (int d = 0; d < 2; ++d) {
        Word &v = buf[(size_t)((b * plane + i) * 2 + d)];
        v = (J[(a * plane + i) * 2 + d] == -1) ? (v | bit) : (v & ~bit);
      }
  }
  rc = cuda_check(cudaMemcpyAsync(h->J, buf.data(), buf.size() * sizeof(Word), cudaMemcpyHostToDevice,
                                  h->stream),
                  "copy J");
  if (rc) return rc;
  return cuda_check(cudaStreamSynchronize(h->stream), "sync");
}

}  // namespace

int samples_init(qisg_handle *h) {
  if (h->n_slots > kMaxSlotsPermute) return fail(QISG_EINVAL, "SAMPLES packing supports up to 32 slots");
  if (h->L > 1024) return fail(QISG_EINVAL, "SAMPLES packing supports L <= 1024");
  return h->W == 64 ? init_t<unsigned long long>(h) : init_t<unsigned int>(h);
}
int samples_materialize(qisg_handle *h) {
  if (!h->fused || !h->perm_pending) return QISG_OK;
  int rc = h->W == 64 ? permute_t<unsigned long long>(h, 0) : permute_t<unsigned int>(h, 0);
  if (!rc) rc = h->W == 64 ? clear_masks<unsigned long long>(h) : clear_masks<unsigned int>(h);
  if (!rc) h->perm_pending = false;
  return rc;
}
int samples_half_sweep(qisg_handle *h, int colour, int count_only) {
  return h->W == 64 ? half_sweep_t<unsigned long long>(h, colour, count_only)
                    : half_sweep_t<unsigned int>(h, colour, count_only);
}
bool samples_persistent_ok(const qisg_handle *h) {
  return h->layout == QISG_LAYOUT_SAMPLES && h->W == 32 && h->fused && h->pt_every == 1 &&
         2 * h->N < (int64_t(1) << 30) && h->n_slots <= kMaxSlotsPT && h->d_bar != nullptr;
}

int samples_persistent(qisg_handle *h, int n_sweeps) {
  if (!samples_persistent_ok(h)) return fail(QISG_EINVAL, "persistent form: needs SAMPLES, 32-bit words, PT every sweep");
  if (n_sweeps <= 0) return QISG_OK;
  PersistArgs a;
  SlotThresholds th, th_blue;
  int tpsite = 1;
  int64_t red_blocks = 0;
  int rc = make_red_args<uint32_t>(h, th, a.red, tpsite, red_blocks);
  if (rc) return rc;
  a.red.n_zero_U = 0;
  // the blue phase's default segmentation fills the persistent grid (every
  // form of the kernel is bounded to the same residency), walks of at most
  // 32 sites
  int per_sm0 = 0;
  rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm0, samples_persistent_kernel<1, 5>, kBlock4, 0),
                  "occupancy");
  if (rc) return rc;
  a.blue = make_args4(h, 1, th_blue, (int64_t)std::max(1, per_sm0) * std::max(1, h->n_sm), 32);
  a.blue.n_zero_U = 0;
  a.blue.n_zero_acc = 0;
  a.blue.t_copy = nullptr;
  const int64_t blue_blocks = h->n_b * h->n_slots * h->n_q * a.blue.blocks_per_set;
  if (blue_blocks > 0x7FFFFFFF) return fail(QISG_EINVAL, "lattice too large for one launch");
  const int ks = counter_planes(a.blue.seg_sites);
  if (a.blue.seg_sites > 32) return fail(QISG_EINVAL, "persistent form: blue tile above 32 sites");
  a.buf[0] = reinterpret_cast<uint32_t *>(h->spins);
  a.buf[1] = reinterpret_cast<uint32_t *>(h->spins_alt);
  a.red_blocks = (int)red_blocks;
  a.blue_blocks = (int)blue_blocks;
  a.walker = h->d_walker;
  a.U = h->d_U;
  a.acc = reinterpret_cast<uint32_t *>(h->d_acc);
  a.ptc = reinterpret_cast<const PTConst *>(h->d_ptc);
  a.sq = h->d_sq;
  a.key = make_uint2((uint32_t)h->seed, (uint32_t)(h->seed >> 32));
  a.n_samples = h->n_samples;
  a.n_rep = h->n_rep;
  a.n_slots = h->n_slots;
  a.n_U = h->n_a_pad * h->n_rep * h->n_slots * 2;
  a.n_acc = h->n_b * h->n_rep * h->n_slots;
  a.d_t = h->d_t;
  a.n_sweeps = n_sweeps;
  a.bar = h->d_bar;
  a.err = h->d_err;
  a.wait_ns = h->wait_ns;
  const int rp = tpsite == 4 ? 1 : tpsite == 2 ? 2 : 4;
  const void *fn = nullptr;
#define QISG_PK(R, K) \
  if (rp == R && ks == K) fn = (const void *)samples_persistent_kernel<R, K>;
  QISG_PK(1, 3) QISG_PK(1, 4) QISG_PK(1, 5) QISG_PK(1, 6) QISG_PK(1, 7) QISG_PK(1, 8)
  QISG_PK(2, 3) QISG_PK(2, 4) QISG_PK(2, 5) QISG_PK(2, 6) QISG_PK(2, 7) QISG_PK(2, 8)
  QISG_PK(4, 3) QISG_PK(4, 4) QISG_PK(4, 5) QISG_PK(4, 6) QISG_PK(4, 7) QISG_PK(4, 8)
#undef QISG_PK
  int per_sm = 0;
  rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlock4, 0), "occupancy");
  if (rc) return rc;
  if (per_sm < 1) return fail(QISG_ECUDA, "persistent kernel does not fit on an SM");
  const int grid = per_sm * std::max(1, h->n_sm);
  rc = cuda_check(cudaMemsetAsync(h->d_bar, 0, 2 * sizeof(unsigned), h->stream), "reset barrier");
  if (rc) return rc;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kBlock4);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = h->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void *args[] = {(void *)&a, (void *)&th};
  const int tok = prof_begin(h, QISG_KERNEL_SWEEP);
  rc = cuda_check(cudaLaunchKernelExC(&cfg, fn, args), "persistent sweep kernel");
  prof_end(h, QISG_KERNEL_SWEEP, tok);
  if (rc) return rc;
  h->launches++;
  if (n_sweeps & 1) std::swap(h->spins, h->spins_alt);
  h->perm_pending = true;
  return QISG_OK;
}

int samples_pt(qisg_handle *h, int explicit_pass, int advance) {
  return h->W == 64 ? pt_t<unsigned long long>(h, explicit_pass, advance)
                    : pt_t<unsigned int>(h, explicit_pass, advance);
}
int samples_measure(qisg_handle *h, int force_to_q) {
  return h->W == 64 ? measure_t<unsigned long long>(h, force_to_q) : measure_t<unsigned int>(h, force_to_q);
}
int samples_energies_by_slot(qisg_handle *h) {
  const int64_t n = h->n_samples * h->n_rep * h->n_slots;
  const int64_t stride = h->n_a_pad * h->n_rep * h->n_slots;
  samples_by_slot_kernel<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(h->d_U, h->d_out, n, stride, h->N);
  h->launches++;
  return cuda_check(cudaGetLastError(), "samples energies");
}
int samples_stage_spins(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *d) {
  const int64_t n = n_a * h->n_rep * h->n_slots * h->N;
  if (n == 0) return QISG_OK;
  int rc = samples_materialize(h);
  if (rc) return rc;
  if (h->W == 64)
    samples_extract_kernel<unsigned long long><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(
        reinterpret_cast<const unsigned long long *>(h->spins), h->d_walker, d, a_lo, n_a, h->N, h->n_slots, h->n_q,
        h->n_rep);
  else
    samples_extract_kernel<unsigned int><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(
        reinterpret_cast<const unsigned int *>(h->spins), h->d_walker, d, a_lo, n_a, h->N, h->n_slots, h->n_q,
        h->n_rep);
  h->launches++;
  return cuda_check(cudaGetLastError(), "unpack spins");
}

int samples_get_spins(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *S) {
  return h->W == 64 ? get_spins_t<unsigned long long>(h, a_lo, n_a, S)
                    : get_spins_t<unsigned int>(h, a_lo, n_a, S);
}
int samples_set_spins(qisg_handle *h, const int8_t *S, const int32_t *walker_at, const int8_t *d_S) {
  return h->W == 64 ? set_spins_t<unsigned long long>(h, S, walker_at, d_S)
                    : set_spins_t<unsigned int>(h, S, walker_at, d_S);
}

// Upload n bytes of +-1 spins to a new device buffer (*d_S, which the caller
// frees) and check them there: QISG_ECORRUPT (and no buffer) if a byte is
// neither +1 nor -1.  n is a multiple of 4.
int samples_upload_checked(qisg_handle *h, const int8_t *S, int64_t n, int8_t **d_S) {
  *d_S = nullptr;
  int8_t *buf = nullptr;
  int rc = cuda_check(cudaMalloc(&buf, (size_t)n + 16), "cudaMalloc");
  if (rc) return rc;
  int *bad = reinterpret_cast<int *>(buf + n);   // n is a multiple of 4
  rc = cuda_check(cudaMemsetAsync(bad, 0, sizeof(int), h->stream), "memset");
  if (!rc) rc = cuda_check(cudaMemcpyAsync(buf, S, (size_t)n, cudaMemcpyHostToDevice, h->stream), "copy spins");
  if (!rc) {
    const int64_t words = n / 4;
    const unsigned blocks = (unsigned)std::min<int64_t>((words + 255) / 256, (int64_t)8 * std::max(1, h->n_sm) * 8);
    pm1_check_kernel<<<std::max(1u, blocks), 256, 0, h->stream>>>(reinterpret_cast<const uint32_t *>(buf), words, bad);
    h->launches++;
    rc = cuda_check(cudaGetLastError(), "check spins");
  }
  int flag = 0;
  if (!rc) rc = cuda_check(cudaMemcpyAsync(&flag, bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "copy flag");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(h->stream), "sync");
  if (!rc && flag) rc = fail(QISG_ECORRUPT, "spins must be +-1");
  if (rc) {
    cudaFree(buf);
    return rc;
  }
  *d_S = buf;
  return QISG_OK;
}
int samples_get_couplings(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *J) {
  return h->W == 64 ? get_couplings_t<unsigned long long>(h, a_lo, n_a, J)
                    : get_couplings_t<unsigned int>(h, a_lo, n_a, J);
}
int samples_set_couplings(qisg_handle *h, const int8_t *J) {
  return h->W == 64 ? set_couplings_t<unsigned long long>(h, J) : set_couplings_t<unsigned int>(h, J);
}

}  // namespace qisg
