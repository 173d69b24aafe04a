// Internal declarations shared by the translation units of libqisg.
//
// Paper: "The QISG suite" (MCQSG code).  The model is Eq. (2)-(3) of Sec. 1
// with one (k, k_tau) pair per ladder slot; the update is Sec. 2.1's
// red/blue Metropolis with precomputed Metropolis factors followed by a
// parallel-tempering pass; random numbers are Philox4x32-10 (Sec. 2.1.1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/qisg.h"

namespace qisg {

// Philox counter domains: one per kind of draw.
enum : uint32_t { DOM_J = 1, DOM_INIT = 2, DOM_SWEEP = 3, DOM_PT = 4, DOM_DAEMON = 5 };

// Index bits of the SITES daemon tables (the words' top bits -> candidate bins).
constexpr int kDaemonLutBits = 12;

constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

// Philox4x32-10 (Salmon et al., SC'11), the generator of Sec. 2.1.1.  The
// low and high halves of each product are taken apart: measured faster here
// than one wide multiply per product (the daemon kernels, whose Philox calls
// sit between table lookups, use the wide form, philox_wide).
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

// Squaring chain length: exponents |A_Y - A_X| <= 4N < 2^40.
constexpr int kSqBits = 40;

// b^e by right-to-left binary powering with round-to-nearest multiplies:
// res = 1; for each bit j of e (low to high) res *= b^(2^j), where the
// chain b^(2^j) = (b^(2^(j-1)))^2 was squared once on the host with IEEE
// multiplies.  The multiplies and their operands are exactly those of the
// textbook loop, so the result is bit-identical to it.
__device__ __forceinline__ double pow_chain(const double *chain, unsigned long long e) {
  double r = 1.0;
  int j = 0;
  while (e) {
    if (e & 1ull) r = __dmul_rn(r, __ldg(chain + j));
    e >>= 1;
    ++j;
  }
  return r;
}

// Unsigned 32-bit division by a run-time invariant d >= 1 through one
// multiply-high, two shifts and two adds (Granlund and Montgomery, "Division
// by invariant integers using multiplication", PLDI 1994, Fig. 4.1):
//   l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
//   q = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0),  t = mulhi(m, n).
struct FastDiv {
  uint32_t d, m, s1, s2;
  __host__ __device__ FastDiv() : d(1), m(1), s1(0), s2(0) {}
  __host__ explicit FastDiv(uint32_t div) : d(div) {
    uint32_t l = 0;
    while (l < 32 && (1ull << l) < div) ++l;
    m = (uint32_t)(((1ull << 32) * ((1ull << l) - div)) / div + 1ull);
    s1 = l < 1 ? l : 1;
    s2 = l > 1 ? l - 1 : 0;
  }
  __device__ __forceinline__ uint32_t div(uint32_t n) const {
    const uint32_t t = __umulhi(m, n);
    return (t + ((n - t) >> s1)) >> s2;
  }
};

// Maximum ladder length of the register-resident PT scan.
constexpr int kMaxSlotsPT = 32;

// Per-pair constants of the PT shortcut, read by lane s of a chain's warp:
// dk = k_s - k_{s+1} and dkt = k_tau,s - k_tau,s+1 rounded to float,
// and ge1[w] bit s set when base w (alpha+, alpha-, beta+, beta-) of pair s
// is >= 1.
struct PTConst {
  float dkf[kMaxSlotsPT];
  float dktf[kMaxSlotsPT];
  uint32_t ge1[4];
};

// PT decision for the pair (s, s+1) of chain (a, r) after sweep t (Sec. 2.1):
// accept iff u < P, P = alpha^|m| beta^|n| with m = A_Y - A_X, n = B_Y - B_X,
// alpha = exp(+-(k_s - k_{s+1})) and beta = exp(+-(k_tau,s - k_tau,s+1))
// chosen by the signs of m and n, u = x 2^-32 with x the pair's Philox word.
//
// The decision is the one of that exact rule; three shortcuts only skip
// work:
//  * when both chosen factors are at least 1 (base >= 1 or exponent 0),
//    P >= 1 > u: products and squares of numbers >= 1 round to numbers >= 1;
//  * when both are at most 1 (m dk <= 0 and n dkt <= 0) and one of them has
//    m dk or n dkt <= -23.5, P <= e^-23.5 (1 + 5e-7) < 6.3e-11 < 2^-32 <= u
//    for x > 0: products and squares of numbers <= 1 stay <= 1, so no size
//    of the exponents can overflow (far candidates of a long ladder, whose
//    exponents pass the range below, land here);
//  * otherwise ln u (lnu, within 2e-5) is compared in float with
//    lnP = m dk + n dkt, whose float evaluation is within
//    (|m dk| + |n dkt|) 2.4e-7 of the double value; the exact power chain
//    is within (2(|m|+|n|)+1) ulps (< 1e-5 in log for up to 2^31 sites) of
//    exp of that value.  A margin err = 1e-4 + (|m dk| + |n dkt|) 4.8e-7
//    covers all of these and the float rounding of the comparison, so
//    outside it the outcome is the exact rule's.  x = 0, factors that could
//    leave the normal range (|m dk| or |n dkt| >= 700) and the margin itself
//    fall through to the exact product.
// Exact evaluation of the rule (kept out of line: it is rarely taken and
// inlining it would bloat the scan loop).
static __device__ __noinline__ bool pt_exact(const double *sq, int s, int ia, int ib, long long m, long long n,
                                      uint32_t x) {
  const double fa = pow_chain(sq + ((size_t)s * 4 + ia) * kSqBits, (unsigned long long)(m >= 0 ? m : -m));
  const double fb = pow_chain(sq + ((size_t)s * 4 + ib) * kSqBits, (unsigned long long)(n >= 0 ? n : -n));
  const double P = __dmul_rn(fa, fb);
  const double u = __dmul_rn((double)x, 0x1p-32);
  return u < P;
}

// PT pass of one chain by one warp (Sec. 2.1).  Lane s holds the walker and
// energies of the configuration at slot s, the constants of pair (s, s+1)
// and that pair's Philox word.  In the sequential pass the configuration
// that meets the original occupant of slot s+1 at pair s is always one of
// the original occupants of slots 0..s (carried up by accepted exchanges).
// So pair s is first decided against every candidate i = 0..s (lane s ends
// with bit i of D: accept; the decisions themselves are spread over the
// lanes), with the shortcuts above and the exact rule, in lane s, for the
// few candidates the shortcuts leave open; the pass is then a uniform scan of
// bit lookups: with c carried, pair s accepts iff bit c of D_s; the slot then
// ends with s+1's configuration and c moves on, else it ends with c and s+1
// is carried.  The decisions are those of the textbook pass.
// BY_SLOT: energies indexed by slot (else by walker).  CG: read the mutable
// state through L2 only (persistent kernel).  WIDE: energies may need more
// than 30 bits (2N >= 2^30); otherwise differences are taken in 32 bits.
// Returns the accepted-pair bitmask (same in every lane).
template <bool CG>
__device__ __forceinline__ long long ld_energy(const unsigned long long *p) {
  return (long long)(CG ? __ldcg(p) : *p);
}

template <bool WIDE>
struct PTEnergy {
  using T = long long;
  __device__ static __forceinline__ T shfl(T v, int src) {
    const uint32_t lo = __shfl_sync(0xffffffffu, (uint32_t)v, src);
    const uint32_t hi = __shfl_sync(0xffffffffu, (uint32_t)((unsigned long long)v >> 32), src);
    return (T)(((unsigned long long)hi << 32) | lo);
  }
  __device__ static __forceinline__ T diff2(T x, T y) { return 2 * (x - y); }
};
template <>
struct PTEnergy<false> {
  using T = uint32_t;
  __device__ static __forceinline__ T shfl(T v, int src) { return __shfl_sync(0xffffffffu, v, src); }
  __device__ static __forceinline__ int diff2(T x, T y) { return 2 * (int)(x - y); }
};

template <bool BY_SLOT, bool CG, bool WIDE>
__device__ __forceinline__ uint32_t pt_chain(int32_t *wa, unsigned long long *Ua, const PTConst *pc,
                                             const double *sq, uint2 key, uint32_t t, int64_t a, int r,
                                             int n_slots) {
  using E = PTEnergy<WIDE>;
  using ET = typename E::T;
  const int lane = threadIdx.x & 31;
  const bool has_pair = lane + 1 < n_slots;
  int w = 0;
  ET us = 0, ut = 0;
  if (lane < n_slots) {
    w = CG ? __ldcg(wa + lane) : wa[lane];
    const int e = BY_SLOT ? lane : w;
    us = (ET)ld_energy<CG>(Ua + 2 * e);
    ut = (ET)ld_energy<CG>(Ua + 2 * e + 1);
  }
  float dk = 0.f, dkt = 0.f, lnu = 0.f;
  uint32_t g = 0, x = 0;
  if (has_pair) {
    dk = pc->dkf[lane];
    dkt = pc->dktf[lane];
#pragma unroll
    for (int k = 0; k < 4; ++k) g |= ((pc->ge1[k] >> lane) & 1u) << k;
    x = pick4(philox(make_uint4((uint32_t)lane, t, (uint32_t)a, (DOM_PT << 28) | (uint32_t)(r >> 2)), key), r & 3);
    lnu = __logf((float)x) - 22.18070977791825f;
  }
  // energies of the original occupant of slot s+1 (the Y of pair s)
  const ET y_us = E::shfl(us, (lane + 1) & 31);
  const ET y_ut = E::shfl(ut, (lane + 1) & 31);
  // The decisions of pair s against candidate i <= s form a triangle,
  // enumerated row by row (f = s (s+1)/2 + i) and taken 32 at a time, one
  // per lane: ceil(n_p (n_p+1) / 64) rounds of independent work for n_p
  // pairs instead of n_p dependent steps of one lane per pair.  Lane r keeps
  // round r's ballots of accepted and of open candidates; row s is then the
  // bits f = s (s+1)/2 .. s (s+1)/2 + s of their concatenation.
  const int n_p = n_slots - 1;
  const int n_tri = n_p * (n_p + 1) / 2;
  uint32_t Mb = 0, Ob = 0;
  for (int r0 = 0; r0 * 32 < n_tri; r0 += 4) {
    // four rounds at a time: every operand gathered first, then the
    // decisions, so the shuffles' latencies overlap (the row of f from the
    // inverse of f = s (s+1)/2 in float, corrected by one either way)
    ET xu[4], xt[4], yu[4], yt[4];
    uint32_t gs[4], xs[4];
    float dks[4], dkts[4], lnus[4];
    bool take[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int f = (r0 + k) * 32 + lane;
      const float q = 8.f * (float)f + 1.f;
      int s = (int)((q * rsqrtf(q) - 1.f) * 0.5f);
      s += (s + 1) * (s + 2) / 2 <= f ? 1 : 0;   // rounding guards
      s -= s * (s + 1) / 2 > f ? 1 : 0;
      take[k] = f < n_tri;
      const int sp = take[k] ? s : 0, ci = take[k] ? f - s * (s + 1) / 2 : 0;
      xu[k] = E::shfl(us, ci);
      xt[k] = E::shfl(ut, ci);
      yu[k] = E::shfl(y_us, sp);
      yt[k] = E::shfl(y_ut, sp);
      gs[k] = __shfl_sync(0xffffffffu, g, sp);
      xs[k] = __shfl_sync(0xffffffffu, x, sp);
      dks[k] = __shfl_sync(0xffffffffu, dk, sp);
      dkts[k] = __shfl_sync(0xffffffffu, dkt, sp);
      lnus[k] = __shfl_sync(0xffffffffu, lnu, sp);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const auto m = E::diff2(xu[k], yu[k]);
      const auto n = E::diff2(xt[k], yt[k]);
      const bool ge =
          (m == 0 || ((gs[k] >> (m > 0 ? 0 : 1)) & 1u)) && (n == 0 || ((gs[k] >> (n > 0 ? 2 : 3)) & 1u));
      const float la = (float)m * dks[k], lb = (float)n * dkts[k];
      const bool ok = xs[k] != 0u && fabsf(la) < 700.f && fabsf(lb) < 700.f;
      const float d = lnus[k] - (la + lb);
      const float err = 1e-4f + (fabsf(la) + fabsf(lb)) * 4.8e-7f;
      const bool lo = ok && d < -err;
      const bool tiny = xs[k] != 0u && la <= 0.f && lb <= 0.f && fminf(la, lb) <= -23.5f;
      const bool und = !ge && !lo && !tiny && !(ok && d > err);
      const uint32_t ma = __ballot_sync(0xffffffffu, take[k] && (ge || lo));
      const uint32_t mo = __ballot_sync(0xffffffffu, take[k] && und);
      if (lane == r0 + k) {
        Mb = ma;
        Ob = mo;
      }
    }
  }
  uint32_t D = 0, open = 0;
  {
    const int f0 = lane * (lane + 1) / 2, k = f0 >> 5;
    const uint32_t a0 = __shfl_sync(0xffffffffu, Mb, k & 31), a1 = __shfl_sync(0xffffffffu, Mb, (k + 1) & 31);
    const uint32_t o0 = __shfl_sync(0xffffffffu, Ob, k & 31), o1 = __shfl_sync(0xffffffffu, Ob, (k + 1) & 31);
    const uint32_t row = lane >= 31 ? 0xffffffffu : (2u << lane) - 1u;   // bits 0 .. lane
    if (has_pair) {
      D = __funnelshift_r(a0, a1, f0 & 31) & row;
      open = __funnelshift_r(o0, o1, f0 & 31) & row;
    }
  }
  while (open) {   // exact rule for the candidates left open (rare)
    const int i = __ffs(open) - 1;
    open &= open - 1;
    const int e = BY_SLOT ? i : (CG ? __ldcg(wa + i) : wa[i]);
    const long long m = 2 * (ld_energy<CG>(Ua + 2 * e) - (long long)y_us);
    const long long n = 2 * (ld_energy<CG>(Ua + 2 * e + 1) - (long long)y_ut);
    if (pt_exact(sq, lane, m >= 0 ? 0 : 1, n >= 0 ? 2 : 3, m, n, x)) D |= 1u << i;
  }
  __syncwarp();
  // the scan in runs of eight pairs: a run's decision words first (shuffles
  // that do not wait on the carried candidate), then its steps in registers
  uint32_t acc = 0;
  int c = 0, mine = lane;   // carried candidate; final occupant of this lane's slot
  for (int s0 = 0; s0 < n_p; s0 += 8) {
    uint32_t Dv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) Dv[k] = __shfl_sync(0xffffffffu, D, (s0 + k) & 31);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int s2 = s0 + k;
      const bool live = s2 < n_p;
      const bool ex = live && ((Dv[k] >> c) & 1u);
      if (live && lane == s2) mine = ex ? s2 + 1 : c;
      acc |= (uint32_t)ex << (s2 & 31);
      if (live && !ex) c = s2 + 1;
    }
  }
  if (lane == n_slots - 1) mine = c;
  const int f_w = __shfl_sync(0xffffffffu, w, mine);
  const ET f_us = E::shfl(us, mine);
  const ET f_ut = E::shfl(ut, mine);
  if (lane < n_slots) {
    wa[lane] = f_w;
    if (BY_SLOT) {
      Ua[2 * lane] = (unsigned long long)f_us;
      Ua[2 * lane + 1] = (unsigned long long)f_ut;
    }
  }
  return acc;
}

// ---- programmatic dependent launch ----
//
// A kernel launched with launch_kernel(pdl = true, ...) may be scheduled
// while the kernel before it on the stream is finishing; it must call
// pdl_begin() before it touches global memory that kernel writes (the wait
// returns once that kernel has completed and its writes are visible; with
// no such dependency it returns at once).  No kernel triggers its
// dependents early: the trigger is each block's exit, so the next kernel is
// launched as the last blocks leave instead of taking SM room while this
// one still runs (the early trigger made the sweep slower than no overlap).
__device__ __forceinline__ void pdl_begin() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                          Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// ---- persistent kernels ----

constexpr long long kBarrierTimeoutNs = 5000000000ll;   // default bound of a grid-barrier wait: 5 s

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch with a bounded wait: bar[0]
// counts arrivals, bar[1] is the generation.  A wait that exceeds wait_ns
// sets *err and gives up; every block checks *err after each barrier and
// leaves (returns false), so the launch always ends.  bar must be zero at
// launch.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int *err, long long wait_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = gtime();
      while (*gen == g) {
        if (*(volatile int *)err) break;
        if (gtime() - t0 > (unsigned long long)wait_ns) {
          atomicExch(err, 1);
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int *)err == 0;
}

// Load through L2 only (CG) where other blocks of the same persistent launch
// wrote the data in an earlier phase (L1 is not coherent across SMs).
template <bool CG, typename T>
__device__ __forceinline__ T ld_g(const T *p) {
  if constexpr (CG)
    return __ldcg(p);
  else
    return *p;
}

// ---- bit-sliced helpers shared by the sweep kernels ----

template <typename Word>
__device__ __forceinline__ Word ones_if(bool b) {
  return b ? ~Word(0) : Word(0);
}

// sel ? a : b, bitwise
template <typename Word>
__device__ __forceinline__ Word mux(Word sel, Word a, Word b) {
  return (sel & a) | (~sel & b);
}

template <typename Word>
__device__ __forceinline__ Word maj3(Word a, Word b, Word c) {
  return (a & b) | (c & (a ^ b));
}

// Bit-sliced per-lane counter: plane p holds bit p of every lane's count.
template <typename Word, int K>
struct VCount {
  Word p[K];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < K; ++i) p[i] = 0;
  }
  // add x0 + 2 x1 + 4 x2 (per lane)
  __device__ __forceinline__ void add3(Word x0, Word x1, Word x2) {
    Word c = p[0] & x0;
    p[0] ^= x0;
    Word s = p[1] ^ x1 ^ c;
    c = maj3(p[1], x1, c);
    p[1] = s;
    s = p[2] ^ x2 ^ c;
    c = maj3(p[2], x2, c);
    p[2] = s;
#pragma unroll
    for (int i = 3; i < K; ++i) {
      const Word t = p[i] & c;
      p[i] ^= c;
      c = t;
    }
  }
  // add x0 + 2 x1
  __device__ __forceinline__ void add2(Word x0, Word x1) {
    Word c = p[0] & x0;
    p[0] ^= x0;
    const Word s = p[1] ^ x1 ^ c;
    c = maj3(p[1], x1, c);
    p[1] = s;
#pragma unroll
    for (int i = 2; i < K; ++i) {
      const Word t = p[i] & c;
      p[i] ^= c;
      c = t;
    }
  }
  // add (a0 + 2 a1 + 4 a2) + (b0 + 2 b1 + 4 b2): the two values are
  // compressed plane by plane before the carry enters the higher planes
  // (15 operations at K = 6 against 24 for two add3 calls)
  __device__ __forceinline__ void add3x2(Word a0, Word a1, Word a2, Word b0, Word b1, Word b2) {
    const Word c1 = maj3(p[0], a0, b0);   // weight 2
    p[0] ^= a0 ^ b0;
    Word s = p[1] ^ a1 ^ b1;
    const Word cA = maj3(p[1], a1, b1), cB = s & c1;   // weight 4
    p[1] = s ^ c1;
    s = p[2] ^ a2 ^ b2;
    const Word d1 = maj3(p[2], a2, b2), d2 = maj3(s, cA, cB);   // weight 8
    p[2] = s ^ cA ^ cB;
    if constexpr (K > 3) {
      Word c = maj3(p[3], d1, d2);
      p[3] ^= d1 ^ d2;
#pragma unroll
      for (int i = 4; i < K; ++i) {
        const Word t = p[i] & c;
        p[i] ^= c;
        c = t;
      }
    }
  }
  // add (a0 + 2 a1) + (b0 + 2 b1), compressed the same way
  __device__ __forceinline__ void add2x2(Word a0, Word a1, Word b0, Word b1) {
    const Word c1 = maj3(p[0], a0, b0);
    p[0] ^= a0 ^ b0;
    const Word s = p[1] ^ a1 ^ b1;
    const Word cA = maj3(p[1], a1, b1), cB = s & c1;
    p[1] = s ^ c1;
    if constexpr (K > 2) {
      Word c = maj3(p[2], cA, cB);
      p[2] ^= cA ^ cB;
#pragma unroll
      for (int i = 3; i < K; ++i) {
        const Word t = p[i] & c;
        p[i] ^= c;
        c = t;
      }
    }
  }
  // add x (one bit per lane)
  __device__ __forceinline__ void add1(Word x) {
    Word c = x;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const Word t = p[i] & c;
      p[i] ^= c;
      c = t;
    }
  }
};

template <typename Word>
__device__ __forceinline__ Word shfl_xor_w(Word v, int m) {
  if (sizeof(Word) == 8) {
    const unsigned long long u = (unsigned long long)v;
    const unsigned lo = __shfl_xor_sync(0xffffffffu, (unsigned)u, m);
    const unsigned hi = __shfl_xor_sync(0xffffffffu, (unsigned)(u >> 32), m);
    return (Word)(((unsigned long long)hi << 32) | lo);
  }
  return (Word)__shfl_xor_sync(0xffffffffu, (unsigned)v, m);
}

template <typename Word>
__device__ __forceinline__ Word shfl_w(Word v, int src) {
  if (sizeof(Word) == 8) {
    const unsigned long long u = (unsigned long long)v;
    const unsigned lo = __shfl_sync(0xffffffffu, (unsigned)u, src);
    const unsigned hi = __shfl_sync(0xffffffffu, (unsigned)(u >> 32), src);
    return (Word)(((unsigned long long)hi << 32) | lo);
  }
  return (Word)__shfl_sync(0xffffffffu, (unsigned)v, src);
}

// Sum a per-thread counter over the warp threads that share (lane % G) and
// add each of the W lanes' totals into acc[key][lane] (shared memory).
// K planes per thread; the warp total needs up to K + 5 planes.  Every
// thread of the warp must call this (full-mask shuffles).
template <typename Word, int K, int G>
__device__ __forceinline__ void flush_counter(const VCount<Word, K> &c, int *acc) {
  constexpr int KT = K + 5;
  constexpr int W = (int)sizeof(Word) * 8;
  Word tot[KT];
#pragma unroll
  for (int i = 0; i < KT; ++i) tot[i] = i < K ? c.p[i] : Word(0);
#pragma unroll
  for (int off = G; off < 32; off <<= 1) {
    Word carry = 0;
#pragma unroll
    for (int i = 0; i < KT; ++i) {
      const Word o = shfl_xor_w(tot[i], off);
      const Word s = tot[i] ^ o ^ carry;
      carry = maj3(tot[i], o, carry);
      tot[i] = s;
    }
  }
  // thread t extracts lanes l = t / G + m * (32 / G) of key t % G from the
  // totals held (identically) by every thread with that key
  const int t = threadIdx.x & 31;
  const int key = t % G;
  Word mine[KT];
#pragma unroll
  for (int i = 0; i < KT; ++i) mine[i] = shfl_w(tot[i], key);
  constexpr int per = W * G / 32;
#pragma unroll
  for (int m = 0; m < per; ++m) {
    const int lane = t / G + m * (32 / G);
    int v = 0;
#pragma unroll
    for (int i = 0; i < KT; ++i) v |= (int)((mine[i] >> lane) & 1u) << i;
    if (v) atomicAdd(&acc[key * W + lane], v);
  }
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
  int tau_ap = 0;   // antiperiodic along tau: the wrap tau bond has the opposite sign
  // set by qisg_pt_given: energies and permutation no longer describe the
  // configurations; sweeps are refused until qisg_set_state
  bool needs_state = false;
  // persistent form (SAMPLES, 32-bit words, PT every sweep): one cooperative
  // launch per run of sweeps between measurements
  bool persistent = false;
  // SAMPLES sweep-path kernels launched with programmatic dependent launch
  bool pdl = true;
  unsigned *d_bar = nullptr;        // grid barrier of the persistent kernel
  long long wait_ns = 5000000000ll; // bound of each barrier wait
  cudaStream_t stream = nullptr;
  size_t mem_budget = 0;
  uint64_t t = 0;          // sweeps done (host mirror of *d_t)
  int64_t n_meas = 0;      // measurements done (host mirror)
  int64_t launches = 0;
  int device = 0;
  int n_sm = 0;
  // SAMPLES sweep schedule per colour (red, blue); none of it changes results.
  // tile: W = 64 and the W = 32 column walk: site groups of 4 per thread
  // quad; W = 32 replica-quad kernel: at most this many sites per thread
  // along tau; W = 32 red pass: threads per site (1: four, 2: two, else
  // one; by default four for lattices with few sites per launch); 0 =
  // default.
  // variant (W = 32 blue pass): 0 the replica-quad kernel, 1 the column walk,
  // 2 the replica-quad kernel bounded to four blocks per SM (no prefetch).
  // The default grid aims at sweep_min_blocks_per_sm blocks of 256 threads
  // per SM.
  int sweep_tile[2] = {0, 0};
  int sweep_variant[2] = {0, 0};
  int blue_occ[2][7] = {};   // resident blocks per SM of the W = 32 blue kernel (variant 0 | 2, 3 .. 9 counter planes)
  int sweep_min_blocks_per_sm = 4;

  // host tables (FP64, built once)
  std::vector<double> k, kt;
  std::vector<uint32_t> T;      // [n_slots][5][3]
  std::vector<double> bases;    // [6][n_slots]: alpha+, alpha-, beta+, beta-, dk, dkt of pair s
  std::vector<double> sq;       // [n_slots-1][4][kSqBits]: b, b^2, b^4, ... of each base

  // LANES geometry: rpw replicas per word, n_groups words per site per sample
  int rpw = 0, n_groups = 0;
  // SAMPLES geometry: n_b words of W samples, n_q groups of 4 replicas
  int64_t n_b = 0;
  int n_q = 0;
  int64_t n_a_pad = 0;          // samples including padding lanes

  // device memory
  void *spins = nullptr;
  size_t spins_bytes = 0;
  // SAMPLES, W = 32: the red pass applies the last PT pass's exchanges while
  // it copies the lattice into the other buffer (spins and spins_alt swap
  // after every red pass); perm_pending: the stored lattice still lacks the
  // exchanges of the last PT pass (its masks are in d_acc)
  bool fused = false;
  // fused mode, 32-bit words: the PT pass runs in the blue pass's last blocks
  // when eligible (pt_folded: it did for the current sweep)
  bool pt_in_blue = true;
  bool pt_folded = false;
  void *spins_alt = nullptr;
  bool perm_pending = false;
  void *J = nullptr;
  size_t J_bytes = 0;
  uint32_t *d_T = nullptr;
  double *d_bases = nullptr;
  double *d_sq = nullptr;           // [n_slots-1][4][kSqBits] squaring chains of the PT bases
  void *d_ptc = nullptr;            // PTConst
  int32_t *d_walker = nullptr;      // [a_pad][r][s]
  unsigned long long *d_U = nullptr;  // LANES: [a][r][w][2] by walker; SAMPLES: [a_pad][r][s][2] by slot
  long long *d_sumA = nullptr, *d_sumB = nullptr, *d_sumq = nullptr, *d_sumq2 = nullptr;
  long long *d_q = nullptr;         // overlap scratch [a][s][pair]
  long long *d_out = nullptr;       // output staging [2][a][r][s]
  unsigned long long *d_t = nullptr;  // sweep counter; d_t[1]: its copy for the PT pass (fused mode)
  void *d_acc = nullptr;            // SAMPLES: PT lane masks of the last pass, Word [b][r][s]
  unsigned long long *d_dcum = nullptr;   // SITES: cumulative tables [n_slots][256]
  uint2 *d_dlut = nullptr;                // SITES: prefix index [n_slots][2^kDaemonLutBits], then the spans (bytes)
  int *d_err = nullptr;
  // records at every measurement (Appendix A): PT walk history and maxit block sums
  int hist_len = 0, maxit = 0, blk_len = 0;
  unsigned long long *d_meas = nullptr;   // measurements taken (device copy of n_meas)
  uint8_t *d_hist = nullptr;              // [hist_len][n_samples][n_rep][n_slots]: slot of each walker
  long long *d_blkA = nullptr, *d_blkB = nullptr;   // [blk_len][n_samples][n_rep][n_slots] by slot
  int64_t rec_base = 0;                   // first measurement the rings hold (checkpoint loads start later)
  size_t device_bytes = 0;

  // launch timing (qisg_profile)
  int prof = 0;                    // bit k: time launches of kernel kind k
  std::vector<cudaEvent_t> prof_ev[5];   // start/stop pairs per internal kernel kind
  int64_t prof_launched[5] = {0, 0, 0, 0, 0};

  // CUDA graph of one sweep cycle (lcm of the PT and measurement cadences),
  // captured on cap_stream and replayed on stream
  bool use_graphs = true;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t cyc_graph = nullptr;
  cudaGraphExec_t cyc_exec = nullptr;
  int cyc_sweeps = 0;
  int64_t cyc_launches = 0, cyc_meas = 0;
  int64_t cyc_prof_launched[5] = {0, 0, 0, 0, 0};
  bool cyc_profiled = false;
  bool cyc_pending = false;         // perm_pending after one replay
  // event-record nodes of a profiled capture: node, kernel kind, 0 start / 1 stop
  std::vector<cudaGraphNode_t> cyc_ev_nodes;
  std::vector<std::pair<int, int>> cyc_ev_kind;
  std::vector<cudaEvent_t> prof_spare;   // untimed events of replays past the pool
  std::vector<cudaEvent_t> cyc_events;   // events referenced by the captured graph

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
int lanes_init_couplings(qisg_handle *h);
int lanes_finalize(qisg_handle *h, int force_to_q);

// SITES packing (sites.cu): the paper's multi-site coding with daemon bits.
int sites_init(qisg_handle *h);
int sites_half_sweep(qisg_handle *h, int colour, int count_only);
int sites_measure(qisg_handle *h, int force_to_q);
int sites_get_spins(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *S);
int sites_set_spins(qisg_handle *h, const int8_t *S);
void daemon_cumulative(double k, uint64_t *cum);

// SAMPLES kernels (samples.cu)
int samples_init(qisg_handle *h);
int samples_half_sweep(qisg_handle *h, int colour, int count_only);
int samples_pt(qisg_handle *h, int explicit_pass, int advance);
int samples_materialize(qisg_handle *h);
int samples_measure(qisg_handle *h, int force_to_q);
int samples_energies_by_slot(qisg_handle *h);
int samples_get_spins(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *S);
int samples_set_spins(qisg_handle *h, const int8_t *S, const int32_t *walker_at, const int8_t *d_S = nullptr);
int samples_upload_checked(qisg_handle *h, const int8_t *S, int64_t n, int8_t **d_S);
int samples_get_couplings(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *J);
int samples_set_couplings(qisg_handle *h, const int8_t *J);
// unpack samples a_lo .. a_lo+n_a-1 by walker into a device int8 buffer
// [n_a][n_rep][n_slots][N] (+-1), on the handle's stream
int lanes_stage_spins(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *d);
int sites_stage_spins(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *d);
int samples_stage_spins(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *d);
// persistent form: n sweeps (red, blue, PT) in one cooperative launch
bool samples_persistent_ok(const qisg_handle *h);
int samples_persistent(qisg_handle *h, int n_sweeps);

// common small kernels (qisg_api.cu)
int advance_counter(qisg_handle *h);
// synchronise the handle's stream and report a device error flag
int handle_sync(qisg_handle *h);

// records of a measurement: walk history and block sums (records.cu)
int record_measurement(qisg_handle *h);

// PT pass of samples a0 .. a0+n_a-1 (pt.cu)
// adv: SAMPLES only, advance the sweep counter after the pass (nullptr: no)
// force_wide: take 64-bit energy differences whatever the lattice size
int pt_pass(qisg_handle *h, int explicit_pass, int64_t a0, int64_t n_a, unsigned long long *adv = nullptr,
            bool force_wide = false);

// Launch timing: call prof_begin(h, kind) before and prof_end(h, kind, tok)
// after a kernel launch on h->stream.  Internal kinds: QISG_KERNEL_SWEEP
// holds the red half sweeps, kProfBlue the blue ones (qisg_profile_read
// reports QISG_KERNEL_SWEEP as their sum).
constexpr int kProfBlue = 4, kProfKinds = 5;
inline int sweep_kind(int colour) { return colour ? kProfBlue : QISG_KERNEL_SWEEP; }
int prof_begin(qisg_handle *h, int kind);
void prof_end(qisg_handle *h, int kind, int tok);

}  // namespace qisg
