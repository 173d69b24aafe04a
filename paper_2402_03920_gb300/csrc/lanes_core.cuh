// Half sweep of one sample in the LANES packing, one thread per site.
//
// A 32- or 64-bit word holds replicas x walkers of the sample: lane =
// (r - g*rpw) * n_slots + w in word group g = r / rpw.  The thread of a site
// loads the site's and its six neighbours' words once, forms the bit-sliced
// counts u_s (4 spatial bonds) and u_t (2 tau bonds) of every lane, and then
// visits every (slot s, replica r): the walker w at slot s of replica r is
// lane (r, w), whose draw R (one Philox call per (slot, replica quad, site,
// sweep)) is compared with the threshold T[s][u_s][u_t] (Sec. 2.1).  Before
// that visit the thread spreads the five count planes into a byte per lane
// in shared memory (the 5-bit class code u_s + 8 u_t, four lanes per word),
// so a lane's class is one load and its threshold one more, from a 32-entry
// row per slot.  The flip mask of the site is built in registers and
// applied once.  In the blue pass
// the unsatisfied bonds after the flip are accumulated per lane in bit-sliced
// counters and flushed per tile (every bond has exactly one blue end).
#pragma once

#include "qisg_internal.cuh"

namespace qisg {

constexpr int kLanesMaxGroups = 2;    // word groups per site held in registers
constexpr int kLanesKs = 7;           // u_s counter planes: <= 4 x 16 sites per thread
constexpr int kLanesKt = 6;           // u_t counter planes: <= 2 x 16 sites per thread
constexpr int kLanesMaxSitesPerThread = 16;
constexpr int kLanesMaxThreads = 256;                    // block size the class-code buffer is sized for
constexpr int kLanesCodeWords = kLanesMaxGroups * 16;    // per thread: 2 groups x 64 lanes, 4 per word

template <typename Word>
struct LanesSample {
  Word *spins;                   // [g][N]
  const uint32_t *T;             // [n_slots][15] (global)
  const int32_t *walker;         // [r][s]
  unsigned long long *U;         // [r][w][2], by walker
  const uint8_t *J;              // [L*L]
  uint2 key;
  uint32_t ctr_w;                // (DOM_SWEEP << 28) | (a >> 6)
  uint32_t t;                    // sweep index
  FastDiv hpd;
  int L, Lt, plane, half_plane, N, n_slots, n_rep, rpw, n_groups;
  int tau_ap;                    // antiperiodic along tau: the wrap tau bond flips sign
};

// Shared memory of one tile: the thresholds by class code, walker labels,
// counter sums, the per-thread class codes and the plane tables.
__host__ __device__ inline size_t lanes_tile_smem(int plane, int n_slots, int n_rep) {
  size_t o = (size_t)(n_slots * 32 + n_rep * n_slots) * 4;   // T5_s, wa_s
  o += (size_t)2 * kLanesMaxGroups * 64 * 4;                  // acc_s, acc_t
  o += (size_t)kLanesCodeWords * kLanesMaxThreads * 4;
  o = (o + 7) & ~size_t(7);
  o += (size_t)plane * (8 + 2 + 1);                           // nb, s2d, Js
  return (o + 15) & ~size_t(15);
}

// Bits 0..3 of x moved to bits 0, 8, 16, 24.
__device__ __forceinline__ uint32_t spread4(uint32_t x) { return ((x & 0xFu) * 0x00204081u) & 0x01010101u; }

template <bool CG, typename Word>
__device__ __forceinline__ Word ld_word(const Word *p) {
  return CG ? __ldcg(p) : *p;
}

// Sites [j0, j0 + n) of one colour; every thread of the block must call it.
// NREP > 0: the sample has exactly NREP replicas (a compile-time count lets
// the per-slot replica loop unroll without bound checks).  NGC > 0: exactly
// NGC word groups per site (registers for those only).
// CG: read mutable state through L2 only (inside a persistent kernel).
// zero_U: clear this sample's bond counters first (red pass, one tile).
template <typename Word, bool CG, bool BLUE, int NREP = 0, int NGC = 0>
__device__ void lanes_tile(const LanesSample<Word> &S, int colour, int j0, int n, int count_only, bool zero_U,
                           unsigned char *smem) {
  constexpr int W = (int)sizeof(Word) * 8;
  const int n_slots = S.n_slots, n_rep = NREP > 0 ? NREP : S.n_rep, plane = S.plane, hp = S.half_plane;
  uint32_t *T5_s = reinterpret_cast<uint32_t *>(smem);   // [slot][code], code = u_s + 8 u_t
  int *wa_s = reinterpret_cast<int *>(T5_s + n_slots * 32);
  int *acc_s = wa_s + n_rep * n_slots;                 // [group][lane]
  int *acc_t = acc_s + kLanesMaxGroups * 64;
  uint32_t *code_s = reinterpret_cast<uint32_t *>(acc_t + kLanesMaxGroups * 64);   // [word][thread]
  size_t off = (size_t)(n_slots * 32 + n_rep * n_slots) * 4 + (size_t)2 * kLanesMaxGroups * 64 * 4 +
               (size_t)kLanesCodeWords * kLanesMaxThreads * 4;
  off = (off + 7) & ~size_t(7);
  uint2 *nb = reinterpret_cast<uint2 *>(smem + off);
  uint16_t *s2d = reinterpret_cast<uint16_t *>(nb + plane);
  uint8_t *Js = reinterpret_cast<uint8_t *>(s2d + plane);

  __syncthreads();   // a previous tile is done with shared memory
  for (int i = threadIdx.x; i < n_slots * 32; i += blockDim.x) {
    const int sl = i >> 5, us = i & 7, ut = (i >> 3) & 3;
    T5_s[i] = (us <= 4 && ut <= 2) ? S.T[sl * 15 + us * 3 + ut] : 0xFFFFFFFFu;
  }
  for (int i = threadIdx.x; i < n_rep * n_slots; i += blockDim.x) wa_s[i] = CG ? __ldcg(S.walker + i) : S.walker[i];
  if (BLUE)
    for (int i = threadIdx.x; i < 2 * kLanesMaxGroups * 64; i += blockDim.x) acc_s[i] = 0;
  for (int i2 = threadIdx.x; i2 < plane; i2 += blockDim.x) {
    const int L = S.L;
    const int y = i2 / L, x = i2 - y * L;
    const int xp = x + 1 == L ? 0 : x + 1, xm = x == 0 ? L - 1 : x - 1;
    const int yp = y + 1 == L ? 0 : y + 1, ym = y == 0 ? L - 1 : y - 1;
    nb[i2] = make_uint2((uint32_t)(xp + L * y) | ((uint32_t)(xm + L * y) << 16),
                        (uint32_t)(x + L * yp) | ((uint32_t)(x + L * ym) << 16));
    s2d[((x + y) & 1) * hp + (i2 >> 1)] = (uint16_t)i2;
    Js[i2] = S.J[i2];
  }
  if (zero_U)
    for (int i = threadIdx.x; i < 2 * n_rep * n_slots; i += blockDim.x) S.U[i] = 0;
  __syncthreads();

  constexpr int MG = NGC > 0 ? NGC : kLanesMaxGroups;   // word groups held in registers
  const int NG = NGC > 0 ? NGC : S.n_groups;             // 1 or 2
  const uint32_t Lt = (uint32_t)S.Lt;
  VCount<Word, kLanesKs> cs[MG];
  VCount<Word, kLanesKt> ct[MG];
  if (BLUE)
#pragma unroll
    for (int g = 0; g < MG; ++g) {
      cs[g].zero();
      ct[g].zero();
    }

  for (int base = 0; base < n; base += blockDim.x) {
    const int jr = base + threadIdx.x;
    if (jr < n) {
      const uint32_t j = (uint32_t)(j0 + jr);
      const uint32_t tau = S.hpd.div(j);
      const uint32_t i2 = s2d[((colour + tau) & 1) * hp + (j - tau * hp)];
      const uint2 nv = nb[i2];
      const uint32_t offt = tau * plane;
      const uint32_t site = i2 + offt;
      const uint32_t i_xp = (nv.x & 0xFFFFu) + offt, i_xm = (nv.x >> 16) + offt;
      const uint32_t i_yp = (nv.y & 0xFFFFu) + offt, i_ym = (nv.y >> 16) + offt;
      const uint32_t i_tp = i2 + (tau + 1 == Lt ? 0u : offt + plane);
      const uint32_t i_tm = i2 + (tau == 0 ? (Lt - 1) * plane : offt - plane);
      // the antiperiodic wrap bond is unsatisfied when its spins agree
      const Word gtp = ones_if<Word>(S.tau_ap && tau + 1 == Lt), gtm = ones_if<Word>(S.tau_ap && tau == 0);
      const uint8_t jh = Js[i2];
      const Word Jxp = ones_if<Word>(jh & 1u), Jyp = ones_if<Word>(jh & 2u);
      const Word Jxm = ones_if<Word>(Js[nv.x >> 16] & 1u);
      const Word Jym = ones_if<Word>(Js[nv.y >> 16] & 2u);
      Word sc[MG], P0[MG], P1[MG], P2[MG], Q0[MG], Q1[MG], fw[MG];
#pragma unroll
      for (int g = 0; g < MG; ++g) {
        sc[g] = P0[g] = P1[g] = P2[g] = Q0[g] = Q1[g] = fw[g] = 0;
        if (g < NG) {
          const Word *w = S.spins + (size_t)g * S.N;
          const Word c = ld_word<CG>(w + site);
          const Word b1 = c ^ ld_word<CG>(w + i_xp) ^ Jxp;
          const Word b2 = c ^ ld_word<CG>(w + i_xm) ^ Jxm;
          const Word b3 = c ^ ld_word<CG>(w + i_yp) ^ Jyp;
          const Word b4 = c ^ ld_word<CG>(w + i_ym) ^ Jym;
          const Word t1 = c ^ ld_word<CG>(w + i_tp) ^ gtp;
          const Word t2 = c ^ ld_word<CG>(w + i_tm) ^ gtm;
          const Word s1 = b1 ^ b2 ^ b3, c1 = maj3(b1, b2, b3);
          sc[g] = c;
          P0[g] = s1 ^ b4;
          const Word c2 = s1 & b4;
          P1[g] = c1 ^ c2;
          P2[g] = c1 & c2;
          Q0[g] = t1 ^ t2;
          Q1[g] = t1 & t2;
        }
      }
      if (!count_only) {
        // class codes of every lane, a byte each: word g*16 + l/4 of this
        // thread holds lanes l .. l+3 of group g
        uint32_t *cw = code_s + threadIdx.x;
#pragma unroll
        for (int g = 0; g < MG; ++g)
          if (g < NG) {
#pragma unroll
            for (int h = 0; h < W / 32; ++h) {
              const uint32_t a0 = (uint32_t)(P0[g] >> (32 * h)), a1 = (uint32_t)(P1[g] >> (32 * h));
              const uint32_t a2 = (uint32_t)(P2[g] >> (32 * h)), a3 = (uint32_t)(Q0[g] >> (32 * h));
              const uint32_t a4 = (uint32_t)(Q1[g] >> (32 * h));
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const uint32_t c = spread4(a0 >> (4 * i)) | (spread4(a1 >> (4 * i)) << 1) |
                                   (spread4(a2 >> (4 * i)) << 2) | (spread4(a3 >> (4 * i)) << 3) |
                                   (spread4(a4 >> (4 * i)) << 4);
                cw[(g * 16 + h * 8 + i) * kLanesMaxThreads] = c;
              }
            }
          }
        for (int s = 0; s < n_slots; ++s) {
          const uint32_t *Trow = T5_s + s * 32;
          for (int q = 0; 4 * q < n_rep; ++q) {
            const uint4 R4 = philox(make_uint4(site, S.t, (uint32_t)s | ((uint32_t)q << 16), S.ctr_w), S.key);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
              const int r = 4 * q + jj;
              if (r >= n_rep) break;
              const int g = (MG > 1 && r >= S.rpw) ? 1 : 0;   // n_groups <= 2
              const int lane = (r - g * S.rpw) * n_slots + wa_s[r * n_slots + s];
              const uint32_t word = cw[(g * 16 + (lane >> 2)) * kLanesMaxThreads];
              const uint32_t thr = Trow[(word >> (8 * (lane & 3))) & 31u];
              if (thr == 0xFFFFFFFFu || pick4(R4, jj) < thr) {
                if (MG > 1 && g) fw[MG - 1] |= Word(1) << lane;
                else fw[0] |= Word(1) << lane;
              }
            }
          }
        }
#pragma unroll
        for (int g = 0; g < MG; ++g)
          if (g < NG && fw[g]) {
            Word *w = S.spins + (size_t)g * S.N + site;
            *w = sc[g] ^ fw[g];
          }
      }
      if (BLUE) {
#pragma unroll
        for (int g = 0; g < MG; ++g)
          if (g < NG) {
            // unsatisfied counts after the flip: u -> 4 - u (spatial), 2 - u (tau)
            const Word f = fw[g];
            const Word v1 = P1[g] ^ (f & P0[g]);
            const Word v2 = mux(f, ~(P0[g] | P1[g] | P2[g]), P2[g]);
            const Word w1 = mux(f, ~(Q0[g] | Q1[g]), Q1[g]);
            cs[g].add3(P0[g], v1, v2);
            ct[g].add2(Q0[g], w1);
          }
      }
    }
  }
  if (BLUE) {
#pragma unroll
    for (int g = 0; g < MG; ++g)
      if (g < NG) {   // uniform across the block
        flush_counter<Word, kLanesKs, 1>(cs[g], acc_s + g * W);
        flush_counter<Word, kLanesKt, 1>(ct[g], acc_t + g * W);
      }
    __syncthreads();
    for (int i = threadIdx.x; i < NG * W; i += blockDim.x) {
      const int g = i / W, lane = i - g * W;
      const int rl = lane / n_slots, w = lane - rl * n_slots;
      const int r = g * S.rpw + rl;
      if (rl >= S.rpw || r >= n_rep) continue;
      unsigned long long *u = S.U + ((size_t)r * n_slots + w) * 2;
      if (acc_s[i]) atomicAdd(u, (unsigned long long)acc_s[i]);
      if (acc_t[i]) atomicAdd(u + 1, (unsigned long long)acc_t[i]);
    }
  }
}

}  // namespace qisg
