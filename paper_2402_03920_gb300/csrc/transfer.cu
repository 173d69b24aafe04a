// The transfer-matrix product of the exact-diagonalisation code (Sec. 2.2,
// Eq. (transfer-matrix); Appendix D), on one GPU for L <= 5: out = T in on
// the even or odd parity sector, vectors of 2^{L^2-1} doubles indexed by the
// parity-aware basis |n>_{e,o}.
//
//   psi[n] = in[n] w[n];   rounds j = 0 .. L^2-2: psi[n] <- jP psi[n] + jM psi[n ^ 2^j];
//   last factor (Eq. (lr)): psi[n] <- jP psi[n] + parity jM psi[2^{L^2-1} - 1 - n];
//   out[n] = psi[n] w[n],
// with w[n] = exp((k/2) sum_bonds J S S) of n read as an L^2-bit spin
// configuration (top bit 0), jP = e^{k_tau} / (e^{k_tau} + e^{-k_tau}) and
// jM = e^{-k_tau} / (...)  (Eq. (expH1) with exp(-2 k_tau) = tanh(k Gamma)).
//
// On this GPU the work is bound by FP64 issue, not by HBM (about 1.25 TFLOP/s
// of FP64 against 6.7 TB/s): since jP + jM = 1, a round's pair update is
// d = x - y, x' = y + jP d, y' = x - jP d, one subtraction and two fused
// multiply-adds for two elements instead of four multiplies and two adds.
// That is the paper's formula rearranged, so the result differs from the
// plain evaluation by rounding only (relative 1e-15 in norm after 25
// rounds).  Rounds are fused in shared-memory tiles so that the vector
// crosses HBM once per pass instead of once per round: a tile
// fixes all index bits except a low run [0, c) (c = 5: 32 consecutive
// doubles, 256-byte segments) and the bits [lo, hi) of the pass's rounds;
// the first pass takes bits [0, 12) whole.  The last pass pairs every tile
// with its bit complement (the tile holding 2^{n} - 1 - n for each n) for
// the parity factor.  w is not stored: each thread computes the bond energy
// of its index with bit rotations and popcounts and looks exp((k/2) E) up in
// a table of the 2 L^2 + 1 possible energies, computed once on the host in
// FP64.  Rounds run in ascending j for every element, as in the paper.
#include <cmath>
#include <vector>

#include "qisg_internal.cuh"

namespace qisg {
namespace {

constexpr int kTransferBlock = 256;
constexpr int kTileLog = 12;   // 4096 doubles, 32 KB of shared memory

struct TransferArgs {
  double jP, jM, parity;
  double wtab[51];            // exp((k/2) E) for E = -2 L^2, -2 L^2 + 2, ..., 2 L^2 (L <= 5)
  int L2;                     // L^2
  int sumJ;                   // sum of the couplings
  uint32_t row_last;          // sites with x1 = L-1
  uint32_t not_row_last;      // sites with x1 < L-1 within the lattice
  uint32_t col_last;          // sites with x2 = L-1
  uint32_t not_col_last;      // sites with x2 < L-1
  uint32_t jxp, jxn, jyp, jyn;   // bonds to +x / +y with J = +1 / -1
  int L;
};

// exp((k/2) E(n)) for the L^2-bit configuration n (bit i set <=> S_i = -1):
// E = sum_bonds J S S = sum J - 2 (sum of J over unsatisfied bonds).
__device__ __forceinline__ double boltzmann(const TransferArgs &a, uint32_t n) {
  const int L = a.L;
  const uint32_t vx = ((n >> 1) & a.not_row_last) | ((n << (L - 1)) & a.row_last);          // spin at (x1+1, x2)
  const uint32_t vy = ((n >> L) & a.not_col_last) | ((n << (L * (L - 1))) & a.col_last);    // spin at (x1, x2+1)
  const uint32_t ux = n ^ vx, uy = n ^ vy;                                                    // unsatisfied bonds
  const int s = __popc(ux & a.jxp) - __popc(ux & a.jxn) + __popc(uy & a.jyp) - __popc(uy & a.jyn);
  const int E = a.sumJ - 2 * s;
  return a.wtab[(E + 2 * a.L2) >> 1];
}

// Global index of tile element t: bits [0, c) of t -> bits [0, c), the next
// (hi - lo) bits -> bits [lo, hi), the fixed bits f -> [c, lo) then [hi, n).
__device__ __forceinline__ uint32_t tile_index(uint32_t t, uint32_t f, int c, int lo, int hi) {
  const uint32_t low = t & ((1u << c) - 1u);
  const uint32_t mid = t >> c;
  const uint32_t f_lo = f & ((1u << (lo - c)) - 1u);   // bits [c, lo)
  const uint32_t f_hi = f >> (lo - c);                  // bits [hi, n)
  return low | (f_lo << c) | (mid << lo) | (f_hi << hi);
}

// Rounds j in [lo, hi) (tile bit c + j - lo) on the tile in shared memory.
__device__ __forceinline__ void tile_rounds(double *v, int T_log, int c, int lo, int hi, double jP, double jM) {
  const int half = 1 << (T_log - 1);
  for (int j = lo; j < hi; ++j) {
    const int tb = c + (j - lo);
    for (int p = threadIdx.x; p < half; p += blockDim.x) {
      const int t0 = ((p >> tb) << (tb + 1)) | (p & ((1 << tb) - 1));
      const int t1 = t0 | (1 << tb);
      const double x = v[t0], y = v[t1];
      const double d = __dsub_rn(x, y);
      v[t0] = __fma_rn(jP, d, y);      // jP x + jM y with jM = 1 - jP
      v[t1] = __fma_rn(-jP, d, x);     // jP y + jM x
    }
    __syncthreads();
  }
}

// One pass over the rounds [lo, hi).  first: multiply by w on load.  last:
// the parity factor and the multiply by w follow; the block then holds the
// tile of fixed bits f and its complement (or, with no fixed bits, the
// whole vector in one tile).
__global__ void __launch_bounds__(kTransferBlock) transfer_pass_kernel(const double *__restrict__ src, double *dst,
                                                                       const TransferArgs a, int c, int lo, int hi,
                                                                       int n_fixed_bits, int first, int last) {
  extern __shared__ double tile[];
  const int T_log = c + (hi - lo);
  const int T = 1 << T_log;
  const uint32_t nF = 1u << n_fixed_bits;
  const bool pair = last && n_fixed_bits > 0;
  const uint32_t f = blockIdx.x;
  const uint32_t fc = nF - 1u - f;   // complement tile (pair mode: f < fc)
  double *A = tile, *B = tile + T;
  for (int t = threadIdx.x; t < T; t += blockDim.x) {
    const uint32_t i = tile_index((uint32_t)t, f, c, lo, hi);
    const double x = src[i];
    A[t] = first ? __dmul_rn(x, boltzmann(a, i)) : x;
    if (pair) {
      const uint32_t ib = tile_index((uint32_t)t, fc, c, lo, hi);
      const double y = src[ib];
      B[t] = first ? __dmul_rn(y, boltzmann(a, ib)) : y;
    }
  }
  __syncthreads();
  tile_rounds(A, T_log, c, lo, hi, a.jP, a.jM);
  if (pair) tile_rounds(B, T_log, c, lo, hi, a.jP, a.jM);
  if (last) {
    const double pjM = __dmul_rn(a.parity, a.jM);
    if (pair) {
      // element t of A pairs with element T-1-t of B (all index bits inverted)
      for (int t = threadIdx.x; t < T; t += blockDim.x) {
        const double x = A[t], y = B[T - 1 - t];
        const uint32_t ia = tile_index((uint32_t)t, f, c, lo, hi);
        const uint32_t ib = tile_index((uint32_t)(T - 1 - t), fc, c, lo, hi);
        dst[ia] = __dmul_rn(__dadd_rn(__dmul_rn(a.jP, x), __dmul_rn(pjM, y)), boltzmann(a, ia));
        dst[ib] = __dmul_rn(__dadd_rn(__dmul_rn(a.jP, y), __dmul_rn(pjM, x)), boltzmann(a, ib));
      }
    } else {
      // one tile holds the whole vector: element t pairs with T-1-t
      for (int t = threadIdx.x; t < T / 2; t += blockDim.x) {
        const double x = A[t], y = A[T - 1 - t];
        const uint32_t ia = tile_index((uint32_t)t, f, c, lo, hi);
        const uint32_t ib = tile_index((uint32_t)(T - 1 - t), f, c, lo, hi);
        dst[ia] = __dmul_rn(__dadd_rn(__dmul_rn(a.jP, x), __dmul_rn(pjM, y)), boltzmann(a, ia));
        dst[ib] = __dmul_rn(__dadd_rn(__dmul_rn(a.jP, y), __dmul_rn(pjM, x)), boltzmann(a, ib));
      }
    }
  } else {
    for (int t = threadIdx.x; t < T; t += blockDim.x) dst[tile_index((uint32_t)t, f, c, lo, hi)] = A[t];
  }
}

struct Pass {
  int lo, hi, c;
};

// Passes over the rounds: the first takes bits [0, 12) whole; later ones a
// 32-element run of low bits and up to 12 - 5 round bits; the last pass
// holds a tile and its complement, so its tile is at most half as large.
std::vector<Pass> plan_passes(int nb) {
  std::vector<Pass> out;
  int lo = 0;
  while (lo < nb) {
    const int c = lo == 0 ? 0 : (lo < 5 ? lo : 5);
    int w = std::min(nb - lo, kTileLog - c);
    if (lo + w == nb && c + w < nb) w = std::min(w, kTileLog - 1 - c);   // paired tiles
    out.push_back(Pass{lo, lo + w, c});
    lo += w;
  }
  return out;
}

}  // namespace
}  // namespace qisg

using namespace qisg;

extern "C" int qisg_transfer_matvec(const double *in, double *out, int L, double k, double k_tau, const int8_t *J,
                                    int parity, void *cuda_stream) {
  if (!in || !out || !J) return fail(QISG_EINVAL, "NULL argument");
  if (L < 2 || L > 5) return fail(QISG_EINVAL, "transfer matvec takes 2 <= L <= 5 on one GPU");
  if (parity != 1 && parity != -1) return fail(QISG_EINVAL, "parity must be +1 (even) or -1 (odd)");
  if (!std::isfinite(k) || !std::isfinite(k_tau) || k < 0 || k_tau < 0)
    return fail(QISG_EINVAL, "couplings must be finite and >= 0");
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 7u)
    return fail(QISG_EINVAL, "vectors must be 8-byte aligned");
  const int L2 = L * L, nb = L2 - 1;
  TransferArgs a{};
  const double ek = std::exp(k_tau), emk = std::exp(-k_tau);
  a.jP = ek / (ek + emk);
  a.jM = emk / (ek + emk);
  a.parity = (double)parity;
  for (int e = -2 * L2, i = 0; e <= 2 * L2; e += 2, ++i) a.wtab[i] = std::exp(0.5 * k * (double)e);
  a.L2 = L2;
  a.L = L;
  for (int x2 = 0; x2 < L; ++x2)
    for (int x1 = 0; x1 < L; ++x1) {
      const int i = x1 + L * x2;
      const int jx = J[2 * i], jy = J[2 * i + 1];
      if ((jx != 1 && jx != -1) || (jy != 1 && jy != -1)) return fail(QISG_EINVAL, "couplings must be +-1");
      a.sumJ += jx + jy;
      (x1 == L - 1 ? a.row_last : a.not_row_last) |= 1u << i;
      (x2 == L - 1 ? a.col_last : a.not_col_last) |= 1u << i;
      (jx > 0 ? a.jxp : a.jxn) |= 1u << i;
      (jy > 0 ? a.jyp : a.jyn) |= 1u << i;
    }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  const std::vector<Pass> plan = plan_passes(nb);
  int rc = QISG_OK;
  for (size_t p = 0; p < plan.size() && !rc; ++p) {
    const Pass &q = plan[p];
    const int width = q.c + (q.hi - q.lo);
    const int fixed = nb - width;
    const bool last = p + 1 == plan.size();
    const unsigned blocks = (unsigned)((last && fixed > 0) ? (1u << (fixed - 1)) : (1u << fixed));
    const size_t smem = (size_t)((last && fixed > 0) ? 2 : 1) << width;
    transfer_pass_kernel<<<blocks, kTransferBlock, smem * sizeof(double), st>>>(
        p == 0 ? in : out, out, a, q.c, q.lo, q.hi, fixed, p == 0, last);
    rc = cuda_check(cudaGetLastError(), "transfer matvec");
  }
  return rc;
}
