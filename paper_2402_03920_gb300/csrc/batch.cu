// Batched form: many independent single-sample instances of uneven size
// (L, L_tau, ladder length, Gamma, seed) advanced together by ONE persistent
// kernel per chunk of sweeps.
//
// Every instance uses the LANES packing (a 64-bit word holds its replicas x
// walkers; Sec. 2.1 multispin coding) and its own counters, so its trajectory
// is the one qisg_create would give for the same parameters (sample 0).  The
// persistent kernel walks a work-list of (instance, colour-site range) tiles
// for the red and the blue half sweep, then one warp per (instance, replica)
// chain for the PT pass (Sec. 2.1), then advances each instance's sweep
// counter; grid-wide barriers with a bounded wait separate the phases.  The
// launch is cooperative, so all blocks are resident.
//
// Device memory comes from one arena (the batch's memory budget) managed by
// a first-fit allocator on the host; instances are admitted into free slots
// and retired when done, which is what the serving loop builds on.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "lanes_core.cuh"
#include "qisg_internal.cuh"

namespace qisg {
namespace {

constexpr int kBatchBlock = 256;
static_assert(kBatchBlock <= kLanesMaxThreads, "the LANES class-code buffer holds kLanesMaxThreads threads");

struct InstDev {
  unsigned long long *spins;   // [g][site]
  const uint8_t *J;            // [L*L] bit0: J(+x) = -1, bit1: J(+y) = -1
  const uint32_t *T;           // [n_slots][15]
  const PTConst *ptc;
  const double *sq;
  int32_t *walker;             // [r][s]
  unsigned long long *U;       // [r][w][2]
  unsigned long long t;        // sweeps done (mutable)
  long long remaining;         // sweeps left; < 0: no limit (mutable)
  uint2 key;
  FastDiv hpd;
  int L, Lt, plane, half_plane, n_slots, n_rep, rpw, n_groups, spb, N;
  int tau_ap;   // antiperiodic along tau: the wrap tau bond flips sign
  int active;
};

struct Tile {
  int inst, j0, n;   // colour-site range [j0, j0 + n) of one instance
};

struct ChainRef {
  int inst, r;
};

// One tile of a half sweep of instance I (sample 0, 64-bit LANES words).
template <bool BLUE>
__device__ void batch_tile(const InstDev &I, int colour, int j0, int n, unsigned char *smem) {
  LanesSample<unsigned long long> S;
  S.spins = I.spins;
  S.T = I.T;
  S.walker = I.walker;
  S.U = I.U;
  S.J = I.J;
  S.key = I.key;
  S.ctr_w = DOM_SWEEP << 28;   // sample 0: sample block 0
  S.t = (uint32_t)__ldcg(&I.t);
  S.hpd = I.hpd;
  S.L = I.L;
  S.Lt = I.Lt;
  S.plane = I.plane;
  S.half_plane = I.half_plane;
  S.N = I.N;
  S.n_slots = I.n_slots;
  S.n_rep = I.n_rep;
  S.rpw = I.rpw;
  S.n_groups = I.n_groups;
  S.tau_ap = I.tau_ap;
  if (I.n_rep == 4)   // the common case (every uneven-batch and serving instance): loops unrolled
    lanes_tile<unsigned long long, true, BLUE, 4>(S, colour, j0, n, 0, colour == 0 && j0 == 0, smem);
  else
    lanes_tile<unsigned long long, true, BLUE>(S, colour, j0, n, 0, colour == 0 && j0 == 0, smem);
}

__device__ __forceinline__ bool live(const InstDev &I) { return I.active && __ldcg(&I.remaining) != 0; }

// The persistent kernel: n_sweeps x (red tiles | barrier | blue tiles |
// barrier | PT chains | barrier | advance | barrier).  Block b takes the
// contiguous tile range [bstart[b], bstart[b+1]) (ranges of about equal cost).
// The tiles are bound by memory latency, so the kernel is held to the
// registers of three blocks per SM: the extra resident warps outweigh the
// spills of the blue tile's counters (measured: 4.30 -> 3.47 ps/update on the
// 512-instance uneven batch, where two blocks per SM fit without the bound).
__global__ void __launch_bounds__(kBatchBlock, 3) batch_kernel(InstDev *insts, int n_inst, const Tile *tiles,
                                                            int n_tiles, const int *bstart, const ChainRef *chains,
                                                            int n_chains, int n_sweeps, unsigned *bar, int *err,
                                                            long long wait_ns) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t lo = bstart[blockIdx.x];
  const int64_t hi = bstart[blockIdx.x + 1];
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int sw = 0; sw < n_sweeps; ++sw) {
    for (int colour = 0; colour < 2; ++colour) {
      for (int64_t k = lo; k < hi; ++k) {
        const Tile tl = tiles[k];
        const InstDev &I = insts[tl.inst];
        if (!live(I)) continue;
        if (colour == 0)
          batch_tile<false>(I, 0, tl.j0, tl.n, smem);
        else
          batch_tile<true>(I, 1, tl.j0, tl.n, smem);
      }
      if (!grid_barrier(bar, err, wait_ns)) return;
    }
    for (int c = gwarp; c < n_chains; c += warps) {
      const ChainRef cr = chains[c];
      const InstDev &I = insts[cr.inst];
      if (!live(I)) continue;
      pt_chain<false, true, true>(I.walker + cr.r * I.n_slots, I.U + (size_t)cr.r * I.n_slots * 2, I.ptc, I.sq,
                                  I.key, (uint32_t)__ldcg(&I.t), 0, cr.r, I.n_slots);
    }
    if (!grid_barrier(bar, err, wait_ns)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_inst; i += gridDim.x * blockDim.x) {
      InstDev &I = insts[i];
      const long long rem = __ldcg(&I.remaining);
      if (I.active && rem != 0) {
        I.t = __ldcg(&I.t) + 1ull;
        if (rem > 0) I.remaining = rem - 1;
      }
    }
    if (!grid_barrier(bar, err, wait_ns)) return;
  }
}

// Start state of instance I (sample 0): J and spins from Philox.
__global__ void batch_init_kernel(InstDev *insts, int i) {
  const InstDev &I = insts[i];
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c < I.plane) {
    uint8_t v = 0;
    for (uint32_t dir = 0; dir < 2; ++dir) {
      const uint4 x = philox(make_uint4((uint32_t)c, dir, 0u, DOM_J << 28), I.key);
      if (!(x.x & 1u)) v |= (uint8_t)(1u << dir);
    }
    const_cast<uint8_t *>(I.J)[c] = v;
  }
  if (c < (int64_t)I.n_groups * I.N) {
    const int64_t site = c % I.N;
    const int g = (int)(c / I.N);
    unsigned long long v = 0;
    const int r_lo = g * I.rpw, r_hi = min(I.n_rep, r_lo + I.rpw);
    for (int r = r_lo; r < r_hi; ++r)
      for (int w = 0; w < I.n_slots; ++w) {
        const uint4 x = philox(make_uint4((uint32_t)site, (uint32_t)w, 0u, (DOM_INIT << 28) | (uint32_t)r), I.key);
        if (!(x.x & 1u)) v |= 1ull << ((r - r_lo) * I.n_slots + w);
      }
    I.spins[c] = v;
  }
  if (c < (int64_t)I.n_rep * I.n_slots) I.walker[c] = (int32_t)(c % I.n_slots);
  if (c < (int64_t)I.n_rep * I.n_slots * 2) I.U[c] = 0;
}

// First-fit allocator over the arena [0, size), 256-byte granules.
class Arena {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
  }
  bool alloc(size_t bytes, size_t *off) {
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it)
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t free_bytes() const {
    size_t s = 0;
    for (auto &kv : free_) s += kv.second;
    return s;
  }

 private:
  std::map<size_t, size_t> free_;
};

struct Slot {
  bool used = false;
  qisg_instance_desc d{};
  std::vector<qisg_slot> ladder;
  size_t off = 0, bytes = 0;
  uint64_t done = 0;            // sweeps done (host mirror)
  InstDev dev{};
};

}  // namespace
}  // namespace qisg

struct qisg_batch {
  cudaStream_t stream = nullptr;
  int device = 0, n_sm = 0;
  size_t budget = 0;
  unsigned char *arena = nullptr;
  qisg::Arena alloc;
  int capacity = 0;
  std::vector<qisg::Slot> slots;
  qisg::InstDev *d_inst = nullptr;
  qisg::Tile *d_tiles = nullptr;
  size_t tiles_cap = 0;
  int *d_bstart = nullptr;   // first tile of each block (grid + 1 entries)
  size_t bstart_cap = 0;
  int n_tiles = 0;
  qisg::ChainRef *d_chains = nullptr;
  size_t chains_cap = 0;
  int n_chains = 0;
  unsigned *d_bar = nullptr;
  int *d_err = nullptr;
  bool dirty = true;
  int tile_rows = 4;      // rows of spb sites per tile
  int schedule = 0;       // 0: instance order; 1: largest instances first
  int grid = 0;
  size_t smem = 0;
  int max_plane = 4, max_slots = 1, max_rep = 1, max_spb_groups = 1;
  int64_t launches = 0;
  long long wait_ns = qisg::kBarrierTimeoutNs;   // bound of each grid-barrier wait
};

using namespace qisg;

namespace {

int build_tables(qisg_batch *B) {
  std::vector<Tile> tiles;
  std::vector<ChainRef> chains;
  std::vector<int> order;
  for (int i = 0; i < B->capacity; ++i)
    if (B->slots[i].used) order.push_back(i);
  if (B->schedule == 1)
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      return B->slots[a].dev.N * (int64_t)B->slots[a].dev.n_slots > B->slots[b].dev.N * (int64_t)B->slots[b].dev.n_slots;
    });
  B->max_plane = 4;
  B->max_slots = B->max_rep = B->max_spb_groups = 1;
  for (int i : order) {
    const InstDev &I = B->slots[i].dev;
    const int per = kBatchBlock * B->tile_rows;
    const int half = I.N / 2;
    for (int j0 = 0; j0 < half; j0 += per) tiles.push_back(Tile{i, j0, std::min(per, half - j0)});
    for (int r = 0; r < I.n_rep; ++r) chains.push_back(ChainRef{i, r});
    B->max_plane = std::max(B->max_plane, I.plane);
    B->max_slots = std::max(B->max_slots, I.n_slots);
    B->max_rep = std::max(B->max_rep, I.n_rep);
    B->max_spb_groups = std::max(B->max_spb_groups, I.spb * I.n_groups);
  }
  int rc = QISG_OK;
  if (tiles.size() > B->tiles_cap) {
    if (B->d_tiles) cudaFree(B->d_tiles);
    B->d_tiles = nullptr;
    B->tiles_cap = std::max<size_t>(tiles.size(), 2 * B->tiles_cap);
    rc = cuda_check(cudaMalloc(&B->d_tiles, B->tiles_cap * sizeof(Tile)), "tile table");
  }
  if (!rc && chains.size() > B->chains_cap) {
    if (B->d_chains) cudaFree(B->d_chains);
    B->d_chains = nullptr;
    B->chains_cap = std::max<size_t>(chains.size(), 2 * B->chains_cap);
    rc = cuda_check(cudaMalloc(&B->d_chains, B->chains_cap * sizeof(ChainRef)), "chain table");
  }
  if (!rc && !tiles.empty())
    rc = cuda_check(cudaMemcpyAsync(B->d_tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice,
                                    B->stream),
                    "copy tiles");
  if (!rc && !chains.empty())
    rc = cuda_check(cudaMemcpyAsync(B->d_chains, chains.data(), chains.size() * sizeof(ChainRef),
                                    cudaMemcpyHostToDevice, B->stream),
                    "copy chains");
  if (rc) return rc;
  B->n_tiles = (int)tiles.size();
  B->n_chains = (int)chains.size();
  B->smem = lanes_tile_smem(B->max_plane, B->max_slots, B->max_rep);
  if (B->smem > 200 * 1024) return fail(QISG_EINVAL, "instance too large for the batch kernel's shared memory");
  cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B->smem);
  int per_sm = 0;
  rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, kBatchBlock, B->smem),
                  "occupancy");
  if (rc) return rc;
  if (per_sm < 1) return fail(QISG_EINVAL, "batch kernel does not fit on an SM");
  B->grid = per_sm * B->n_sm;
  // contiguous tile ranges of about equal cost per block (a tile costs its
  // sites times its lanes, plus a fixed share for its set-up), so that blocks
  // reach the grid barriers together
  std::vector<int> bstart((size_t)B->grid + 1, (int)tiles.size());
  {
    std::vector<double> cum(tiles.size() + 1, 0.0);
    for (size_t k = 0; k < tiles.size(); ++k) {
      const InstDev &I = B->slots[tiles[k].inst].dev;
      cum[k + 1] = cum[k] + (double)tiles[k].n * (double)(I.n_rep * I.n_slots + 32) + 4096.0;
    }
    size_t k = 0;
    for (int b = 0; b <= B->grid; ++b) {
      const double target = cum.back() * (double)b / (double)B->grid;
      while (k < tiles.size() && cum[k] < target) ++k;
      bstart[(size_t)b] = (int)k;
    }
    bstart[(size_t)B->grid] = (int)tiles.size();
  }
  if (bstart.size() > B->bstart_cap) {
    if (B->d_bstart) cudaFree(B->d_bstart);
    B->d_bstart = nullptr;
    B->bstart_cap = std::max<size_t>(bstart.size(), 2 * B->bstart_cap);
    rc = cuda_check(cudaMalloc(&B->d_bstart, B->bstart_cap * sizeof(int)), "block table");
    if (rc) return rc;
  }
  rc = cuda_check(cudaMemcpyAsync(B->d_bstart, bstart.data(), bstart.size() * sizeof(int), cudaMemcpyHostToDevice,
                                  B->stream),
                  "copy block table");
  if (rc) return rc;
  B->dirty = false;
  return QISG_OK;
}

// Build the host tables of a slot and upload its device state.
int setup_slot(qisg_batch *B, int i) {
  Slot &S = B->slots[i];
  const qisg_instance_desc &d = S.d;
  const int n = d.n_slots;
  const int64_t N = (int64_t)d.L * d.L * d.L_tau;
  const int rpw = 64 / n, n_groups = (d.n_replicas + rpw - 1) / rpw;
  // tables (same formulas as qisg_create)
  std::vector<uint32_t> T((size_t)n * 15);
  for (int s = 0; s < n; ++s)
    for (int us = 0; us <= 4; ++us)
      for (int ut = 0; ut <= 2; ++ut) {
        const double dk = (double)(4 * (2 - us)) * S.ladder[s].k;
        const double dkt = (double)(4 * (1 - ut)) * S.ladder[s].k_tau;
        const double p = std::exp(-dk - dkt);
        uint32_t v;
        if (p >= 1.0) {
          v = 0xFFFFFFFFu;
        } else {
          const double f = std::floor(std::ldexp(p, 32));
          v = f >= 4294967294.0 ? 0xFFFFFFFEu : (uint32_t)f;
        }
        T[(size_t)s * 15 + us * 3 + ut] = v;
      }
  std::vector<double> sq((size_t)(n > 1 ? n - 1 : 1) * 4 * kSqBits, 1.0);
  PTConst ptc;
  std::memset(&ptc, 0, sizeof(ptc));
  for (int s = 0; s + 1 < n; ++s) {
    const double dk = S.ladder[s].k - S.ladder[s + 1].k;
    const double dkt = S.ladder[s].k_tau - S.ladder[s + 1].k_tau;
    const double bases[4] = {std::exp(dk), std::exp(-dk), std::exp(dkt), std::exp(-dkt)};
    ptc.dkf[s] = (float)dk;
    ptc.dktf[s] = (float)dkt;
    for (int w = 0; w < 4; ++w) {
      if (bases[w] >= 1.0) ptc.ge1[w] |= 1u << s;
      double b = bases[w];
      for (int j = 0; j < kSqBits; ++j) {
        sq[((size_t)s * 4 + w) * kSqBits + j] = b;
        volatile double sqr = b * b;
        b = sqr;
      }
    }
  }
  // layout inside the slot's arena block
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = (o + bytes + 255) & ~size_t(255);
    return at;
  };
  const size_t o_spins = take((size_t)n_groups * N * 8), o_J = take((size_t)d.L * d.L), o_T = take(T.size() * 4),
               o_ptc = take(sizeof(PTConst)), o_sq = take(sq.size() * 8),
               o_w = take((size_t)d.n_replicas * n * 4), o_U = take((size_t)d.n_replicas * n * 16);
  const size_t bytes = o;
  size_t off = 0;
  if (!B->alloc.alloc(bytes, &off)) return fail(QISG_ENOMEM, "batch memory budget exhausted");
  S.off = off;
  S.bytes = bytes;
  unsigned char *base = B->arena + off;
  InstDev &I = S.dev;
  I.spins = reinterpret_cast<unsigned long long *>(base + o_spins);
  I.J = base + o_J;
  I.T = reinterpret_cast<const uint32_t *>(base + o_T);
  I.ptc = reinterpret_cast<const PTConst *>(base + o_ptc);
  I.sq = reinterpret_cast<const double *>(base + o_sq);
  I.walker = reinterpret_cast<int32_t *>(base + o_w);
  I.U = reinterpret_cast<unsigned long long *>(base + o_U);
  I.t = 0;
  I.remaining = d.n_sweeps > 0 ? (long long)d.n_sweeps : -1;
  I.key = make_uint2((uint32_t)d.seed, (uint32_t)(d.seed >> 32));
  I.L = d.L;
  I.Lt = d.L_tau;
  I.plane = d.L * d.L;
  I.half_plane = I.plane / 2;
  I.hpd = FastDiv((uint32_t)I.half_plane);
  I.n_slots = n;
  I.n_rep = d.n_replicas;
  I.rpw = rpw;
  I.n_groups = n_groups;
  I.spb = kBatchBlock / n;
  I.N = (int)N;
  I.tau_ap = d.tau_antiperiodic;
  I.active = 1;
  S.done = 0;
  int rc = cuda_check(cudaMemcpyAsync(base + o_T, T.data(), T.size() * 4, cudaMemcpyHostToDevice, B->stream), "T");
  if (!rc) rc = cuda_check(cudaMemcpyAsync(base + o_ptc, &ptc, sizeof(ptc), cudaMemcpyHostToDevice, B->stream), "ptc");
  if (!rc) rc = cuda_check(cudaMemcpyAsync(base + o_sq, sq.data(), sq.size() * 8, cudaMemcpyHostToDevice, B->stream), "sq");
  if (!rc) rc = cuda_check(cudaMemcpyAsync(B->d_inst + i, &I, sizeof(I), cudaMemcpyHostToDevice, B->stream), "desc");
  if (!rc) {
    const int64_t nth = std::max<int64_t>((int64_t)n_groups * N, std::max<int64_t>(I.plane, 2LL * I.n_rep * n));
    batch_init_kernel<<<(unsigned)((nth + 255) / 256), 256, 0, B->stream>>>(B->d_inst, i);
    B->launches++;
    rc = cuda_check(cudaGetLastError(), "batch init");
  }
  // the uploaded descriptor must outlive this function: synchronise
  if (!rc) rc = cuda_check(cudaStreamSynchronize(B->stream), "sync");
  if (rc) {
    B->alloc.release(S.off, S.bytes);
    return rc;
  }
  B->dirty = true;
  return QISG_OK;
}

int check_desc(const qisg_instance_desc *d) {
  if (!d || !d->ladder) return fail(QISG_EINVAL, "NULL descriptor or ladder");
  if (d->L < 2 || (d->L & 1) || d->L > 128) return fail(QISG_EINVAL, "L must be even, 2..128");
  if (d->L_tau < 2 || (d->L_tau & 1)) return fail(QISG_EINVAL, "L_tau must be even and >= 2");
  if (d->n_slots < 1 || d->n_slots > 32) return fail(QISG_EINVAL, "n_slots must be 1..32");
  if (d->n_replicas < 1 || d->n_replicas > 2 * (64 / d->n_slots))
    return fail(QISG_EINVAL, "n_replicas must be 1 .. 2 * (64 / n_slots)");
  if ((int64_t)d->L * d->L * d->L_tau > ((int64_t)1 << 30)) return fail(QISG_EINVAL, "instance too large");
  if (d->n_sweeps < 0) return fail(QISG_EINVAL, "n_sweeps < 0");
  if (d->tau_antiperiodic != 0 && d->tau_antiperiodic != 1) return fail(QISG_EINVAL, "tau_antiperiodic must be 0 or 1");
  for (int s = 0; s < d->n_slots; ++s)
    if (!std::isfinite(d->ladder[s].k) || !std::isfinite(d->ladder[s].k_tau) || d->ladder[s].k < 0 ||
        d->ladder[s].k_tau < 0)
      return fail(QISG_EINVAL, "ladder couplings must be finite and >= 0");
  return QISG_OK;
}

int sync_batch(qisg_batch *B) {
  int rc = cuda_check(cudaStreamSynchronize(B->stream), "stream synchronize");
  if (rc) return rc;
  int err = 0;
  rc = cuda_check(cudaMemcpy(&err, B->d_err, sizeof(int), cudaMemcpyDeviceToHost), "error flag");
  if (rc) return rc;
  if (err) return fail(QISG_ETIMEOUT, "a grid barrier of the batch kernel timed out");
  return QISG_OK;
}

}  // namespace

extern "C" {

int qisg_batch_create(qisg_batch **out, int capacity, size_t mem_budget, void *cuda_stream) {
  if (!out || capacity < 1) return fail(QISG_EINVAL, "need out and capacity >= 1");
  *out = nullptr;
  qisg_batch *B = new (std::nothrow) qisg_batch();
  if (!B) return fail(QISG_ENOMEM, "host allocation");
  B->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  B->capacity = capacity;
  B->slots.resize((size_t)capacity);
  int rc = cuda_check(cudaGetDevice(&B->device), "device");
  if (!rc) rc = cuda_check(cudaDeviceGetAttribute(&B->n_sm, cudaDevAttrMultiProcessorCount, B->device), "SMs");
  int coop = 0;
  if (!rc) rc = cuda_check(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, B->device), "coop");
  if (!rc && !coop) rc = fail(QISG_ECUDA, "device lacks cooperative launch");
  if (!rc) {
    if (mem_budget == 0) {
      size_t fr = 0, tot = 0;
      rc = cuda_check(cudaMemGetInfo(&fr, &tot), "mem info");
      mem_budget = fr / 2;
    }
    B->budget = mem_budget;
  }
  if (!rc) rc = cuda_check(cudaMalloc(&B->arena, B->budget), "arena");
  if (!rc) rc = cuda_check(cudaMalloc(&B->d_inst, sizeof(InstDev) * (size_t)capacity), "descriptors");
  if (!rc) rc = cuda_check(cudaMalloc(&B->d_bar, 2 * sizeof(unsigned)), "barrier");
  if (!rc) rc = cuda_check(cudaMalloc(&B->d_err, sizeof(int)), "error flag");
  // on the batch's stream (it may be non-blocking, so a default-stream memset
  // would not be ordered before the first launch)
  if (!rc) rc = cuda_check(cudaMemsetAsync(B->d_bar, 0, 2 * sizeof(unsigned), B->stream), "barrier");
  if (!rc) rc = cuda_check(cudaMemsetAsync(B->d_err, 0, sizeof(int), B->stream), "error flag");
  if (!rc) rc = cuda_check(cudaMemsetAsync(B->d_inst, 0, sizeof(InstDev) * (size_t)capacity, B->stream),
                           "descriptors");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(B->stream), "stream synchronize");
  if (rc) {
    qisg_batch_destroy(B);
    return rc;
  }
  B->alloc.reset(B->budget);
  *out = B;
  return QISG_OK;
}

int qisg_batch_admit(qisg_batch *B, const qisg_instance_desc *d, int *slot) {
  if (!B || !slot) return fail(QISG_EINVAL, "NULL argument");
  int rc = check_desc(d);
  if (rc) return rc;
  int i = -1;
  for (int k = 0; k < B->capacity; ++k)
    if (!B->slots[k].used) {
      i = k;
      break;
    }
  if (i < 0) return fail(QISG_ENOMEM, "no free slot");
  rc = sync_batch(B);
  if (rc) return rc;
  Slot &S = B->slots[i];
  S.d = *d;
  S.ladder.assign(d->ladder, d->ladder + d->n_slots);
  S.d.ladder = S.ladder.data();
  rc = setup_slot(B, i);
  if (rc) return rc;
  S.used = true;
  *slot = i;
  return QISG_OK;
}

int qisg_batch_retire(qisg_batch *B, int slot) {
  if (!B || slot < 0 || slot >= B->capacity || !B->slots[slot].used) return fail(QISG_EINVAL, "bad slot");
  int rc = sync_batch(B);
  if (rc) return rc;
  Slot &S = B->slots[slot];
  S.dev.active = 0;
  rc = cuda_check(cudaMemcpyAsync(B->d_inst + slot, &S.dev, sizeof(InstDev), cudaMemcpyHostToDevice, B->stream),
                  "descriptor");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(B->stream), "sync");
  B->alloc.release(S.off, S.bytes);
  S.used = false;
  B->dirty = true;
  return rc;
}

int qisg_batch_run(qisg_batch *B, int64_t n_sweeps) {
  if (!B || n_sweeps < 0) return fail(QISG_EINVAL, "bad batch or n_sweeps");
  if (n_sweeps == 0) return QISG_OK;
  int rc = QISG_OK;
  if (B->dirty) rc = build_tables(B);
  if (rc) return rc;
  if (B->n_tiles == 0) return QISG_OK;
  const int chunk = (int)std::min<int64_t>(n_sweeps, 1 << 20);
  int64_t left = n_sweeps;
  while (left > 0 && !rc) {
    int ns = (int)std::min<int64_t>(left, chunk);
    void *args[] = {&B->d_inst, &B->capacity, &B->d_tiles, &B->n_tiles, &B->d_bstart, &B->d_chains, &B->n_chains,
                    &ns, &B->d_bar, &B->d_err, &B->wait_ns};
    rc = cuda_check(cudaMemsetAsync(B->d_bar, 0, 2 * sizeof(unsigned), B->stream), "reset barrier");
    if (rc) break;
    rc = cuda_check(cudaLaunchCooperativeKernel((const void *)batch_kernel, dim3((unsigned)B->grid),
                                                dim3(kBatchBlock), args, B->smem, B->stream),
                    "batch kernel");
    B->launches++;
    for (int i = 0; i < B->capacity; ++i) {
      Slot &S = B->slots[i];
      if (!S.used) continue;
      const uint64_t target = S.d.n_sweeps > 0 ? (uint64_t)S.d.n_sweeps : UINT64_MAX;
      S.done = std::min<uint64_t>(target, S.done + (uint64_t)ns);
    }
    left -= ns;
  }
  return rc;
}

int qisg_batch_set_wait_limit(qisg_batch *B, int64_t wait_ns) {
  if (!B || wait_ns < 0) return fail(QISG_EINVAL, "bad batch or wait_ns < 0");
  B->wait_ns = wait_ns == 0 ? kBarrierTimeoutNs : (long long)wait_ns;
  return QISG_OK;
}

int qisg_batch_set_schedule(qisg_batch *B, int tile_rows, int schedule) {
  if (!B || tile_rows < 1 || tile_rows > kLanesMaxSitesPerThread || schedule < 0 || schedule > 1)
    return fail(QISG_EINVAL, "bad schedule");
  B->tile_rows = tile_rows;
  B->schedule = schedule;
  B->dirty = true;
  return QISG_OK;
}

int qisg_batch_autotune(qisg_batch *B, int sweeps_per_candidate, int *tile_rows, int *schedule) {
  if (!B || sweeps_per_candidate < 1) return fail(QISG_EINVAL, "bad arguments");
  float best_ms = -1.f;
  int best_rows = B->tile_rows, best_sched = B->schedule;
  cudaEvent_t e0, e1;
  int rc = cuda_check(cudaEventCreate(&e0), "event");
  if (!rc) rc = cuda_check(cudaEventCreate(&e1), "event");
  const int rows_c[] = {1, 2, 4, 8, 16};
  for (int sc = 0; sc < 2 && !rc; ++sc)
    for (int ri = 0; ri < 5 && !rc; ++ri) {
      B->tile_rows = rows_c[ri];
      B->schedule = sc;
      B->dirty = true;
      rc = build_tables(B);
      if (!rc) rc = cuda_check(cudaEventRecord(e0, B->stream), "record");
      if (!rc) rc = qisg_batch_run(B, sweeps_per_candidate);
      if (!rc) rc = cuda_check(cudaEventRecord(e1, B->stream), "record");
      if (!rc) rc = sync_batch(B);
      float ms = 0.f;
      if (!rc) rc = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
      if (!rc && (best_ms < 0.f || ms < best_ms)) {
        best_ms = ms;
        best_rows = B->tile_rows;
        best_sched = B->schedule;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  B->tile_rows = best_rows;
  B->schedule = best_sched;
  B->dirty = true;
  if (tile_rows) *tile_rows = best_rows;
  if (schedule) *schedule = best_sched;
  return QISG_OK;
}

int qisg_batch_status(qisg_batch *B, int slot, uint64_t *sweeps_done, int *done) {
  if (!B || slot < 0 || slot >= B->capacity || !B->slots[slot].used) return fail(QISG_EINVAL, "bad slot");
  const Slot &S = B->slots[slot];
  if (sweeps_done) *sweeps_done = S.done;
  if (done) *done = S.d.n_sweeps > 0 && S.done >= (uint64_t)S.d.n_sweeps;
  return QISG_OK;
}

int qisg_batch_results(qisg_batch *B, int slot, int64_t *A, int64_t *Bt, int32_t *walker_at, int8_t *S_out) {
  if (!B || slot < 0 || slot >= B->capacity || !B->slots[slot].used) return fail(QISG_EINVAL, "bad slot");
  int rc = sync_batch(B);
  if (rc) return rc;
  const Slot &S = B->slots[slot];
  const InstDev &I = S.dev;
  const int n = I.n_slots, nr = I.n_rep;
  std::vector<int32_t> wa((size_t)nr * n);
  std::vector<unsigned long long> U((size_t)nr * n * 2);
  rc = cuda_check(cudaMemcpy(wa.data(), I.walker, wa.size() * 4, cudaMemcpyDeviceToHost), "walker");
  if (!rc) rc = cuda_check(cudaMemcpy(U.data(), I.U, U.size() * 8, cudaMemcpyDeviceToHost), "U");
  if (rc) return rc;
  if (walker_at) std::memcpy(walker_at, wa.data(), wa.size() * 4);
  for (int r = 0; r < nr; ++r)
    for (int s = 0; s < n; ++s) {
      const int w = wa[(size_t)r * n + s];
      if (A) A[(size_t)r * n + s] = 2LL * I.N - 2LL * (long long)U[((size_t)r * n + w) * 2];
      if (Bt) Bt[(size_t)r * n + s] = (long long)I.N - 2LL * (long long)U[((size_t)r * n + w) * 2 + 1];
    }
  if (S_out) {
    std::vector<unsigned long long> words((size_t)I.n_groups * I.N);
    rc = cuda_check(cudaMemcpy(words.data(), I.spins, words.size() * 8, cudaMemcpyDeviceToHost), "spins");
    if (rc) return rc;
    for (int r = 0; r < nr; ++r)
      for (int w = 0; w < n; ++w) {
        const int g = r / I.rpw, lane = (r - g * I.rpw) * n + w;
        int8_t *dst = S_out + ((size_t)r * n + w) * I.N;
        const unsigned long long *src = words.data() + (size_t)g * I.N;
        for (int i = 0; i < I.N; ++i) dst[i] = ((src[i] >> lane) & 1ull) ? -1 : 1;
      }
  }
  return QISG_OK;
}

int qisg_batch_info(qisg_batch *B, size_t *free_bytes, int *free_slots, int64_t *launches) {
  if (!B) return fail(QISG_EINVAL, "NULL batch");
  if (free_bytes) *free_bytes = B->alloc.free_bytes();
  if (free_slots) {
    int f = 0;
    for (auto &S : B->slots) f += S.used ? 0 : 1;
    *free_slots = f;
  }
  if (launches) *launches = B->launches;
  return QISG_OK;
}

size_t qisg_batch_instance_bytes(const qisg_instance_desc *d) {
  if (check_desc(d)) return 0;
  const int n = d->n_slots;
  const int64_t N = (int64_t)d->L * d->L * d->L_tau;
  const int rpw = 64 / n, n_groups = (d->n_replicas + rpw - 1) / rpw;
  auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
  return up((size_t)n_groups * N * 8) + up((size_t)d->L * d->L) + up((size_t)n * 60) + up(sizeof(PTConst)) +
         up((size_t)(n > 1 ? n - 1 : 1) * 4 * kSqBits * 8) + up((size_t)d->n_replicas * n * 4) +
         up((size_t)d->n_replicas * n * 16);
}

int qisg_batch_sync(qisg_batch *B) {
  if (!B) return fail(QISG_EINVAL, "NULL batch");
  return sync_batch(B);
}

void qisg_batch_destroy(qisg_batch *B) {
  if (!B) return;
  cudaStreamSynchronize(B->stream);
  if (B->arena) cudaFree(B->arena);
  if (B->d_inst) cudaFree(B->d_inst);
  if (B->d_tiles) cudaFree(B->d_tiles);
  if (B->d_bstart) cudaFree(B->d_bstart);
  if (B->d_chains) cudaFree(B->d_chains);
  if (B->d_bar) cudaFree(B->d_bar);
  if (B->d_err) cudaFree(B->d_err);
  delete B;
}

}  // extern "C"
