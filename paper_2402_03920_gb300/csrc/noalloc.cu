// Replica overlaps without any device allocation.
//
// Some callers cannot call cudaMalloc: a host application whose allocator
// owns all device memory under a fixed budget, a serving loop that must never
// stall on the device-wide synchronisation an allocation can cause, or a
// component that runs while another library holds the memory it would need.
// For them this file offers one entry point that works in a fixed scratch
// area compiled into the library: a file-scope __device__ array that every
// GPU loading the library keeps until the process exits.
//
// Host code cannot pass the array's name to a kernel (on the host it names a
// stand-in, not device memory), so its device address is looked up with
// cudaGetSymbolAddress while the caller's device is current.  The address
// belongs to one CUDA context: it is cached per (device, context id) and
// looked up again for a context not seen before (after a device reset, or
// when a thread makes another context current).  A call whose stream is being
// captured uses the cache only, so the first call on each device and context
// must come before any stream capture.
//
// Every call shares the one scratch array, and a call clears the part it
// uses before counting.  Calls whose work overlaps on the GPU (for example on
// two streams, or from two threads) race on the array; serialise them.
#include <cuda.h>

#include <mutex>
#include <vector>

#include "qisg_internal.cuh"

namespace qisg {
namespace {

// Scratch: per (sample, slot, replica pair) count of sites where two replicas
// differ.  1 << 18 counters (2 MiB) cover, e.g., 1024 samples x 32 slots x 6
// pairs.
__device__ __align__(256) unsigned long long g_noalloc_counts[QISG_NOALLOC_MAX_COUNTS];

// Driver entry points that name the current context (resolved through the
// runtime, so the library needs no link against the driver library).
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

struct ScratchEntry {
  int device;
  unsigned long long ctx_id;
  void *addr;
};

std::mutex g_mu;
std::vector<ScratchEntry> g_cache;
CtxGetCurrentFn g_get_current = nullptr;
CtxGetIdFn g_get_id = nullptr;
bool g_resolved = false;

// Id of the context current on this thread: 1 = none current yet.
int current_context(unsigned long long *id) {
  if (!g_resolved) {
    void *f1 = nullptr, *f2 = nullptr;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return fail(QISG_ECUDA, "cannot resolve the driver's context queries");
    g_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    g_get_id = reinterpret_cast<CtxGetIdFn>(f2);
    g_resolved = true;
  }
  CUcontext c = nullptr;
  if (g_get_current(&c) != CUDA_SUCCESS) return fail(QISG_ECUDA, "cuCtxGetCurrent failed");
  if (!c) return 1;
  if (g_get_id(c, id) != CUDA_SUCCESS) return fail(QISG_ECUDA, "cuCtxGetId failed");
  return QISG_OK;
}

// Device address of the scratch array in the current context.
int scratch_address(cudaStream_t st, void **out) {
  int dev = 0;
  int rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (rc) return rc;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const bool capturing = cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
  if (capturing) cudaGetLastError();   // a refused query leaves an error behind
  std::lock_guard<std::mutex> lock(g_mu);
  unsigned long long id = 0;
  rc = current_context(&id);
  if (rc < 0) return rc;
  if (rc == 1) {   // no context current yet: the runtime creates the device's primary one
    if (capturing) return fail(QISG_ESTATE, "make the first call on this device before stream capture");
    void *p = nullptr;
    rc = cuda_check(cudaGetSymbolAddress(&p, g_noalloc_counts), "cudaGetSymbolAddress");
    if (rc) return rc;
    rc = current_context(&id);
    if (rc < 0) return rc;
    if (rc == 1) return fail(QISG_ECUDA, "no CUDA context is current");
  }
  for (const ScratchEntry &e : g_cache)
    if (e.device == dev && e.ctx_id == id) {
      *out = e.addr;
      return QISG_OK;
    }
  if (capturing) return fail(QISG_ESTATE, "make the first call on this device and context before stream capture");
  void *p = nullptr;
  rc = cuda_check(cudaGetSymbolAddress(&p, g_noalloc_counts), "cudaGetSymbolAddress");
  if (rc) return rc;
  g_cache.push_back({dev, id, p});
  *out = p;
  return QISG_OK;
}

__global__ void clear_counts_kernel(unsigned long long *c, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    c[i] = 0;
}

// Thread per site, block per site chunk (x) and, striding over y, per
// (sample block b, slot s) set, for every replica pair in turn: for each lane
// (sample) of the word, count the sites where the two replicas'
// configurations at slot s differ.  The lanes of one word are counted with a
// warp ballot per lane bit.
template <typename Word>
__global__ void overlap_count_kernel(const Word *spins, unsigned long long *counts, int64_t N,
                                     int n_slots, int n_q, int n_rep, int64_t n_samples,
                                     int64_t chunk_sites, int64_t n_sets) {
  constexpr int W = (int)sizeof(Word) * 8;
  const int n_pairs = n_rep * (n_rep - 1) / 2;
  const int64_t lo = (int64_t)blockIdx.x * chunk_sites;
  const int64_t hi = lo + chunk_sites < N ? lo + chunk_sites : N;
  for (int64_t bs = blockIdx.y; bs < n_sets; bs += gridDim.y) {   // (sample block, slot) sets
    const int s = (int)(bs % n_slots);
    const int64_t b = bs / n_slots;
    for (int p = 0; p < n_pairs; ++p) {
      int r1 = 0, r2 = 1, k = 0;
      for (int x = 0; x < n_rep; ++x)
        for (int y = x + 1; y < n_rep; ++y, ++k)
          if (k == p) {
            r1 = x;
            r2 = y;
          }
      const Word *w1 = spins + ((b * n_slots + s) * n_q + (r1 >> 2)) * N * 4 + (r1 & 3);
      const Word *w2 = spins + ((b * n_slots + s) * n_q + (r2 >> 2)) * N * 4 + (r2 & 3);
      // per-thread counts for the lanes this thread owns after the ballots
      unsigned int mine[W / 32];
#pragma unroll
      for (int h = 0; h < W / 32; ++h) mine[h] = 0;
      for (int64_t base = lo; base < hi; base += blockDim.x) {
        const int64_t site = base + threadIdx.x;
        const Word d = site < hi ? (w1[site * 4] ^ w2[site * 4]) : Word(0);
#pragma unroll
        for (int l = 0; l < W; ++l) {
          const unsigned cnt = __popc(__ballot_sync(0xffffffffu, (unsigned)((d >> l) & 1u)));
          if ((threadIdx.x & 31) == (l & 31)) mine[l >> 5] += cnt;
        }
      }
#pragma unroll
      for (int h = 0; h < W / 32; ++h) {
        const int64_t a = b * W + h * 32 + (threadIdx.x & 31);
        if (a < n_samples && mine[h])
          atomicAdd(&counts[(a * n_slots + s) * n_pairs + p], (unsigned long long)mine[h]);
      }
    }
  }
}

__global__ void overlap_finish_kernel(const unsigned long long *counts, int64_t *q, int64_t n, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    q[i] = N - 2 * (int64_t)counts[i];
}

template <typename Word>
int run(const void *spins, int L, int L_tau, int n_slots, int n_rep, int64_t n_samples, int64_t *q,
        cudaStream_t st, unsigned long long *counts) {
  constexpr int W = (int)sizeof(Word) * 8;
  const int64_t N = (int64_t)L * L * L_tau;
  const int n_pairs = n_rep * (n_rep - 1) / 2;
  const int64_t n = n_samples * n_slots * n_pairs;
  const int64_t n_b = (n_samples + W - 1) / W;
  const int n_q = (n_rep + 3) / 4;
  const int64_t chunk = 4096;
  const int64_t bx = (N + chunk - 1) / chunk;
  const int64_t n_sets = n_b * n_slots;
  const unsigned by = (unsigned)(n_sets < 65535 ? n_sets : 65535);
  clear_counts_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(counts, n);
  overlap_count_kernel<Word><<<dim3((unsigned)bx, by), 256, 0, st>>>(
      reinterpret_cast<const Word *>(spins), counts, N, n_slots, n_q, n_rep, n_samples, chunk, n_sets);
  overlap_finish_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(counts, q, n, N);
  return cuda_check(cudaGetLastError(), "overlaps (no allocation)");
}

}  // namespace
}  // namespace qisg

extern "C" int qisg_overlaps_noalloc(const void *spins, int word_bits, int L, int L_tau, int n_slots,
                                     int n_replicas, int64_t n_samples, int64_t *q, void *cuda_stream) {
  using namespace qisg;
  if (!spins || !q) return fail(QISG_EINVAL, "NULL device pointer");
  if (word_bits != 32 && word_bits != 64) return fail(QISG_EINVAL, "word_bits must be 32 or 64");
  if ((reinterpret_cast<uintptr_t>(spins) & (uintptr_t)(word_bits / 8 - 1)) || (reinterpret_cast<uintptr_t>(q) & 7u))
    return fail(QISG_EINVAL, "spins or q is not aligned to its element size");
  if (L < 2 || (L & 1) || L_tau < 2 || (L_tau & 1)) return fail(QISG_EINVAL, "L and L_tau must be even, >= 2");
  if ((int64_t)L * L > ((int64_t)1 << 31) || (int64_t)L * L * L_tau > ((int64_t)1 << 31))
    return fail(QISG_EINVAL, "lattice larger than 2^31 sites");
  if (n_slots < 1 || n_replicas < 2 || n_samples < 1) return fail(QISG_EINVAL, "need slots, >= 2 replicas, samples");
  // each factor is bounded before the product is formed
  const int64_t n_pairs = (int64_t)n_replicas * (n_replicas - 1) / 2;
  if (n_samples > QISG_NOALLOC_MAX_COUNTS || n_slots > QISG_NOALLOC_MAX_COUNTS || n_pairs > QISG_NOALLOC_MAX_COUNTS ||
      n_samples * n_slots * n_pairs > QISG_NOALLOC_MAX_COUNTS)
    return fail(QISG_EINVAL, "n_samples * n_slots * n_pairs exceeds QISG_NOALLOC_MAX_COUNTS");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  void *addr = nullptr;
  int rc = scratch_address(st, &addr);
  if (rc) return rc;
  unsigned long long *counts = reinterpret_cast<unsigned long long *>(addr);
  return word_bits == 64 ? run<unsigned long long>(spins, L, L_tau, n_slots, n_replicas, n_samples, q, st, counts)
                         : run<unsigned int>(spins, L, L_tau, n_slots, n_replicas, n_samples, q, st, counts);
}
