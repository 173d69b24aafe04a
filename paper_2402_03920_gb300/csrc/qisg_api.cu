// Host side of the C ABI declared in include/qisg.h: argument checks, the
// FP64 tables built once per instance (Sec. 2.1: Metropolis factors
// precomputed for every possible value; the PT bases), device memory, and the
// sweep schedule (Appendix A: EMCS = pt_every sweeps + one PT update, an
// energy measurement every measure_every sweeps).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "qisg_internal.cuh"

namespace {
thread_local std::string g_last_error;
}

namespace qisg {

int fail(int code, const std::string &msg) {
  g_last_error = msg;
  return code;
}

int cuda_check(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return QISG_OK;
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return QISG_ENOMEM;
  return QISG_ECUDA;
}

constexpr int kProfMax = 65536;

// While the stream is being captured into the sweep graph, an event record
// must be external to become an event-record node (a plain record is only a
// capture dependency); outside capture the plain record is the one allowed.
void prof_record(cudaEvent_t e, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  if (cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
  else
    cudaEventRecord(e, st);
}

int prof_begin(qisg_handle *h, int kind) {
  if (!((h->prof >> kind) & 1)) return -1;
  h->prof_launched[kind]++;
  std::vector<cudaEvent_t> &v = h->prof_ev[kind];
  if ((int)v.size() >= 2 * kProfMax) return -1;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return -1;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return -1;
  }
  prof_record(a, h->stream);
  v.push_back(a);
  v.push_back(b);
  return (int)v.size() - 1;
}

void prof_end(qisg_handle *h, int kind, int tok) {
  if (tok < 0) return;
  prof_record(h->prof_ev[kind][(size_t)tok], h->stream);
}

void prof_clear(qisg_handle *h) {
  for (cudaEvent_t e : h->prof_spare) cudaEventDestroy(e);
  h->prof_spare.clear();
  for (int k = 0; k < kProfKinds; ++k) {
    for (cudaEvent_t e : h->prof_ev[k]) cudaEventDestroy(e);
    h->prof_ev[k].clear();
    h->prof_launched[k] = 0;
  }
}

__global__ void advance_kernel(unsigned long long *d_t) { *d_t += 1ull; }

int advance_counter(qisg_handle *h) {
  advance_kernel<<<1, 1, 0, h->stream>>>(h->d_t);
  h->launches++;
  h->t++;
  return cuda_check(cudaGetLastError(), "advance counter");
}

__global__ void philox_kernel(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
  const uint4 r = philox(c, make_uint2(key[2 * i], key[2 * i + 1]));
  out[4 * i] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

}  // namespace qisg

using namespace qisg;

namespace {

// FP64 table of the Metropolis test (Sec. 2.1).  Flipping a spin with u_s of
// its 4 spatial bonds and u_t of its 2 tau bonds unsatisfied multiplies the
// weight exp(k A + k_tau B) by exp(Delta), Delta = -4k(2-u_s) - 4k_tau(1-u_t).
// Both products are exact (k times 8, 4, 0, -4 or -8), so Delta is rounded
// once.  T = 0xFFFFFFFF when e^Delta >= 1, else min(0xFFFFFFFE,
// floor(e^Delta 2^32)); a spin flips iff T == 0xFFFFFFFF or its draw R < T.
void build_thresholds(qisg_handle *h) {
  h->T.assign((size_t)h->n_slots * 15, 0);
  for (int s = 0; s < h->n_slots; ++s)
    for (int us = 0; us <= 4; ++us)
      for (int ut = 0; ut <= 2; ++ut) {
        const double dk = (double)(4 * (2 - us)) * h->k[s];
        const double dkt = (double)(4 * (1 - ut)) * h->kt[s];
        const double p = std::exp(-dk - dkt);
        uint32_t v;
        if (p >= 1.0) {
          v = 0xFFFFFFFFu;
        } else {
          const double f = std::floor(std::ldexp(p, 32));
          v = f >= 4294967294.0 ? 0xFFFFFFFEu : (uint32_t)f;
        }
        h->T[(size_t)s * 15 + us * 3 + ut] = v;
      }
}

// PT bases of the pair (s, s+1): alpha+- = exp(+-(k_s - k_{s+1})),
// beta+- = exp(+-(k_tau,s - k_tau,s+1)).
void build_bases(qisg_handle *h) {
  const int n = h->n_slots;
  h->bases.assign((size_t)6 * n, 1.0);
  for (int s = 0; s + 1 < n; ++s) {
    const double dk = h->k[s] - h->k[s + 1];
    const double dkt = h->kt[s] - h->kt[s + 1];
    h->bases[s] = std::exp(dk);
    h->bases[n + s] = std::exp(-dk);
    h->bases[2 * n + s] = std::exp(dkt);
    h->bases[3 * n + s] = std::exp(-dkt);
    h->bases[4 * n + s] = dk;
    h->bases[5 * n + s] = dkt;
  }
  // squaring chains of the four bases of every pair
  h->sq.assign((size_t)(n > 1 ? n - 1 : 1) * 4 * kSqBits, 1.0);
  for (int s = 0; s + 1 < n; ++s)
    for (int w = 0; w < 4; ++w) {
      double b = h->bases[(size_t)w * n + s];
      double *c = &h->sq[((size_t)s * 4 + w) * kSqBits];
      for (int j = 0; j < kSqBits; ++j) {
        c[j] = b;
        volatile double sqr = b * b;   // one rounded IEEE multiply, never contracted
        b = sqr;
      }
    }
}

template <typename T>
int dalloc(qisg_handle *h, T **p, size_t bytes) {
  if (h->mem_budget && h->device_bytes + bytes > h->mem_budget)
    return fail(QISG_ENOMEM, "state exceeds the memory budget");
  void *q = nullptr;
  const cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
  if (e != cudaSuccess) return cuda_check(e, "cudaMalloc");
  h->device_bytes += bytes;
  *p = reinterpret_cast<T *>(q);
  return QISG_OK;
}

int recompute_energies(qisg_handle *h) {
  int rc;
  if (h->layout == QISG_LAYOUT_LANES) {
    if ((rc = lanes_half_sweep(h, 0, 1))) return rc;
    return lanes_half_sweep(h, 1, 1);
  }
  if (h->layout == QISG_LAYOUT_SITES) {
    if ((rc = sites_half_sweep(h, 0, 1))) return rc;
    return sites_half_sweep(h, 1, 1);
  }
  if ((rc = samples_materialize(h))) return rc;
  if ((rc = samples_half_sweep(h, 0, 1))) return rc;
  return samples_half_sweep(h, 1, 1);
}

int sync_handle(qisg_handle *h) {
  int rc = cuda_check(cudaStreamSynchronize(h->stream), "stream synchronize");
  if (rc) return rc;
  int err = 0;
  rc = cuda_check(cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost), "read error flag");
  if (rc) return rc;
  if (err) return fail(QISG_ETIMEOUT, "a bounded device wait expired");
  return QISG_OK;
}

}  // namespace

namespace qisg {
int handle_sync(qisg_handle *h) { return sync_handle(h); }
}  // namespace qisg

extern "C" {

void qisg_opts_default(qisg_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->pt_every = 1;
}

int qisg_ladder_linear(double lo, double hi, int n, double gamma, qisg_slot *out) {
  if (!out || n < 1 || !(gamma > 0) || !(lo > 0) || !std::isfinite(hi))
    return fail(QISG_EINVAL, "ladder: need n >= 1, gamma > 0, lo > 0");
  for (int s = 0; s < n; ++s) {
    const double k = (n == 1) ? lo : lo + (hi - lo) * (double)s / (double)(n - 1);
    const double kt = -0.5 * std::log(std::tanh(k * gamma));
    if (!std::isfinite(kt) || kt < 0 || !(k > 0)) return fail(QISG_EINVAL, "ladder: k_tau not finite");
    out[s].k = k;
    out[s].k_tau = kt;
  }
  return QISG_OK;
}

int qisg_create(qisg_handle **out, int L, int L_tau, const qisg_slot *ladder, int n_slots,
                int n_replicas, int64_t n_samples, uint64_t seed, const qisg_opts *opts) {
  if (!out) return fail(QISG_EINVAL, "out is NULL");
  *out = nullptr;
  if (L < 2 || (L & 1)) return fail(QISG_EINVAL, "L must be even and >= 2");
  if (L_tau < 2 || (L_tau & 1)) return fail(QISG_EINVAL, "L_tau must be even and >= 2");
  if (n_slots < 1 || !ladder) return fail(QISG_EINVAL, "need at least one ladder slot");
  if (n_replicas < 1 || n_replicas > 1024) return fail(QISG_EINVAL, "n_replicas must be in 1..1024");
  if (n_samples < 1) return fail(QISG_EINVAL, "n_samples must be >= 1");
  if (n_slots > 32) return fail(QISG_EINVAL, "n_slots must be <= 32");
  if ((int64_t)L * L * L_tau > ((int64_t)1 << 31)) return fail(QISG_EINVAL, "lattice too large");
  for (int s = 0; s < n_slots; ++s)
    if (!std::isfinite(ladder[s].k) || !std::isfinite(ladder[s].k_tau) || ladder[s].k < 0 ||
        ladder[s].k_tau < 0)
      return fail(QISG_EINVAL, "ladder couplings must be finite and >= 0");
  qisg_opts o;
  qisg_opts_default(&o);
  if (opts) o = *opts;
  if (o.word_bits != 0 && o.word_bits != 32 && o.word_bits != 64)
    return fail(QISG_EINVAL, "word_bits must be 0, 32 or 64");
  if (o.pt_every < 0 || o.measure_every < 0) return fail(QISG_EINVAL, "negative cadence");
  if (o.layout < 0 || o.layout > 3) return fail(QISG_EINVAL, "unknown layout");
  if (o.layout == QISG_LAYOUT_SITES) {
    if (o.word_bits != 0 && o.word_bits != 32)
      return fail(QISG_EINVAL, "the SITES packing holds 32 tau-sites per 32-bit word");
    if (L_tau % 64 != 0) return fail(QISG_EINVAL, "the SITES packing needs L_tau to be a multiple of 64");
    if (n_samples >= ((int64_t)1 << 24)) return fail(QISG_EINVAL, "the SITES packing takes fewer than 2^24 samples");
    for (int s = 0; s < n_slots; ++s)
      if (ladder[s].k != ladder[s].k_tau || ladder[s].k > 16.0)
        return fail(QISG_EINVAL, "the daemon rule needs k_tau = k <= 16 at every slot");
  }
  if (o.tau_antiperiodic != 0 && o.tau_antiperiodic != 1) return fail(QISG_EINVAL, "tau_antiperiodic must be 0 or 1");
  if (o.history_len < 0 || o.maxit < 0 || o.blocks_len < 0) return fail(QISG_EINVAL, "negative record length");
  if (o.maxit > 0 && o.blocks_len < 1) return fail(QISG_EINVAL, "maxit > 0 needs blocks_len >= 1");

  qisg_handle *h = new (std::nothrow) qisg_handle();
  if (!h) return fail(QISG_ENOMEM, "host allocation");
  h->L = L;
  h->Lt = L_tau;
  h->N = (int64_t)L * L * L_tau;
  h->n_slots = n_slots;
  h->n_rep = n_replicas;
  h->n_samples = n_samples;
  h->seed = seed;
  h->pt_every = o.pt_every;
  h->measure_every = o.measure_every;
  h->stream = reinterpret_cast<cudaStream_t>(o.cuda_stream);
  h->mem_budget = o.mem_budget;
  h->per_sample_launch = o.per_sample_launch;
  h->tau_ap = o.tau_antiperiodic;
  h->hist_len = o.history_len;
  h->maxit = o.maxit;
  h->blk_len = o.maxit > 0 ? o.blocks_len : 0;
  h->k.resize(n_slots);
  h->kt.resize(n_slots);
  for (int s = 0; s < n_slots; ++s) {
    h->k[s] = ladder[s].k;
    h->kt[s] = ladder[s].k_tau;
  }
  int layout = o.layout;
  if (layout == QISG_LAYOUT_AUTO) layout = n_samples >= 32 ? QISG_LAYOUT_SAMPLES : QISG_LAYOUT_LANES;
  h->layout = layout;
  if (layout == QISG_LAYOUT_SITES) {
    h->W = 32;
    h->n_a_pad = n_samples;
  } else if (layout == QISG_LAYOUT_LANES) {
    int W = o.word_bits;
    if (W == 0) W = (n_slots * n_replicas <= 32) ? 32 : 64;
    if (n_slots > W) {
      delete h;
      return fail(QISG_EINVAL, "LANES packing needs n_slots <= word bits");
    }
    if (n_replicas > 2 * (W / n_slots)) {
      delete h;
      return fail(QISG_EINVAL, "LANES packing needs n_replicas <= 2 * (word bits / n_slots)");
    }
    h->W = W;
    h->rpw = W / n_slots;
    h->n_groups = (n_replicas + h->rpw - 1) / h->rpw;
    h->n_a_pad = n_samples;
  } else {
    int W = o.word_bits;
    if (W == 0) W = n_samples <= 32 ? 32 : 64;
    h->W = W;
    h->n_b = (n_samples + W - 1) / W;
    h->n_q = (n_replicas + 3) / 4;
    h->n_a_pad = h->n_b * W;
  }
  build_thresholds(h);
  build_bases(h);

  int rc = cuda_check(cudaGetDevice(&h->device), "cudaGetDevice");
  if (!rc) rc = cuda_check(cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device),
                           "device attribute");
  const int64_t n_chain_slots = h->n_a_pad * n_replicas * n_slots;
  const int n_pairs = h->n_pairs();
  if (!rc) {
    if (layout == QISG_LAYOUT_LANES) {
      h->spins_bytes = (size_t)n_samples * h->n_groups * h->N * (h->W / 8);
      h->J_bytes = (size_t)n_samples * L * L;
    } else if (layout == QISG_LAYOUT_SITES) {
      h->spins_bytes = (size_t)n_samples * n_replicas * n_slots * (h->N / 8);
      h->J_bytes = (size_t)n_samples * L * L;
    } else {
      h->spins_bytes = (size_t)h->n_b * n_slots * h->n_q * h->N * 4 * (h->W / 8);
      h->J_bytes = (size_t)h->n_b * L * L * 2 * (h->W / 8);
    }
    rc = dalloc(h, &h->spins, h->spins_bytes);
    h->fused = layout == QISG_LAYOUT_SAMPLES;
    if (!rc && h->fused) rc = dalloc(h, &h->spins_alt, h->spins_bytes);
  }
  if (!rc) rc = dalloc(h, &h->J, h->J_bytes);
  if (!rc) rc = dalloc(h, &h->d_T, h->T.size() * 4);
  if (!rc) rc = dalloc(h, &h->d_bases, h->bases.size() * 8);
  if (!rc) rc = dalloc(h, &h->d_sq, h->sq.size() * 8);
  if (!rc) rc = dalloc(h, &h->d_ptc, sizeof(PTConst));
  if (!rc) rc = dalloc(h, &h->d_walker, (size_t)n_chain_slots * 4);
  if (!rc) rc = dalloc(h, &h->d_U, (size_t)n_chain_slots * 2 * 8);
  if (!rc) rc = dalloc(h, &h->d_sumA, (size_t)n_chain_slots * 8);
  if (!rc) rc = dalloc(h, &h->d_sumB, (size_t)n_chain_slots * 8);
  const size_t qn = (size_t)h->n_a_pad * n_slots * (n_pairs > 0 ? n_pairs : 1);
  if (!rc) rc = dalloc(h, &h->d_sumq, qn * 8);
  if (!rc) rc = dalloc(h, &h->d_sumq2, qn * 8);
  if (!rc) rc = dalloc(h, &h->d_q, qn * 8);
  if (!rc) rc = dalloc(h, &h->d_out, (size_t)2 * n_chain_slots * 8 + qn * 8);
  if (!rc) rc = dalloc(h, &h->d_t, 16);
  if (!rc) rc = dalloc(h, &h->d_err, 4);
  if (!rc) rc = dalloc(h, &h->d_meas, 8);
  const size_t n_rows = (size_t)n_samples * n_replicas * n_slots;
  if (!rc && h->hist_len) rc = dalloc(h, &h->d_hist, (size_t)h->hist_len * n_rows);
  if (!rc && h->blk_len) rc = dalloc(h, &h->d_blkA, (size_t)h->blk_len * n_rows * 8);
  if (!rc && h->blk_len) rc = dalloc(h, &h->d_blkB, (size_t)h->blk_len * n_rows * 8);
  if (!rc && layout == QISG_LAYOUT_SAMPLES)
    rc = dalloc(h, &h->d_acc, (size_t)h->n_b * n_replicas * n_slots * (h->W / 8));
  // the persistent kernel's grid barrier (two words) and the blue pass's PT ticket
  if (!rc && layout == QISG_LAYOUT_SAMPLES) rc = dalloc(h, &h->d_bar, 3 * sizeof(unsigned));
  if (!rc && layout == QISG_LAYOUT_SITES) rc = dalloc(h, &h->d_dcum, (size_t)n_slots * 256 * 8);
  if (!rc && layout == QISG_LAYOUT_SITES) rc = dalloc(h, &h->d_dlut, ((size_t)n_slots << kDaemonLutBits) * 9);
  if (rc) {
    qisg_destroy(h);
    return rc;
  }
  // walker w starts at slot w
  std::vector<int32_t> wa((size_t)n_chain_slots);
  for (int64_t i = 0; i < n_chain_slots; ++i) wa[(size_t)i] = (int32_t)(i % n_slots);
  rc = cuda_check(cudaMemcpyAsync(h->d_walker, wa.data(), wa.size() * 4, cudaMemcpyHostToDevice, h->stream),
                  "copy walker");
  if (!rc) rc = cuda_check(cudaMemcpyAsync(h->d_T, h->T.data(), h->T.size() * 4, cudaMemcpyHostToDevice, h->stream),
                           "copy T");
  if (!rc) rc = cuda_check(cudaMemcpyAsync(h->d_bases, h->bases.data(), h->bases.size() * 8,
                                           cudaMemcpyHostToDevice, h->stream),
                           "copy bases");
  if (!rc) rc = cuda_check(cudaMemcpyAsync(h->d_sq, h->sq.data(), h->sq.size() * 8, cudaMemcpyHostToDevice,
                                           h->stream),
                           "copy squaring chains");
  PTConst ptc;
  std::memset(&ptc, 0, sizeof(ptc));
  for (int s = 0; s + 1 < n_slots; ++s) {
    ptc.dkf[s] = (float)h->bases[(size_t)4 * n_slots + s];
    ptc.dktf[s] = (float)h->bases[(size_t)5 * n_slots + s];
    for (int w = 0; w < 4; ++w)
      if (h->bases[(size_t)w * n_slots + s] >= 1.0) ptc.ge1[w] |= 1u << s;
  }
  if (!rc) rc = cuda_check(cudaMemcpyAsync(h->d_ptc, &ptc, sizeof(ptc), cudaMemcpyHostToDevice, h->stream),
                           "copy PT constants");
  if (!rc) rc = cuda_check(cudaMemsetAsync(h->d_sumA, 0, (size_t)n_chain_slots * 8, h->stream), "memset");
  if (!rc) rc = cuda_check(cudaMemsetAsync(h->d_sumB, 0, (size_t)n_chain_slots * 8, h->stream), "memset");
  if (!rc) rc = cuda_check(cudaMemsetAsync(h->d_sumq, 0, qn * 8, h->stream), "memset");
  if (!rc) rc = cuda_check(cudaMemsetAsync(h->d_sumq2, 0, qn * 8, h->stream), "memset");
  if (!rc) rc = cuda_check(cudaMemsetAsync(h->d_q, 0, qn * 8, h->stream), "memset");
  if (!rc) rc = cuda_check(cudaMemsetAsync(h->d_t, 0, 16, h->stream), "memset");
  if (!rc) rc = cuda_check(cudaMemsetAsync(h->d_err, 0, 4, h->stream), "memset");
  if (!rc) rc = cuda_check(cudaMemsetAsync(h->d_meas, 0, 8, h->stream), "memset");
  if (!rc && h->d_bar) rc = cuda_check(cudaMemsetAsync(h->d_bar, 0, 3 * sizeof(unsigned), h->stream), "memset");
  if (!rc && h->d_acc)
    rc = cuda_check(cudaMemsetAsync(h->d_acc, 0, (size_t)h->n_b * n_replicas * n_slots * (h->W / 8), h->stream),
                    "memset");
  if (!rc) rc = (layout == QISG_LAYOUT_LANES) ? lanes_init(h) : (layout == QISG_LAYOUT_SITES) ? sites_init(h) : samples_init(h);
  if (!rc) rc = recompute_energies(h);
  if (!rc) rc = sync_handle(h);
  if (rc) {
    qisg_destroy(h);
    return rc;
  }
  *out = h;
  return QISG_OK;
}

}  // extern "C"

namespace {

// One sweep t = h->t, enqueued on h->stream: red, blue (+ energies), PT when
// due, measurement when due, advance of the device counter.
// One sweep (Sec. 2.1): red, blue, PT pass when due, measurement when due.
// ev: optional events recorded before the red pass, between the passes and
// after the blue pass (autotuning).
int one_sweep(qisg_handle *h, cudaEvent_t *ev = nullptr) {
  const bool lanes = h->layout != QISG_LAYOUT_SAMPLES;   // walker-major: LANES and SITES
  const bool sites = h->layout == QISG_LAYOUT_SITES;
  const uint64_t t = h->t;
  int rc = ev ? cuda_check(cudaEventRecord(ev[0], h->stream), "record") : QISG_OK;
  if (!rc) rc = sites ? sites_half_sweep(h, 0, 0) : lanes ? lanes_half_sweep(h, 0, 0) : samples_half_sweep(h, 0, 0);
  if (!rc && ev) rc = cuda_check(cudaEventRecord(ev[1], h->stream), "record");
  if (!rc) rc = sites ? sites_half_sweep(h, 1, 0) : lanes ? lanes_half_sweep(h, 1, 0) : samples_half_sweep(h, 1, 0);
  if (!rc && ev) rc = cuda_check(cudaEventRecord(ev[2], h->stream), "record");
  bool advanced = false;
  if (!rc && h->pt_every > 0 && (t + 1) % (uint64_t)h->pt_every == 0) {
    if (lanes) {
      rc = lanes_pt(h, 0);
    } else {
      rc = samples_pt(h, 0, 1);   // the permute kernel advances the counter
      advanced = true;
    }
  }
  if (!rc && h->measure_every > 0 && (t + 1) % (uint64_t)h->measure_every == 0) {
    rc = sites ? sites_measure(h, 0) : lanes ? lanes_measure(h, 0) : samples_measure(h, 0);
    if (!rc && (h->hist_len || h->maxit)) rc = record_measurement(h);
    h->n_meas++;
  }
  if (!rc) {
    if (advanced)
      h->t++;
    else
      rc = advance_counter(h);
  }
  return rc;
}

int64_t gcd64(int64_t a, int64_t b) { return b ? gcd64(b, a % b) : a; }

// Persistent form: sweeps per launch when nothing is measured.
constexpr int kPersistChunk = 64;

// k sweeps in the persistent form (the caller keeps a due measurement at
// the end of the run, never inside it), then the measurement if due.
int persistent_chunk(qisg_handle *h, int k) {
  int rc = samples_persistent(h, k);
  if (rc) return rc;
  h->t += (uint64_t)k;
  if (h->measure_every > 0 && h->t % (uint64_t)h->measure_every == 0) {
    rc = samples_measure(h, 0);
    if (!rc && (h->hist_len || h->maxit)) rc = record_measurement(h);
    h->n_meas++;
  }
  return rc;
}

// Sweeps per persistent launch: up to the next measurement.
int persistent_run(const qisg_handle *h) { return h->measure_every > 0 ? h->measure_every : kPersistChunk; }

int cycle_length(const qisg_handle *h) {
  if (h->persistent) {   // whole launches; an even count returns to the lattice buffer
    const int r = persistent_run(h);
    return (r & 1) ? 2 * r : r;
  }
  const int64_t p = h->pt_every > 0 ? h->pt_every : 1;
  const int64_t m = h->measure_every > 0 ? h->measure_every : 1;
  int64_t l = p / gcd64(p, m) * m;
  if (h->fused && (l & 1)) l *= 2;   // every red pass swaps the lattice buffers
  return (int)(l > 4096 ? 0 : l);   // no graph for very long cycles
}

void drop_cycle(qisg_handle *h) {
  if (h->cyc_exec) cudaGraphExecDestroy(h->cyc_exec);
  if (h->cyc_graph) cudaGraphDestroy(h->cyc_graph);
  h->cyc_exec = nullptr;
  h->cyc_graph = nullptr;
  h->cyc_sweeps = 0;
  h->cyc_ev_nodes.clear();
  h->cyc_ev_kind.clear();
  for (cudaEvent_t e : h->cyc_events) cudaEventDestroy(e);
  h->cyc_events.clear();
}

// Capture C sweeps (starting at a multiple of C) into a graph.  The host
// mirrors (t, measurements, launch counts) are restored afterwards and
// advanced per replay instead.
int build_cycle(qisg_handle *h, int C) {
  drop_cycle(h);
  int rc = QISG_OK;
  if (!h->cap_stream)
    rc = cuda_check(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking), "create capture stream");
  if (rc) return rc;
  const uint64_t t0 = h->t;
  const int64_t meas0 = h->n_meas, launches0 = h->launches;
  const bool pending0 = h->perm_pending;
  void *const spins0 = h->spins;
  int64_t pl0[kProfKinds];
  size_t ev0[kProfKinds];
  for (int k = 0; k < kProfKinds; ++k) {
    pl0[k] = h->prof_launched[k];
    ev0[k] = h->prof_ev[k].size();
  }
  cudaStream_t user = h->stream;
  h->stream = h->cap_stream;
  rc = cuda_check(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (!rc && h->persistent)
    for (int i = 0; i < C && !rc; i += persistent_run(h)) rc = persistent_chunk(h, persistent_run(h));
  else if (!rc)
    for (int i = 0; i < C && !rc; ++i) rc = one_sweep(h);
  cudaGraph_t g = nullptr;
  const int rc_end = cuda_check(cudaStreamEndCapture(h->cap_stream, &g), "end capture");
  h->stream = user;
  if (!rc) rc = rc_end;
  h->cyc_launches = h->launches - launches0;
  h->cyc_meas = h->n_meas - meas0;
  h->cyc_pending = h->perm_pending;
  h->perm_pending = pending0;
  if (!rc && h->spins != spins0) rc = fail(QISG_ECUDA, "sweep cycle does not return to its lattice buffer");
  h->t = t0;
  h->n_meas = meas0;
  h->launches = launches0;
  // events recorded during capture belong to the graph's record nodes
  std::map<cudaEvent_t, std::pair<int, int>> which;
  for (int k = 0; k < kProfKinds; ++k) {
    h->cyc_prof_launched[k] = h->prof_launched[k] - pl0[k];
    h->prof_launched[k] = pl0[k];
    for (size_t i = ev0[k]; i < h->prof_ev[k].size(); ++i) which[h->prof_ev[k][i]] = {k, (int)((i - ev0[k]) & 1)};
  }
  if (!rc) {
    size_t n_nodes = 0;
    rc = cuda_check(cudaGraphGetNodes(g, nullptr, &n_nodes), "graph nodes");
    std::vector<cudaGraphNode_t> nodes(n_nodes);
    if (!rc && n_nodes) rc = cuda_check(cudaGraphGetNodes(g, nodes.data(), &n_nodes), "graph nodes");
    // walk the linear chain from its root so that record nodes keep their order
    // (edges may carry programmatic-launch data, so every query takes edge data)
    std::vector<cudaGraphNode_t> order;
    if (!rc) {
      cudaGraphNode_t cur = nullptr;
      for (cudaGraphNode_t nd : nodes) {
        size_t nd_deps = 0;
        rc = cuda_check(cudaGraphNodeGetDependencies(nd, nullptr, nullptr, &nd_deps), "graph node dependencies");
        if (rc) break;
        if (nd_deps == 0) cur = nd;
      }
      while (!rc && cur) {
        order.push_back(cur);
        size_t nd_out = 0;
        rc = cuda_check(cudaGraphNodeGetDependentNodes(cur, nullptr, nullptr, &nd_out), "graph node dependents");
        if (rc || nd_out != 1) break;
        cudaGraphNode_t nxt = nullptr;
        cudaGraphEdgeData ed;
        rc = cuda_check(cudaGraphNodeGetDependentNodes(cur, &nxt, &ed, &nd_out), "graph node dependents");
        cur = nxt;
      }
      if (order.size() != n_nodes) rc = fail(QISG_ECUDA, "captured sweep graph is not a chain");
    }
    for (size_t i = 0; !rc && i < order.size(); ++i) {
      cudaGraphNodeType ty;
      cudaGraphNodeGetType(order[i], &ty);
      if (ty != cudaGraphNodeTypeEventRecord) continue;
      cudaEvent_t e = nullptr;
      cudaGraphEventRecordNodeGetEvent(order[i], &e);
      auto it = which.find(e);
      if (it == which.end()) continue;
      h->cyc_ev_nodes.push_back(order[i]);
      h->cyc_ev_kind.push_back(it->second);
    }
    if (!rc) rc = cuda_check(cudaGraphInstantiate(&h->cyc_exec, g, 0), "instantiate sweep graph");
  }
  for (int k = 0; k < kProfKinds; ++k) {   // the capture's own events are not timings; the
    for (size_t i = ev0[k]; i < h->prof_ev[k].size(); ++i)   // graph keeps them until dropped
      h->cyc_events.push_back(h->prof_ev[k][i]);
    h->prof_ev[k].resize(ev0[k]);
  }
  h->cyc_graph = g;
  if (rc) {
    drop_cycle(h);
    return rc;
  }
  h->cyc_sweeps = C;
  h->cyc_profiled = h->prof;
  return QISG_OK;
}

constexpr int kProfMaxPairs = 65536;

int replay_cycle(qisg_handle *h) {
  if (h->prof) {
    // fresh events for this replay's record nodes, paired as recorded
    std::vector<cudaEvent_t> fresh(h->cyc_ev_nodes.size(), nullptr);
    bool room = true;
    for (int k = 0; k < kProfKinds; ++k)
      if ((int)h->prof_ev[k].size() >= 2 * kProfMaxPairs) room = false;
    for (size_t i = 0; i < fresh.size(); ++i) {
      if (room) cudaEventCreate(&fresh[i]);
      else cudaEventCreateWithFlags(&fresh[i], cudaEventDisableTiming);
      const cudaError_t e = cudaGraphExecEventRecordNodeSetEvent(h->cyc_exec, h->cyc_ev_nodes[i], fresh[i]);
      const int rc = cuda_check(e, ("rebind graph event " + std::to_string(i) + " of " +
                                    std::to_string(h->cyc_ev_nodes.size())).c_str());
      if (rc) return rc;
    }
    if (room)
      for (size_t i = 0; i < fresh.size(); ++i) h->prof_ev[h->cyc_ev_kind[i].first].push_back(fresh[i]);
    else
      for (cudaEvent_t e : fresh) h->prof_spare.push_back(e);
    for (int k = 0; k < kProfKinds; ++k) h->prof_launched[k] += h->cyc_prof_launched[k];
  }
  const int rc = cuda_check(cudaGraphLaunch(h->cyc_exec, h->stream), "launch sweep graph");
  if (rc) return rc;
  h->t += (uint64_t)h->cyc_sweeps;
  h->n_meas += h->cyc_meas;
  h->perm_pending = h->cyc_pending;
  h->launches += h->cyc_launches;
  return QISG_OK;
}

}  // namespace

extern "C" {

int qisg_sweep(qisg_handle *h, int64_t n_sweeps) {
  if (!h || n_sweeps < 0) return fail(QISG_EINVAL, "bad handle or n_sweeps < 0");
  if (h->needs_state) return fail(QISG_ESTATE, "energies were replaced by qisg_pt_given: call qisg_set_state");
  const int C = h->use_graphs ? cycle_length(h) : 0;
  while (n_sweeps > 0) {
    int rc;
    if (C > 0 && n_sweeps >= C && h->t % (uint64_t)C == 0) {
      if (!h->cyc_exec || h->cyc_sweeps != C || h->cyc_profiled != h->prof) {
        rc = build_cycle(h, C);
        if (rc) return rc;
      }
      rc = replay_cycle(h);
      n_sweeps -= C;
    } else if (h->persistent) {   // up to the next measurement (or a full run)
      const int r = persistent_run(h);
      const int k = (int)std::min<int64_t>(n_sweeps, r - (int64_t)(h->t % (uint64_t)r));
      rc = persistent_chunk(h, k);
      n_sweeps -= k;
    } else {
      rc = one_sweep(h);
      n_sweeps -= 1;
    }
    if (rc) return rc;
  }
  return QISG_OK;
}

int qisg_set_launch_overlap(qisg_handle *h, int enable) {
  if (!h) return fail(QISG_EINVAL, "NULL handle");
  int rc = sync_handle(h);
  if (rc) return rc;
  h->pdl = enable != 0;
  drop_cycle(h);
  return QISG_OK;
}

int qisg_set_pt_in_blue(qisg_handle *h, int enable, int64_t wait_ns) {
  if (!h || wait_ns < 0) return fail(QISG_EINVAL, "bad handle or wait_ns < 0");
  int rc = sync_handle(h);
  if (rc) return rc;
  h->pt_in_blue = enable != 0;
  h->wait_ns = wait_ns > 0 ? wait_ns : 5000000000ll;
  drop_cycle(h);
  return QISG_OK;
}

int qisg_set_persistent(qisg_handle *h, int enable, int64_t wait_ns) {
  if (!h || wait_ns < 0) return fail(QISG_EINVAL, "bad handle or wait_ns < 0");
  if (enable && !samples_persistent_ok(h))
    return fail(QISG_EINVAL, "the persistent form needs the SAMPLES packing, 32-bit words, PT every sweep");
  int rc = sync_handle(h);
  if (rc) return rc;
  h->persistent = enable != 0;
  h->wait_ns = wait_ns == 0 ? kBarrierTimeoutNs : (long long)wait_ns;
  drop_cycle(h);
  return QISG_OK;
}

// Persistent form: time whole runs of sweeps for every (red tile, blue tile)
// pair -- the red pass's threads per site and the number of sites each blue
// thread walks along tau -- on the handle's own state; keep the fastest.
static int autotune_persistent(qisg_handle *h, int sweeps_per_candidate, int *chosen) {
  const int red_tiles[3] = {1, 2, 4}, blue_tiles[7] = {0, 1, 2, 4, 8, 16, 32};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = cuda_check(cudaEventCreate(&e0), "event");
  if (!rc) rc = cuda_check(cudaEventCreate(&e1), "event");
  float best = -1.f;
  int best_r = 4, best_b = 8;
  auto run = [&](int n) {
    int r = QISG_OK;
    while (n > 0 && !r) {
      const int rr = persistent_run(h);
      const int k = (int)std::min<int64_t>(n, rr - (int64_t)(h->t % (uint64_t)rr));
      r = persistent_chunk(h, k);
      n -= k;
    }
    return r;
  };
  for (int i = 0; i < 3 && !rc; ++i)
    for (int j = 0; j < 7 && !rc; ++j) {
      h->sweep_tile[0] = red_tiles[i];
      h->sweep_tile[1] = blue_tiles[j];
      h->sweep_variant[0] = h->sweep_variant[1] = 0;
      rc = run(1);   // warm the candidate
      if (!rc) rc = cuda_check(cudaEventRecord(e0, h->stream), "record");
      if (!rc) rc = run(sweeps_per_candidate);
      if (!rc) rc = cuda_check(cudaEventRecord(e1, h->stream), "record");
      if (!rc) rc = cuda_check(cudaEventSynchronize(e1), "sync");
      float ms = 0.f;
      if (!rc) rc = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
      if (!rc && (best < 0.f || ms < best)) {
        best = ms;
        best_r = red_tiles[i];
        best_b = blue_tiles[j];
      }
    }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc) return rc;
  h->sweep_tile[0] = best_r;
  h->sweep_tile[1] = best_b;
  drop_cycle(h);
  if (chosen) *chosen = best_b;
  return sync_handle(h);
}

int qisg_set_graphs(qisg_handle *h, int enable) {
  if (!h) return fail(QISG_EINVAL, "NULL handle");
  h->use_graphs = enable != 0;
  if (!h->use_graphs) drop_cycle(h);
  return QISG_OK;
}

int qisg_autotune(qisg_handle *h, int sweeps_per_candidate, int *chosen) {
  if (!h || sweeps_per_candidate < 1) return fail(QISG_EINVAL, "bad handle or sweep count");
  if (h->layout != QISG_LAYOUT_SAMPLES) {
    if (chosen) *chosen = 0;
    return QISG_OK;
  }
  if (h->persistent) return autotune_persistent(h, sweeps_per_candidate, chosen);
  // candidates: tiles 1, 2, ..., 64 and the default (0), and for W = 32 each
  // with the three blue kernel variants; the red and blue passes are timed
  // apart and tuned apart
  static const int kTiles[8] = {1, 2, 4, 8, 16, 32, 64, 0};
  const int n_tiles = 8, n_cand = h->W == 32 ? 3 * n_tiles : n_tiles;
  float best_ms[2] = {0.f, 0.f};
  int best[2] = {0, 0};
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  int rc = QISG_OK;
  for (int i = 0; i < 3 && !rc; ++i) rc = cuda_check(cudaEventCreate(&ev[i]), "event");
  const bool graphs = h->use_graphs;
  h->use_graphs = false;
  for (int c = 0; c < n_cand && !rc; ++c) {
    const int tile = kTiles[c % n_tiles], variant = c / n_tiles;
    h->sweep_tile[0] = h->sweep_tile[1] = tile;
    h->sweep_variant[0] = h->sweep_variant[1] = variant;
    rc = one_sweep(h);   // warm the candidate
    float ms[2] = {0.f, 0.f};
    for (int i = 0; i < sweeps_per_candidate && !rc; ++i) {
      rc = one_sweep(h, ev);
      if (!rc) rc = cuda_check(cudaEventSynchronize(ev[2]), "sync");
      float a = 0.f, b = 0.f;
      if (!rc) rc = cuda_check(cudaEventElapsedTime(&a, ev[0], ev[1]), "elapsed");
      if (!rc) rc = cuda_check(cudaEventElapsedTime(&b, ev[1], ev[2]), "elapsed");
      ms[0] += a;
      ms[1] += b;
    }
    for (int col = 0; col < 2 && !rc; ++col)
      if (best[col] == 0 || ms[col] < best_ms[col]) {
        best[col] = c + 1;
        best_ms[col] = ms[col];
      }
  }
  for (int i = 0; i < 3; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  h->use_graphs = graphs;
  if (rc) return rc;
  for (int col = 0; col < 2; ++col) {
    h->sweep_tile[col] = kTiles[(best[col] - 1) % n_tiles];
    h->sweep_variant[col] = (best[col] - 1) / n_tiles;
  }
  drop_cycle(h);
  if (chosen) *chosen = h->sweep_tile[1];
  return QISG_OK;
}

int qisg_get_tiles(qisg_handle *h, int tile[2], int variant[2]) {
  if (!h || !tile || !variant) return fail(QISG_EINVAL, "NULL argument");
  for (int c = 0; c < 2; ++c) {
    tile[c] = h->sweep_tile[c];
    variant[c] = h->sweep_variant[c];
  }
  return QISG_OK;
}

int qisg_set_tiles(qisg_handle *h, const int tile[2], const int variant[2]) {
  if (!h || !tile || !variant) return fail(QISG_EINVAL, "NULL argument");
  for (int c = 0; c < 2; ++c)
    if (tile[c] < 0 || tile[c] > 64 || variant[c] < 0 || variant[c] > 2)
      return fail(QISG_EINVAL, "tile must be 0 .. 64, variant 0, 1 or 2");
  int rc = sync_handle(h);
  if (rc) return rc;
  for (int c = 0; c < 2; ++c) {
    h->sweep_tile[c] = tile[c];
    h->sweep_variant[c] = variant[c];
  }
  drop_cycle(h);
  return QISG_OK;
}

int qisg_pt_swap(qisg_handle *h) {
  if (!h) return fail(QISG_EINVAL, "NULL handle");
  if (h->needs_state) return fail(QISG_ESTATE, "energies were replaced by qisg_pt_given: call qisg_set_state");
  if (h->t == 0) return fail(QISG_ESTATE, "no sweep has run yet");
  return h->layout != QISG_LAYOUT_SAMPLES ? lanes_pt(h, 1) : samples_pt(h, 1, 0);
}

int qisg_energies(qisg_handle *h, int64_t *A, int64_t *B) {
  if (!h || !A || !B) return fail(QISG_EINVAL, "NULL argument");
  int rc = h->layout != QISG_LAYOUT_SAMPLES ? lanes_energies_by_slot(h) : samples_energies_by_slot(h);
  if (rc) return rc;
  const size_t n = (size_t)h->n_samples * h->n_rep * h->n_slots;
  const size_t stride = (size_t)h->n_a_pad * h->n_rep * h->n_slots;
  rc = cuda_check(cudaMemcpyAsync(A, h->d_out, n * 8, cudaMemcpyDeviceToHost, h->stream), "copy A");
  if (!rc) rc = cuda_check(cudaMemcpyAsync(B, h->d_out + stride, n * 8, cudaMemcpyDeviceToHost, h->stream),
                           "copy B");
  if (!rc) rc = sync_handle(h);
  return rc;
}

int qisg_overlaps(qisg_handle *h, int64_t *q) {
  if (!h || !q) return fail(QISG_EINVAL, "NULL argument");
  const int n_pairs = h->n_pairs();
  if (n_pairs == 0) return QISG_OK;
  int rc = h->layout == QISG_LAYOUT_LANES ? lanes_measure(h, 1)
           : h->layout == QISG_LAYOUT_SITES ? sites_measure(h, 1)
                                             : samples_measure(h, 1);
  if (rc) return rc;
  const size_t n = (size_t)h->n_samples * h->n_slots * n_pairs;
  rc = cuda_check(cudaMemcpyAsync(q, h->d_q, n * 8, cudaMemcpyDeviceToHost, h->stream), "copy q");
  if (!rc) rc = cuda_check(cudaMemsetAsync(h->d_q, 0, (size_t)h->n_a_pad * h->n_slots * n_pairs * 8, h->stream),
                           "memset");
  if (!rc) rc = sync_handle(h);
  return rc;
}

int qisg_permutation(qisg_handle *h, int32_t *walker_at) {
  if (!h || !walker_at) return fail(QISG_EINVAL, "NULL argument");
  const size_t n = (size_t)h->n_samples * h->n_rep * h->n_slots;
  int rc = cuda_check(cudaMemcpyAsync(walker_at, h->d_walker, n * 4, cudaMemcpyDeviceToHost, h->stream),
                      "copy walker");
  if (!rc) rc = sync_handle(h);
  return rc;
}

int qisg_get_spins(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *S) {
  if (!h || (!S && n_a > 0)) return fail(QISG_EINVAL, "NULL argument");
  if (a_lo < 0 || n_a < 0 || a_lo + n_a > h->n_samples) return fail(QISG_EINVAL, "sample range");
  int rc = sync_handle(h);
  if (rc) return rc;
  return h->layout == QISG_LAYOUT_LANES   ? lanes_get_spins(h, a_lo, n_a, S)
         : h->layout == QISG_LAYOUT_SITES ? sites_get_spins(h, a_lo, n_a, S)
                                          : samples_get_spins(h, a_lo, n_a, S);
}

int qisg_get_couplings(qisg_handle *h, int64_t a_lo, int64_t n_a, int8_t *J) {
  if (!h || (!J && n_a > 0)) return fail(QISG_EINVAL, "NULL argument");
  if (a_lo < 0 || n_a < 0 || a_lo + n_a > h->n_samples) return fail(QISG_EINVAL, "sample range");
  int rc = sync_handle(h);
  if (rc) return rc;
  return h->layout != QISG_LAYOUT_SAMPLES ? lanes_get_couplings(h, a_lo, n_a, J)
                                          : samples_get_couplings(h, a_lo, n_a, J);
}

int qisg_set_couplings(qisg_handle *h, const int8_t *J) {
  if (!h || !J) return fail(QISG_EINVAL, "NULL argument");
  const int64_t n = h->n_samples * h->L * h->L * 2;
  for (int64_t i = 0; i < n; ++i)
    if (J[i] != 1 && J[i] != -1) return fail(QISG_EINVAL, "couplings must be +-1");
  int rc = sync_handle(h);
  if (!rc) rc = h->layout != QISG_LAYOUT_SAMPLES ? lanes_set_couplings(h, J) : samples_set_couplings(h, J);
  if (!rc) rc = recompute_energies(h);
  if (!rc) rc = sync_handle(h);
  return rc;
}

// Every byte of S[0 .. n) is +1 or -1: (s + 1) & 0xFD == 0, a loop the
// compiler vectorises, split over host threads for large states.
static bool spins_are_pm1(const int8_t *S, int64_t n) {
  auto scan = [S](int64_t lo, int64_t hi) {
    uint8_t bad = 0;
    for (int64_t i = lo; i < hi; ++i) bad |= (uint8_t)((uint8_t)S[i] + 1u) & 0xFDu;
    return bad == 0;
  };
  const int64_t per = int64_t(1) << 24;
  const int nt = (int)std::min<int64_t>(std::max(1u, std::min(16u, std::thread::hardware_concurrency())),
                                        (n + per - 1) / per);
  if (nt <= 1) return scan(0, n);
  std::vector<char> ok((size_t)nt, 1);
  std::vector<std::thread> pool;
  for (int k = 0; k < nt; ++k)
    pool.emplace_back([&, k] { ok[(size_t)k] = scan(n * k / nt, n * (k + 1) / nt) ? 1 : 0; });
  for (auto &th : pool) th.join();
  return std::all_of(ok.begin(), ok.end(), [](char c) { return c != 0; });
}

int qisg_set_state(qisg_handle *h, const int8_t *S, const int32_t *walker_at, uint64_t sweep) {
  if (!h || !S || !walker_at) return fail(QISG_EINVAL, "NULL argument");
  const int64_t rows = h->n_samples * h->n_rep;
  std::vector<char> seen((size_t)h->n_slots);
  for (int64_t c = 0; c < rows; ++c) {
    std::fill(seen.begin(), seen.end(), 0);
    for (int s = 0; s < h->n_slots; ++s) {
      const int32_t w = walker_at[c * h->n_slots + s];
      if (w < 0 || w >= h->n_slots || seen[(size_t)w]) return fail(QISG_ECORRUPT, "walker_at row is not a permutation");
      seen[(size_t)w] = 1;
    }
  }
  const int64_t nS = rows * h->n_slots * h->N;
  int rc = sync_handle(h);
  if (rc) return rc;
  // SAMPLES states up to 256 MB go up in one copy and are checked on the
  // device before anything of the handle changes; others are checked here
  int8_t *d_S = nullptr;
  if (h->layout == QISG_LAYOUT_SAMPLES && nS <= ((int64_t)256 << 20)) {
    rc = samples_upload_checked(h, S, nS, &d_S);
    if (rc) return rc;
  } else if (!spins_are_pm1(S, nS)) {
    return fail(QISG_ECORRUPT, "spins must be +-1");
  }
  // the permutation first (padding lanes keep the identity): SAMPLES packs by
  // slot with the device labels
  std::vector<int32_t> wa((size_t)h->n_a_pad * h->n_rep * h->n_slots);
  for (size_t i = 0; i < wa.size(); ++i) wa[i] = (int32_t)(i % h->n_slots);
  std::memcpy(wa.data(), walker_at, (size_t)rows * h->n_slots * 4);
  rc = cuda_check(cudaMemcpyAsync(h->d_walker, wa.data(), wa.size() * 4, cudaMemcpyHostToDevice, h->stream),
                  "copy walker");
  if (!rc)
    rc = h->layout == QISG_LAYOUT_LANES   ? lanes_set_spins(h, S)
         : h->layout == QISG_LAYOUT_SITES ? sites_set_spins(h, S)
                                          : samples_set_spins(h, S, walker_at, d_S);
  if (d_S) cudaFree(d_S);
  if (rc) return rc;
  unsigned long long tt = sweep;
  rc = cuda_check(cudaMemcpyAsync(h->d_t, &tt, 8, cudaMemcpyHostToDevice, h->stream), "copy t");
  const size_t n_cs = (size_t)h->n_a_pad * h->n_rep * h->n_slots;
  const size_t qn = (size_t)h->n_a_pad * h->n_slots * (h->n_pairs() > 0 ? h->n_pairs() : 1);
  if (!rc) rc = cuda_check(cudaMemsetAsync(h->d_sumA, 0, n_cs * 8, h->stream), "memset");
  if (!rc) rc = cuda_check(cudaMemsetAsync(h->d_sumB, 0, n_cs * 8, h->stream), "memset");
  if (!rc) rc = cuda_check(cudaMemsetAsync(h->d_sumq, 0, qn * 8, h->stream), "memset");
  if (!rc) rc = cuda_check(cudaMemsetAsync(h->d_sumq2, 0, qn * 8, h->stream), "memset");
  if (!rc) rc = cuda_check(cudaMemsetAsync(h->d_q, 0, qn * 8, h->stream), "memset");
  if (!rc) rc = cuda_check(cudaMemsetAsync(h->d_meas, 0, 8, h->stream), "memset");
  if (!rc) rc = recompute_energies(h);
  if (!rc) rc = sync_handle(h);
  if (!rc) {
    h->t = sweep;
    h->n_meas = 0;
    h->rec_base = 0;
    h->needs_state = false;
  }
  return rc;
}

int qisg_pt_given(qisg_handle *h, const int64_t *U, int32_t *walker_at, uint64_t t, int wide) {
  if (!h || !U || !walker_at) return fail(QISG_EINVAL, "NULL argument");
  if (wide != 0 && wide != 1) return fail(QISG_EINVAL, "wide must be 0 or 1");
  if (h->n_slots > kMaxSlotsPT) return fail(QISG_EINVAL, "ladder longer than the PT kernel takes");
  const bool w64 = wide || 2 * h->N >= (int64_t(1) << 30);
  const int64_t lim = w64 ? (int64_t(1) << 38) : (int64_t(1) << 29);
  const int64_t rows = h->n_samples * h->n_rep;
  const int64_t n_u = rows * h->n_slots * 2;
  for (int64_t i = 0; i < n_u; ++i)
    if (U[i] < 0 || U[i] >= lim) return fail(QISG_EINVAL, "bond count outside the energy width");
  std::vector<char> seen((size_t)h->n_slots);
  for (int64_t c = 0; c < rows; ++c) {
    std::fill(seen.begin(), seen.end(), 0);
    for (int s = 0; s < h->n_slots; ++s) {
      const int32_t w = walker_at[c * h->n_slots + s];
      if (w < 0 || w >= h->n_slots || seen[(size_t)w]) return fail(QISG_ECORRUPT, "walker_at row is not a permutation");
      seen[(size_t)w] = 1;
    }
  }
  int rc = sync_handle(h);
  if (rc) return rc;
  const size_t n_cs = (size_t)h->n_a_pad * h->n_rep * h->n_slots;
  std::vector<int32_t> wa(n_cs);
  for (size_t i = 0; i < n_cs; ++i) wa[i] = (int32_t)(i % h->n_slots);
  std::memcpy(wa.data(), walker_at, (size_t)rows * h->n_slots * 4);
  // LANES and SITES count by walker, SAMPLES by slot
  std::vector<unsigned long long> u(n_cs * 2, 0ull);
  const bool by_slot = h->layout == QISG_LAYOUT_SAMPLES;
  for (int64_t c = 0; c < rows; ++c)
    for (int s = 0; s < h->n_slots; ++s) {
      const int64_t src = c * h->n_slots + (by_slot ? wa[(size_t)(c * h->n_slots + s)] : s);
      u[(size_t)(c * h->n_slots + s) * 2] = (unsigned long long)U[src * 2];
      u[(size_t)(c * h->n_slots + s) * 2 + 1] = (unsigned long long)U[src * 2 + 1];
    }
  h->needs_state = true;
  h->perm_pending = false;
  drop_cycle(h);
  unsigned long long tt[2] = {t + 1ull, t + 1ull};   // an explicit pass reads the sweep it follows as t + 1 - 1
  rc = cuda_check(cudaMemcpyAsync(h->d_walker, wa.data(), n_cs * 4, cudaMemcpyHostToDevice, h->stream), "copy walker");
  if (!rc) rc = cuda_check(cudaMemcpyAsync(h->d_U, u.data(), u.size() * 8, cudaMemcpyHostToDevice, h->stream), "copy U");
  if (!rc) rc = cuda_check(cudaMemcpyAsync(h->d_t, tt, 16, cudaMemcpyHostToDevice, h->stream), "copy t");
  if (!rc && h->d_acc)
    rc = cuda_check(cudaMemsetAsync(h->d_acc, 0, (size_t)h->n_b * h->n_rep * h->n_slots * (h->W / 8), h->stream),
                    "clear PT masks");
  if (!rc) rc = pt_pass(h, 1, 0, h->n_samples, nullptr, wide != 0);
  if (!rc) rc = cuda_check(cudaMemcpyAsync(walker_at, h->d_walker, (size_t)rows * h->n_slots * 4,
                                           cudaMemcpyDeviceToHost, h->stream), "copy walker");
  if (!rc) rc = sync_handle(h);
  return rc;
}

int qisg_measurements(qisg_handle *h, int64_t *sumA, int64_t *sumB, int64_t *sumq, int64_t *sumq2,
                      int64_t *n_meas) {
  if (!h) return fail(QISG_EINVAL, "NULL handle");
  int rc = QISG_OK;
  const size_t ncs = (size_t)h->n_samples * h->n_rep * h->n_slots;
  const size_t nq = (size_t)h->n_samples * h->n_slots * h->n_pairs();
  if (sumA) rc = cuda_check(cudaMemcpyAsync(sumA, h->d_sumA, ncs * 8, cudaMemcpyDeviceToHost, h->stream), "copy");
  if (!rc && sumB) rc = cuda_check(cudaMemcpyAsync(sumB, h->d_sumB, ncs * 8, cudaMemcpyDeviceToHost, h->stream), "copy");
  if (!rc && sumq && nq) rc = cuda_check(cudaMemcpyAsync(sumq, h->d_sumq, nq * 8, cudaMemcpyDeviceToHost, h->stream), "copy");
  if (!rc && sumq2 && nq) rc = cuda_check(cudaMemcpyAsync(sumq2, h->d_sumq2, nq * 8, cudaMemcpyDeviceToHost, h->stream), "copy");
  if (!rc) rc = sync_handle(h);
  if (!rc && n_meas) *n_meas = h->n_meas;
  return rc;
}

int qisg_slot_means(qisg_handle *h, double *e_s, double *e_t, double *q2) {
  if (!h || !e_s || !e_t || !q2) return fail(QISG_EINVAL, "NULL argument");
  if (h->n_meas == 0) return fail(QISG_ESTATE, "no measurement taken yet");
  const int n_pairs = h->n_pairs();
  std::vector<int64_t> A((size_t)h->n_samples * h->n_rep * h->n_slots), B(A.size()),
      Q2((size_t)h->n_samples * h->n_slots * (n_pairs > 0 ? n_pairs : 1), 0);
  int rc = qisg_measurements(h, A.data(), B.data(), nullptr, n_pairs ? Q2.data() : nullptr, nullptr);
  if (rc) return rc;
  const double m = (double)h->n_meas, N = (double)h->N;
  for (int s = 0; s < h->n_slots; ++s) {
    double sa = 0.0, sb = 0.0, sq = 0.0;
    for (int64_t a = 0; a < h->n_samples; ++a)
      for (int r = 0; r < h->n_rep; ++r) {
        sa += (double)A[((size_t)a * h->n_rep + r) * h->n_slots + s];
        sb += (double)B[((size_t)a * h->n_rep + r) * h->n_slots + s];
      }
    for (int64_t a = 0; a < h->n_samples; ++a)
      for (int p = 0; p < n_pairs; ++p) sq += (double)Q2[((size_t)a * h->n_slots + s) * n_pairs + p];
    e_s[s] = sa / (m * (double)h->n_samples * (double)h->n_rep * 2.0 * N);
    e_t[s] = sb / (m * (double)h->n_samples * (double)h->n_rep * N);
    q2[s] = sq / (m * (double)h->n_samples * (double)(n_pairs > 0 ? n_pairs : 1) * N * N);
  }
  return QISG_OK;
}

int qisg_thresholds(qisg_handle *h, uint32_t *T) {
  if (!h || !T) return fail(QISG_EINVAL, "NULL argument");
  std::memcpy(T, h->T.data(), h->T.size() * 4);
  return QISG_OK;
}

int qisg_sweep_count(qisg_handle *h, uint64_t *t) {
  if (!h || !t) return fail(QISG_EINVAL, "NULL argument");
  *t = h->t;
  return QISG_OK;
}

int qisg_layout(qisg_handle *h, int *layout, int *word_bits) {
  if (!h) return fail(QISG_EINVAL, "NULL handle");
  if (layout) *layout = h->layout;
  if (word_bits) *word_bits = h->W;
  return QISG_OK;
}

int qisg_launch_count(qisg_handle *h, int64_t *n) {
  if (!h || !n) return fail(QISG_EINVAL, "NULL argument");
  *n = h->launches;
  return QISG_OK;
}

int qisg_profile(qisg_handle *h, int enable) {
  if (!h) return fail(QISG_EINVAL, "NULL handle");
  int rc = sync_handle(h);
  if (rc) return rc;
  if (enable) prof_clear(h);
  // bit 0 (the half sweeps) times both internal sweep kinds
  const int bits = (enable & QISG_PROFILE_ONLY) ? (enable & 0xF) : 0xF;
  h->prof = !enable ? 0 : bits | ((bits & 1) << kProfBlue);
  return QISG_OK;
}

int qisg_profile_read(qisg_handle *h, int kind, double *total_ms, int64_t *n_timed,
                      int64_t *n_launched) {
  if (!h || kind < 0 || kind > QISG_KERNEL_RED) return fail(QISG_EINVAL, "bad handle or kind");
  int rc = sync_handle(h);
  if (rc) return rc;
  // public kind -> internal kinds: SWEEP = red + blue, RED = internal SWEEP
  int parts[2] = {kind, -1};
  if (kind == QISG_KERNEL_SWEEP) parts[1] = kProfBlue;
  if (kind == QISG_KERNEL_RED) parts[0] = QISG_KERNEL_SWEEP;
  double tot = 0.0;
  int64_t timed = 0, launched = 0;
  for (int k : parts) {
    if (k < 0) continue;
    const std::vector<cudaEvent_t> &v = h->prof_ev[k];
    for (size_t i = 0; i + 1 < v.size(); i += 2) {
      float ms = 0.f;
      rc = cuda_check(cudaEventElapsedTime(&ms, v[i], v[i + 1]), "event elapsed");
      if (rc) return rc;
      tot += ms;
    }
    timed += (int64_t)(v.size() / 2);
    launched += h->prof_launched[k];
  }
  if (total_ms) *total_ms = tot;
  if (n_timed) *n_timed = timed;
  if (n_launched) *n_launched = launched;
  return QISG_OK;
}

int qisg_sync(qisg_handle *h) {
  if (!h) return fail(QISG_EINVAL, "NULL handle");
  return sync_handle(h);
}

void qisg_destroy(qisg_handle *h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  void *ptrs[] = {h->spins, h->spins_alt, h->J, h->d_T, h->d_bases, h->d_sq, h->d_ptc, h->d_walker, h->d_U, h->d_sumA, h->d_sumB,
                  h->d_sumq, h->d_sumq2, h->d_q, h->d_out, h->d_t, h->d_acc, h->d_err, h->d_dcum, h->d_dlut,
                  h->d_meas, h->d_hist, h->d_blkA, h->d_blkB, h->d_bar};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  drop_cycle(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  prof_clear(h);
  delete h;
}

const char *qisg_strerror(int code) {
  switch (code) {
    case QISG_OK: return "ok";
    case QISG_EINVAL: return "invalid argument";
    case QISG_ENOMEM: return "out of device memory or over budget";
    case QISG_ECUDA: return "CUDA error";
    case QISG_ETIMEOUT: return "bounded device wait expired";
    case QISG_ECORRUPT: return "corrupt state";
    case QISG_ESTATE: return "call not valid in this state";
    default: return "unknown error";
  }
}

const char *qisg_last_error(void) { return g_last_error.c_str(); }

int qisg_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n,
                       void *cuda_stream) {
  if (n < 0 || (n > 0 && (!ctr || !key || !out))) return fail(QISG_EINVAL, "bad arguments");
  if (n == 0) return QISG_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  philox_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ctr, key, out, n);
  return cuda_check(cudaGetLastError(), "philox kernel");
}

}  // extern "C"
