// Checkpoint files: the paper writes spin configurations to disk at every
// block of maxit measurements, and they double as checkpoints for backup
// runs (Sec. 2.1 I/O, Appendix A: "simulation is a back-up or a new run").
// Here a checkpoint holds everything a bit-exact resume needs -- the
// problem (lattice, ladder, seed, cadences, boundary, update rule), the
// couplings, the spins by walker (one bit each), the PT permutation, the
// sweep counter and the measurement sums -- followed by a CRC-32 of all of
// it, which loading checks before it touches the handle (QISG_ECORRUPT).
// Host code only; the device is reached through the public getters/setters.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "qisg_internal.cuh"

namespace qisg {
namespace {

constexpr char kMagic[8] = {'Q', 'I', 'S', 'G', 'C', 'K', 'P', '1'};
constexpr uint32_t kVersion = 1;
constexpr uint32_t kHeaderBytes = 128;

// CRC-32 of IEEE 802.3 (reflected, polynomial 0xEDB88320, initial value and
// final complement 0xFFFFFFFF), table-driven, one byte at a time.
struct Crc32 {
  uint32_t table[256];
  Crc32() {
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t c = i;
      for (int b = 0; b < 8; ++b) c = (c & 1u) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
      table[i] = c;
    }
  }
  uint32_t update(uint32_t crc, const void *data, size_t n) const {
    const unsigned char *p = static_cast<const unsigned char *>(data);
    uint32_t c = ~crc;
    for (size_t i = 0; i < n; ++i) c = table[(c ^ p[i]) & 0xFFu] ^ (c >> 8);
    return ~c;
  }
};
const Crc32 &crc32() {
  static const Crc32 c;
  return c;
}

// Little-endian scalar I/O into a byte buffer (the layout is fixed, whatever
// the host's byte order).
void put_le(std::vector<unsigned char> &b, size_t at, uint64_t v, int bytes) {
  for (int i = 0; i < bytes; ++i) b[at + (size_t)i] = (unsigned char)(v >> (8 * i));
}
uint64_t get_le(const unsigned char *p, int bytes) {
  uint64_t v = 0;
  for (int i = 0; i < bytes; ++i) v |= (uint64_t)p[i] << (8 * i);
  return v;
}

struct Header {
  int L, Lt, n_slots, n_rep;
  int64_t n_samples;
  uint64_t seed, sweep;
  int64_t n_meas;
  int pt_every, measure_every, tau_ap, rule;
};

// Byte counts of the sections after the header.
struct Sections {
  size_t ladder, J, spins, walker, sums, total;   // total includes the header, excludes the CRC
};
bool sections_of(const Header &h, Sections *s) {
  if (h.L < 2 || h.Lt < 2 || h.n_slots < 1 || h.n_slots > 32 || h.n_rep < 1 || h.n_rep > 1024 || h.n_samples < 1)
    return false;
  const int64_t N = (int64_t)h.L * h.L * h.Lt;
  if (N > ((int64_t)1 << 31) || h.n_samples > ((int64_t)1 << 40)) return false;
  const int64_t rows = h.n_samples * h.n_rep * h.n_slots;
  const int64_t n_pairs = (int64_t)h.n_rep * (h.n_rep - 1) / 2;
  s->ladder = (size_t)h.n_slots * 16;
  s->J = (size_t)h.n_samples * h.L * h.L * 2;
  s->spins = (size_t)((rows * N + 7) / 8);
  s->walker = (size_t)rows * 4;
  s->sums = (size_t)rows * 16 + (size_t)(h.n_samples * h.n_slots * n_pairs) * 16;
  s->total = kHeaderBytes + s->ladder + s->J + s->spins + s->walker + s->sums;
  return true;
}

Header header_of(const qisg_handle *h) {
  Header x;
  x.L = h->L;
  x.Lt = h->Lt;
  x.n_slots = h->n_slots;
  x.n_rep = h->n_rep;
  x.n_samples = h->n_samples;
  x.seed = h->seed;
  x.sweep = h->t;
  x.n_meas = h->n_meas;
  x.pt_every = h->pt_every;
  x.measure_every = h->measure_every;
  x.tau_ap = h->tau_ap;
  x.rule = h->layout == QISG_LAYOUT_SITES ? 1 : 0;
  return x;
}

std::vector<unsigned char> encode_header(const Header &x) {
  std::vector<unsigned char> b(kHeaderBytes, 0);
  std::memcpy(b.data(), kMagic, 8);
  put_le(b, 8, kVersion, 4);
  put_le(b, 12, kHeaderBytes, 4);
  put_le(b, 16, (uint32_t)x.L, 4);
  put_le(b, 20, (uint32_t)x.Lt, 4);
  put_le(b, 24, (uint32_t)x.n_slots, 4);
  put_le(b, 28, (uint32_t)x.n_rep, 4);
  put_le(b, 32, (uint64_t)x.n_samples, 8);
  put_le(b, 40, x.seed, 8);
  put_le(b, 48, x.sweep, 8);
  put_le(b, 56, (uint64_t)x.n_meas, 8);
  put_le(b, 64, (uint32_t)x.pt_every, 4);
  put_le(b, 68, (uint32_t)x.measure_every, 4);
  put_le(b, 72, (uint32_t)x.tau_ap, 4);
  put_le(b, 76, (uint32_t)x.rule, 4);
  return b;
}

int decode_header(const unsigned char *b, Header *x) {
  if (std::memcmp(b, kMagic, 8) != 0) return fail(QISG_ECORRUPT, "checkpoint: bad magic");
  if (get_le(b + 8, 4) != kVersion || get_le(b + 12, 4) != kHeaderBytes)
    return fail(QISG_ECORRUPT, "checkpoint: unknown version or header size");
  x->L = (int)(int32_t)get_le(b + 16, 4);
  x->Lt = (int)(int32_t)get_le(b + 20, 4);
  x->n_slots = (int)(int32_t)get_le(b + 24, 4);
  x->n_rep = (int)(int32_t)get_le(b + 28, 4);
  x->n_samples = (int64_t)get_le(b + 32, 8);
  x->seed = get_le(b + 40, 8);
  x->sweep = get_le(b + 48, 8);
  x->n_meas = (int64_t)get_le(b + 56, 8);
  x->pt_every = (int)(int32_t)get_le(b + 64, 4);
  x->measure_every = (int)(int32_t)get_le(b + 68, 4);
  x->tau_ap = (int)(int32_t)get_le(b + 72, 4);
  x->rule = (int)(int32_t)get_le(b + 76, 4);
  for (uint32_t i = 80; i < kHeaderBytes; ++i)
    if (b[i]) return fail(QISG_ECORRUPT, "checkpoint: header padding is not zero");
  return QISG_OK;
}

// Read and check a whole file: header, sizes, CRC.  On success `data` holds
// every byte before the CRC.
int read_checked(const char *path, Header *x, Sections *sec, std::vector<unsigned char> *data) {
  if (!path) return fail(QISG_EINVAL, "NULL path");
  FILE *f = std::fopen(path, "rb");
  if (!f) return fail(QISG_EINVAL, std::string("cannot open checkpoint ") + path);
  unsigned char hb[kHeaderBytes];
  if (std::fread(hb, 1, kHeaderBytes, f) != kHeaderBytes) {
    std::fclose(f);
    return fail(QISG_ECORRUPT, "checkpoint: truncated header");
  }
  int rc = decode_header(hb, x);
  if (!rc && !sections_of(*x, sec)) rc = fail(QISG_ECORRUPT, "checkpoint: impossible sizes in the header");
  if (rc) {
    std::fclose(f);
    return rc;
  }
  data->resize(sec->total);
  std::memcpy(data->data(), hb, kHeaderBytes);
  const size_t rest = sec->total - kHeaderBytes;
  unsigned char tail[5];
  const size_t got = std::fread(data->data() + kHeaderBytes, 1, rest, f);
  const size_t got_crc = std::fread(tail, 1, 5, f);   // exactly 4 bytes must follow
  std::fclose(f);
  if (got != rest || got_crc != 4) return fail(QISG_ECORRUPT, "checkpoint: file size does not match its header");
  const uint32_t want = (uint32_t)get_le(tail, 4);
  if (crc32().update(0, data->data(), data->size()) != want) return fail(QISG_ECORRUPT, "checkpoint: CRC mismatch");
  return QISG_OK;
}

}  // namespace
}  // namespace qisg

using namespace qisg;

extern "C" {

int qisg_checkpoint_verify(const char *path, qisg_checkpoint_info *info) {
  Header x;
  Sections sec;
  std::vector<unsigned char> data;
  const int rc = read_checked(path, &x, &sec, &data);
  if (rc) return rc;
  if (info) {
    info->L = x.L;
    info->L_tau = x.Lt;
    info->n_slots = x.n_slots;
    info->n_replicas = x.n_rep;
    info->n_samples = x.n_samples;
    info->seed = x.seed;
    info->sweep = x.sweep;
    info->n_meas = x.n_meas;
    info->pt_every = x.pt_every;
    info->measure_every = x.measure_every;
    info->tau_antiperiodic = x.tau_ap;
    info->rule = x.rule;
  }
  return QISG_OK;
}

int qisg_checkpoint_save(qisg_handle *h, const char *path) {
  if (!h || !path) return fail(QISG_EINVAL, "NULL argument");
  const Header x = header_of(h);
  Sections sec;
  if (!sections_of(x, &sec)) return fail(QISG_EINVAL, "state too large for a checkpoint");
  const int64_t N = h->N, rows = h->n_samples * h->n_rep * h->n_slots;
  const int n_pairs = h->n_pairs();
  std::vector<int8_t> J((size_t)sec.J);
  std::vector<int32_t> wa((size_t)rows);
  std::vector<int64_t> sA((size_t)rows), sB((size_t)rows), sq((size_t)(h->n_samples * h->n_slots * n_pairs)),
      sq2(sq.size());
  int64_t n_meas = 0;
  int rc = qisg_get_couplings(h, 0, h->n_samples, J.data());
  if (!rc) rc = qisg_permutation(h, wa.data());
  if (!rc) rc = qisg_measurements(h, sA.data(), sB.data(), n_pairs ? sq.data() : nullptr,
                                  n_pairs ? sq2.data() : nullptr, &n_meas);
  if (rc) return rc;
  const std::string tmp = std::string(path) + ".tmp";
  FILE *f = std::fopen(tmp.c_str(), "wb");
  if (!f) return fail(QISG_EINVAL, std::string("cannot write ") + tmp);
  uint32_t crc = 0;
  bool ok = true;
  auto out = [&](const void *p, size_t n) {
    if (!ok || n == 0) return;
    crc = crc32().update(crc, p, n);
    ok = std::fwrite(p, 1, n, f) == n;
  };
  const std::vector<unsigned char> hb = encode_header(x);
  out(hb.data(), hb.size());
  std::vector<unsigned char> lad((size_t)sec.ladder);
  for (int s = 0; s < h->n_slots; ++s) {
    uint64_t a, b;
    std::memcpy(&a, &h->k[(size_t)s], 8);
    std::memcpy(&b, &h->kt[(size_t)s], 8);
    std::vector<unsigned char> tmpb(16);
    put_le(tmpb, 0, a, 8);
    put_le(tmpb, 8, b, 8);
    std::memcpy(&lad[(size_t)s * 16], tmpb.data(), 16);
  }
  out(lad.data(), lad.size());
  out(J.data(), J.size());
  // spins in chunks of samples (at most 256 MB of int8 at a time)
  const int64_t per_a = (int64_t)h->n_rep * h->n_slots * N;
  const int64_t chunk = std::max<int64_t>(1, ((int64_t)256 << 20) / per_a);
  std::vector<int8_t> S;
  unsigned char acc = 0;
  int nbits = 0;
  std::vector<unsigned char> packed;
  for (int64_t a0 = 0; a0 < h->n_samples && ok && !rc; a0 += chunk) {
    const int64_t na = std::min<int64_t>(chunk, h->n_samples - a0);
    S.resize((size_t)(na * per_a));
    rc = qisg_get_spins(h, a0, na, S.data());
    if (rc) break;
    packed.clear();
    packed.reserve(S.size() / 8 + 1);
    for (int8_t v : S) {
      acc |= (unsigned char)((v < 0 ? 1u : 0u) << nbits);
      if (++nbits == 8) {
        packed.push_back(acc);
        acc = 0;
        nbits = 0;
      }
    }
    out(packed.data(), packed.size());
  }
  if (nbits) out(&acc, 1);
  std::vector<unsigned char> buf;
  auto out_ints = [&](const void *p, size_t count, int bytes) {
    buf.assign(count * (size_t)bytes, 0);
    const unsigned char *q = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < count; ++i) {
      uint64_t v = 0;
      std::memcpy(&v, q + i * (size_t)bytes, (size_t)bytes);
      put_le(buf, i * (size_t)bytes, v, bytes);
    }
    out(buf.data(), buf.size());
  };
  out_ints(wa.data(), wa.size(), 4);
  out_ints(sA.data(), sA.size(), 8);
  out_ints(sB.data(), sB.size(), 8);
  out_ints(sq.data(), n_pairs ? sq.size() : 0, 8);
  out_ints(sq2.data(), n_pairs ? sq2.size() : 0, 8);
  unsigned char cb[4];
  for (int i = 0; i < 4; ++i) cb[i] = (unsigned char)(crc >> (8 * i));
  if (ok && !rc) ok = std::fwrite(cb, 1, 4, f) == 4;
  ok = (std::fclose(f) == 0) && ok;
  if (rc || !ok) {
    std::remove(tmp.c_str());
    return rc ? rc : fail(QISG_EINVAL, std::string("write failed: ") + tmp);
  }
  if (std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return fail(QISG_EINVAL, std::string("cannot rename to ") + path);
  }
  return QISG_OK;
}

int qisg_checkpoint_load(qisg_handle *h, const char *path) {
  if (!h) return fail(QISG_EINVAL, "NULL handle");
  Header x;
  Sections sec;
  std::vector<unsigned char> data;
  int rc = read_checked(path, &x, &sec, &data);
  if (rc) return rc;
  const Header mine = header_of(h);
  if (x.L != mine.L || x.Lt != mine.Lt || x.n_slots != mine.n_slots || x.n_rep != mine.n_rep ||
      x.n_samples != mine.n_samples || x.seed != mine.seed || x.pt_every != mine.pt_every ||
      x.measure_every != mine.measure_every || x.tau_ap != mine.tau_ap || x.rule != mine.rule)
    return fail(QISG_EINVAL, "checkpoint of another problem (lattice, ladder size, seed, cadence, boundary or rule)");
  const unsigned char *p = data.data() + kHeaderBytes;
  for (int s = 0; s < h->n_slots; ++s) {
    const uint64_t a = get_le(p + (size_t)s * 16, 8), b = get_le(p + (size_t)s * 16 + 8, 8);
    uint64_t ka, kb;
    std::memcpy(&ka, &h->k[(size_t)s], 8);
    std::memcpy(&kb, &h->kt[(size_t)s], 8);
    if (a != ka || b != kb) return fail(QISG_EINVAL, "checkpoint of another ladder");
  }
  p += sec.ladder;
  const int8_t *J = reinterpret_cast<const int8_t *>(p);
  p += sec.J;
  const int64_t N = h->N, rows = h->n_samples * h->n_rep * h->n_slots;
  std::vector<int8_t> S((size_t)(rows * N));
  for (size_t i = 0; i < S.size(); ++i) S[i] = ((p[i >> 3] >> (i & 7)) & 1u) ? int8_t(-1) : int8_t(1);
  p += sec.spins;
  std::vector<int32_t> wa((size_t)rows);
  for (size_t i = 0; i < wa.size(); ++i) wa[i] = (int32_t)(uint32_t)get_le(p + 4 * i, 4);
  p += sec.walker;
  const int n_pairs = h->n_pairs();
  const size_t nq = (size_t)(h->n_samples * h->n_slots * n_pairs);
  std::vector<int64_t> sums((size_t)rows * 2 + nq * 2);
  for (size_t i = 0; i < sums.size(); ++i) sums[i] = (int64_t)get_le(p + 8 * i, 8);
  // every value is checked before the handle is touched: couplings +-1,
  // rows of walker_at permutations (the spins are bits, always +-1)
  for (size_t i = 0; i < sec.J; ++i)
    if (J[i] != 1 && J[i] != -1) return fail(QISG_ECORRUPT, "checkpoint: a coupling is not +-1");
  std::vector<char> seen((size_t)h->n_slots);
  for (int64_t c = 0; c < h->n_samples * h->n_rep; ++c) {
    std::fill(seen.begin(), seen.end(), 0);
    for (int s = 0; s < h->n_slots; ++s) {
      const int32_t w = wa[(size_t)(c * h->n_slots + s)];
      if (w < 0 || w >= h->n_slots || seen[(size_t)w]) return fail(QISG_ECORRUPT, "checkpoint: walker_at row is not a permutation");
      seen[(size_t)w] = 1;
    }
  }
  rc = qisg_set_couplings(h, J);
  if (!rc) rc = qisg_set_state(h, S.data(), wa.data(), x.sweep);
  if (rc) return rc;
  long long *dst[4] = {h->d_sumA, h->d_sumB, h->d_sumq, h->d_sumq2};
  const size_t cnt[4] = {(size_t)rows, (size_t)rows, nq, nq};
  size_t off = 0;
  for (int k = 0; k < 4 && !rc; ++k) {
    if (cnt[k])
      rc = cuda_check(cudaMemcpyAsync(dst[k], sums.data() + off, cnt[k] * 8, cudaMemcpyHostToDevice, h->stream),
                      "restore sums");
    off += cnt[k];
  }
  const unsigned long long m = (unsigned long long)x.n_meas;
  if (!rc) rc = cuda_check(cudaMemcpyAsync(h->d_meas, &m, 8, cudaMemcpyHostToDevice, h->stream), "restore count");
  if (!rc) rc = handle_sync(h);
  if (!rc) {
    h->n_meas = x.n_meas;
    h->rec_base = x.n_meas;   // records from before the checkpoint are not in it
  }
  return rc;
}

}  // extern "C"
