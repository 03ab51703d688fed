// lbm_checkpoint.cu -- self-describing checkpoints: a header naming the
// lattice, the current post-collision populations and the force history
// still held in the ring, guarded by a checksum, so that a truncated,
// corrupted or mismatched image is refused instead of restored.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "lbm_ctx.h"
#include "lbm_host.h"

using namespace gblbm;

namespace {

constexpr char kMagic[8] = {'G', 'B', 'L', 'B', 'M', 'C', 'K', '1'};
constexpr uint32_t kVersion = 1;

// Fixed little-endian layout (the host ABI of every supported machine).
struct CkHeader {
  char magic[8];
  uint32_t version, header_bytes;
  int32_t nx, ny, storage, collision, bc, bounce;
  double tau, U;
  uint64_t history_count;    // lbm_force_count at the time of the checkpoint
  uint64_t history_entries;  // entries stored: [history_count - n, history_count)
  uint64_t payload_bytes;    // populations then history
  uint64_t checksum;         // over the payload
};
static_assert(sizeof(CkHeader) == 88, "checkpoint header layout");

// FNV-1a (Fowler, Noll, Vo) taken over little-endian 64-bit words instead of
// bytes; a short tail is zero-padded.  Every step (xor with a word, multiply
// by an odd constant) is a bijection of the running state, so an image that
// differs from the original in any single word always gives another sum.
uint64_t checksum64(const unsigned char *p, size_t n, uint64_t h) {
  const uint64_t prime = 0x100000001b3ull;
  size_t i = 0;
  for (; i + 8 <= n; i += 8) {
    uint64_t w;
    std::memcpy(&w, p + i, 8);
    h = (h ^ w) * prime;
  }
  if (i < n) {
    uint64_t w = 0;
    std::memcpy(&w, p + i, n - i);
    h = (h ^ w) * prime;
  }
  return h;
}
constexpr uint64_t kBasis = 0xcbf29ce484222325ull;

size_t pop_bytes(const lbm_ctx *c) { return (size_t)9 * c->nx * c->ny * c->elem; }

int history_now(lbm_ctx *c, int64_t *count, int64_t *entries) {
  int rc = lbm_force_count(c, count);
  if (rc) return rc;
  *entries = std::min<int64_t>(*count, c->hist_cap);
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_checkpoint_bytes(lbm_ctx *c, size_t *bytes) {
  if (!c || !bytes) return LBM_ERR_ARG;
  int64_t count = 0, entries = 0;
  const int rc = history_now(c, &count, &entries);
  if (rc) return rc;
  *bytes = sizeof(CkHeader) + pop_bytes(c) + (size_t)entries * 2 * sizeof(double);
  return LBM_OK;
}

int lbm_checkpoint_save(lbm_ctx *c, void *dst, size_t bytes) {
  if (!c || !dst) return LBM_ERR_ARG;
  int64_t count = 0, entries = 0;
  int rc = history_now(c, &count, &entries);
  if (rc) return rc;
  const size_t pb = pop_bytes(c), hb = (size_t)entries * 2 * sizeof(double);
  if (bytes != sizeof(CkHeader) + pb + hb) return LBM_ERR_ARG;
  unsigned char *out = (unsigned char *)dst;
  unsigned char *pay = out + sizeof(CkHeader);
  rc = lbm_get_populations(c, pay, pb);
  if (rc) return rc;
  if (entries > 0) {
    rc = lbm_forces_raw(c, count - entries, entries, (double *)(pay + pb));
    if (rc) return rc;
  }
  CkHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  h.header_bytes = (uint32_t)sizeof(CkHeader);
  h.nx = c->nx;
  h.ny = c->ny;
  h.storage = c->o.storage;
  h.collision = c->o.collision;
  h.bc = c->o.bc_top_bottom;
  h.bounce = c->o.bounce;
  h.tau = c->o.tau;
  h.U = c->o.U;
  h.history_count = (uint64_t)count;
  h.history_entries = (uint64_t)entries;
  h.payload_bytes = pb + hb;
  h.checksum = checksum64(pay, pb + hb, kBasis);
  std::memcpy(out, &h, sizeof(h));
  return LBM_OK;
}

int lbm_checkpoint_load(lbm_ctx *c, const void *src, size_t bytes) {
  if (!c || !src || bytes < sizeof(CkHeader)) return LBM_ERR_ARG;
  CkHeader h;
  std::memcpy(&h, src, sizeof(h));
  if (std::memcmp(h.magic, kMagic, 8) != 0 || h.version != kVersion || h.header_bytes != sizeof(CkHeader))
    return LBM_ERR_ARG;
  // the image must describe this lattice
  if (h.nx != c->nx || h.ny != c->ny || h.storage != c->o.storage || h.collision != c->o.collision ||
      h.bc != c->o.bc_top_bottom || h.bounce != c->o.bounce || h.tau != c->o.tau || h.U != c->o.U)
    return LBM_ERR_ARG;
  const size_t pb = pop_bytes(c);
  if (h.history_entries > h.history_count ||
      h.payload_bytes != pb + h.history_entries * 2 * sizeof(double) || bytes != sizeof(CkHeader) + h.payload_bytes)
    return LBM_ERR_ARG;  // truncated, padded or inconsistent
  const unsigned char *pay = (const unsigned char *)src + sizeof(CkHeader);
  if (checksum64(pay, h.payload_bytes, kBasis) != h.checksum) return LBM_ERR_ARG;  // corrupted
  int rc = lbm_set_populations(c, pay, pb, (int64_t)h.history_count);
  if (rc) return rc;
  // history entries [count - n, count) back into their ring slots (the last
  // hist_cap of them if this context's ring is shorter)
  const int64_t count = (int64_t)h.history_count;
  const int64_t n = std::min<int64_t>((int64_t)h.history_entries, c->hist_cap);
  const double *hist = (const double *)(pay + pb) + 2 * ((int64_t)h.history_entries - n);
  CK(cudaSetDevice(c->dev));
  int64_t done = 0;
  while (done < n) {
    const int64_t e = count - n + done;
    const int64_t r = e % c->hist_cap;
    const int64_t run = std::min<int64_t>(n - done, c->hist_cap - r);
    CK(cudaMemcpyAsync(c->hist + 2 * r, hist + 2 * done, (size_t)run * 2 * sizeof(double), cudaMemcpyHostToDevice,
                       c->stream));
    done += run;
  }
  CK(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

}  // extern "C"
