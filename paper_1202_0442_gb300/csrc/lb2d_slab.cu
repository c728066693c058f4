// lb2d_slab.cu -- slabs of a lattice split by the processors command: the
// halo rows between neighbouring slabs, exchanged device to device in one
// process (lb_exchange) or packed into messages for other ranks
// (lb_halo_pack / lb_halo_unpack).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "lb2d.h"
#include "lbapi.h"
#include "lbbatch.h"
#include "lbctx.h"
#include "lbint.h"

using namespace lbk;

// ======================================================================
// slabs (processors command): the halo rows between neighbouring slabs
// ======================================================================

namespace {

struct Run {
  uint8_t *p;
  size_t bytes;
};

// The rows of the current state buffers across face `face` of a slab (0:
// its low-y side, 1: its high-y side): the rows it sends (ghost = false:
// its first or last `halo` own rows) or the ghost rows it receives into
// (ghost = true), one run per population plane.  With one ghost row only
// the populations the pull takes across the face travel (e_y = +1 for data
// moving towards +y, e_y = -1 for data moving towards -y); with two ghost
// rows every population does.
void face_runs(lb_ctx *ctx, int face, bool ghost, std::vector<Run> &runs) {
  runs.clear();
  const Geometry &g = ctx->g;
  const int H = ctx->halo;
  const size_t r0 = (size_t)(face == 0 ? (ghost ? 0 : g.ylo) : (ghost ? g.yhi : g.yhi - H));
  const int dir = ((face == 1) != ghost) ? 1 : -1;  // e_y of the data crossing
  const size_t row = (size_t)g.pitch, sb = storage_bytes(ctx->storage);
  for (int c = 0; c < ctx->nc; c++)
    for (int q = 0; q < 9; q++)
      if (H > 1 || EYD[q] == dir)
        runs.push_back({(uint8_t *)ctx->fbuf[ctx->cur] + (((size_t)c * 9 + q) * g.plane + r0 * row) * sb, H * row * sb});
  for (int q = 0; q < ctx->qs; q++) {
    const int ey = ctx->qs == 4 ? EY4D[q] : EYD[q];
    if (H > 1 || ey == dir)
      runs.push_back({(uint8_t *)ctx->gbuf[ctx->cur] + ((size_t)q * g.plane + r0 * row) * 4, H * row * 4});
  }
  if (ctx->react) {
    // growth changes the mask and the deposits: their rows travel too
    runs.push_back({(uint8_t *)(ctx->mask + r0 * g.mw), H * (size_t)g.mw * 4});
    runs.push_back({(uint8_t *)(ctx->b + r0 * row), H * row * 8});
  }
}

// after ghost rows of a slab with surface reaction changed (face 0, 1 or
// -1 both), the neighbour codes of the rows whose 3 x 3 neighbourhood
// reaches them
int refresh_codes(lb_ctx *ctx, int face) {
  if (!ctx->react) return LB_OK;
  const Geometry &g = ctx->g;
  if (face != 1) LAUNCH(launch_nbcode(ctx->mask, ctx->nbc, g, ctx->stream, 0, g.ylo + 1));
  if (face != 0) LAUNCH(launch_nbcode(ctx->mask, ctx->nbc, g, ctx->stream, g.yhi - 1, g.ny));
  return LB_OK;
}

// device-to-device copies src[k] -> dst[k] of bytes[k], MAX_RUNS per launch
int copy_runs(lb_ctx *ctx, const std::vector<const void *> &src, const std::vector<void *> &dst,
              const std::vector<size_t> &bytes) {
  for (size_t k0 = 0; k0 < src.size(); k0 += MAX_RUNS) {
    CopyRuns r{};
    r.n = (int)std::min(src.size() - k0, (size_t)MAX_RUNS);
    for (int k = 0; k < r.n; k++) {
      r.src[k] = src[k0 + k];
      r.dst[k] = dst[k0 + k];
      r.bytes[k] = (unsigned)bytes[k0 + k];
    }
    LAUNCH(launch_copy_runs(r, ctx->stream));
  }
  return LB_OK;
}

int slab_check(lb_ctx *ctx) {
  if (ctx->rank < 0) return ctx->fail(LB_E_ORDER, "not a slab: call lb_processors(1, py) and lb_processor_rank first");
  if (!ctx->committed) return ctx->fail(LB_E_ORDER, "the slab has no device state yet: set its initial state first");
  return LB_OK;
}

// every slab's first and last own rows into its neighbours' ghost rows
// (periodic in y: slab py - 1 and slab 0 are neighbours)
}  // namespace

int exchange_slabs(lb_ctx *const *ctxs, int n) {
  std::vector<const void *> src;
  std::vector<void *> dst;
  std::vector<size_t> bytes;
  std::vector<Run> a, b;
  for (int r = 0; r < n; r++) {
    for (int face = 0; face < 2; face++) {
      lb_ctx *to = ctxs[face == 1 ? (r + 1) % n : (r + n - 1) % n];
      face_runs(ctxs[r], face, false, a);
      face_runs(to, 1 - face, true, b);
      for (size_t k = 0; k < a.size(); k++) {
        src.push_back(a[k].p);
        dst.push_back(b[k].p);
        bytes.push_back(a[k].bytes);
      }
    }
  }
  TRY(copy_runs(ctxs[0], src, dst, bytes));
  for (int r = 0; r < n; r++) TRY(refresh_codes(ctxs[r], -1));
  return LB_OK;
}

namespace {

// offset of each run in a packed halo message (16-byte aligned)
size_t pad16(size_t n) { return (n + 15) / 16 * 16; }

}  // namespace

extern "C" {

int lb_halo_size(lb_ctx *ctx, size_t *bytes) {
  NEED_CTX();
  if (!bytes) return ctx->fail(LB_E_ARG, "null output");
  TRY(slab_check(ctx));
  std::vector<Run> runs;
  face_runs(ctx, 1, false, runs);
  size_t n = 0;
  for (const Run &r : runs) n += pad16(r.bytes);
  *bytes = n;
  return LB_OK;
}

static int halo_move(lb_ctx *ctx, int face, void *buf, bool pack) {
  NEED_CTX();
  TRY(slab_check(ctx));
  if (face != 0 && face != 1) return ctx->fail(LB_E_ARG, "face must be 0 (low y) or 1 (high y)");
  if (!buf || (uintptr_t)buf % 16) return ctx->fail(LB_E_ARG, "halo buffer must be a 16-byte aligned device pointer");
  TRY(set_device(ctx));
  std::vector<Run> runs;
  face_runs(ctx, face, !pack, runs);
  std::vector<const void *> src;
  std::vector<void *> dst;
  std::vector<size_t> bytes;
  size_t off = 0;
  for (const Run &r : runs) {
    uint8_t *b = (uint8_t *)buf + off;
    src.push_back(pack ? (const void *)r.p : (const void *)b);
    dst.push_back(pack ? (void *)b : (void *)r.p);
    bytes.push_back(r.bytes);
    off += pad16(r.bytes);
  }
  TRY(copy_runs(ctx, src, dst, bytes));
  return pack ? LB_OK : refresh_codes(ctx, face);
}

int lb_halo_pack(lb_ctx *ctx, int face, void *buf) { return halo_move(ctx, face, buf, true); }

int lb_halo_unpack(lb_ctx *ctx, int face, const void *buf) { return halo_move(ctx, face, (void *)buf, false); }

int lb_exchange(lb_ctx *const *ctxs, int n) {
  NvtxRange range("lb_exchange");
  if (!ctxs || n < 1) return LB_E_ARG;
  for (int r = 0; r < n; r++)
    if (!ctxs[r]) return LB_E_ARG;
  lb_ctx *c0 = ctxs[0];
  for (int r = 0; r < n; r++) {
    lb_ctx *c = ctxs[r];
    TRY(slab_check(c));
    if (c->rank != r || c->py != n)
      return c->fail(LB_E_ARG, "lb_exchange takes the %d slabs of one lattice in rank order", c->py);
    if (c->nx != c0->nx || c->ny != c0->ny || c->nc != c0->nc || c->qs != c0->qs || c->storage != c0->storage ||
        c->halo != c0->halo || c->cur != c0->cur || c->t != c0->t)
      return c->fail(LB_E_ARG, "slab %d does not belong to the same lattice and step as slab 0", r);
    if (c->device != c0->device || c->stream != c0->stream)
      return c->fail(LB_E_UNSUPPORTED, "lb_exchange moves rows within one device and stream; "
                     "across devices use lb_halo_pack/lb_halo_unpack");
  }
  TRY(set_device(c0));
  return exchange_slabs(ctxs, n);
}

}  // extern "C"
