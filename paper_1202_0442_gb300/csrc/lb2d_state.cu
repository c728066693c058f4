// lb2d_state.cu -- binary snapshots of a lattice's device state
// (lb_state_size, lb_save_state, lb_load_state): resume bit for bit.
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

extern "C" {

// snapshot layout: header, populations (current buffer), mask, solute
// populations, and with surface_reaction the precipitate, removed tallies
// and flip count (without it they stay zero and are not part of the state)
struct SnapHeader {
  uint64_t magic, nx, ny, nc, qs, storage, t;
};
static const uint64_t SNAP_MAGIC = 0x4c42324453543031ULL;  // "LB2DST01"

static void snap_parts(lb_ctx *ctx, std::vector<std::pair<void *, size_t>> &parts) {
  const Geometry &g = ctx->g;
  parts.clear();
  parts.push_back({ctx->fbuf[ctx->cur], (size_t)ctx->nc * 9 * g.plane * storage_bytes(ctx->storage)});
  parts.push_back({ctx->mask, (size_t)g.ny * g.mw * 4});
  if (ctx->qs) parts.push_back({ctx->gbuf[ctx->cur], (size_t)ctx->qs * g.plane * 4});
  if (ctx->react) {
    parts.push_back({ctx->b, g.plane * 8});
    parts.push_back({ctx->removed, (size_t)(ctx->nc + 1) * g.plane * 8});
    parts.push_back({ctx->nflips, 8});
  }
}

int lb_state_size(lb_ctx *ctx, size_t *bytes) {
  NEED_CTX();
  if (!bytes) return ctx->fail(LB_E_ARG, "null output");
  TRY(commit(ctx));
  std::vector<std::pair<void *, size_t>> parts;
  snap_parts(ctx, parts);
  size_t n = sizeof(SnapHeader);
  for (auto &p : parts) n += p.second;
  *bytes = n;
  return LB_OK;
}

int lb_save_state(lb_ctx *ctx, void *host, size_t bytes) {
  NEED_CTX();
  size_t need = 0;
  TRY(lb_state_size(ctx, &need));
  if (!host || bytes != need) return ctx->fail(LB_E_ARG, "snapshot buffer must be %zu bytes", need);
  TRY(set_device(ctx));
  SnapHeader h{SNAP_MAGIC, (uint64_t)ctx->nx, (uint64_t)ctx->ny, (uint64_t)ctx->nc, (uint64_t)ctx->qs,
               (uint64_t)ctx->storage, (uint64_t)ctx->t};
  memcpy(host, &h, sizeof h);
  std::vector<std::pair<void *, size_t>> parts;
  snap_parts(ctx, parts);
  size_t off = sizeof h;
  for (auto &p : parts) {
    CK(cudaMemcpyAsync((uint8_t *)host + off, p.first, p.second, cudaMemcpyDeviceToHost, ctx->stream));
    off += p.second;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return LB_OK;
}

int lb_load_state(lb_ctx *ctx, const void *host, size_t bytes) {
  NEED_CTX();
  ctx->fields_step = -1;  // the live state no longer matches the field planes
  size_t need = 0;
  TRY(lb_state_size(ctx, &need));
  if (!host || bytes != need) return ctx->fail(LB_E_ARG, "snapshot must be %zu bytes", need);
  SnapHeader h;
  memcpy(&h, host, sizeof h);
  if (h.magic != SNAP_MAGIC || h.nx != (uint64_t)ctx->nx || h.ny != (uint64_t)ctx->ny ||
      h.nc != (uint64_t)ctx->nc || h.qs != (uint64_t)ctx->qs || h.storage != (uint64_t)ctx->storage)
    return ctx->fail(LB_E_ARG, "snapshot does not match this lattice");
  TRY(set_device(ctx));
  std::vector<std::pair<void *, size_t>> parts;
  snap_parts(ctx, parts);
  size_t off = sizeof h;
  const uint8_t *mask_src = nullptr;
  for (auto &p : parts) {
    if (p.first == (void *)ctx->mask)
      mask_src = (const uint8_t *)host + off;  // below, once the other copies are queued
    else
      CK(cudaMemcpyAsync(p.first, (const uint8_t *)host + off, p.second, cudaMemcpyHostToDevice, ctx->stream));
    off += p.second;
  }
  // the mask and its neighbour codes only when the snapshot's mask differs
  // from the one on the device (compared on the host while the copies run)
  const size_t mbytes = ctx->mask_host.size() * 4;
  if (!(ctx->mask_host_valid && !memcmp(mask_src, ctx->mask_host.data(), mbytes))) {
    CK(cudaMemcpyAsync(ctx->mask, mask_src, mbytes, cudaMemcpyHostToDevice, ctx->stream));
    LAUNCH(launch_nbcode(ctx->mask, ctx->nbc, ctx->g, ctx->stream));
    ctx->slist_valid = false;
    memcpy(ctx->mask_host.data(), mask_src, mbytes);
    ctx->mask_host_valid = true;
  }
  ctx->t = (int64_t)h.t;
  if (ctx->fcount) CK(cudaMemsetAsync(ctx->fcount, 0, 2 * sizeof(unsigned int), ctx->stream));
  for (int c = 0; c < ctx->nc; c++) ctx->state_set[c] = true;
  if (ctx->qs) ctx->solute_set = true;
  return LB_OK;
}

}  // extern "C"
