// lb2d_batch.cu -- many independent lattices advanced by one persistent
// launch (lb_batch_*): the tile lists, the autotuner and its cache, and the
// captured graph of iterations.
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
// batched lattices
// ======================================================================

struct lb_batch {
  std::vector<lb_ctx *> ctxs;
  int device = 0;
  cudaStream_t stream = nullptr;
  int storage = ST_FP32;
  std::string err;
  uint64_t launches = 0;
  BatchLat *d_lat = nullptr;
  int4 *d_tiles = nullptr;
  unsigned int *d_counters = nullptr;
  unsigned int *d_tick = nullptr;
  std::vector<BatchLat> h_lat;
  int shape = 0, dynamic = 1, order = 1;
  int ntiles = 0, grid = 0;
  cudaGraphExec_t gexec = nullptr;
  int graph_steps = 0;
  // graphs are captured and replayed on a private stream (the caller's may
  // be the legacy default stream, which cannot be captured), fenced to the
  // caller's stream by events
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    err = buf;
    return code;
  }
};

namespace {

int batch_cuda(lb_batch *b, cudaError_t e, const char *what) {
  return b->fail(LB_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define BCK(call)                                            \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return batch_cuda(b, e_, #call);  \
  } while (0)

void drop_graph(lb_batch *b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  b->graph_steps = 0;
}

// tile list for the current shape and order: 0 = lattice by lattice,
// 1 = round robin over lattices, 2 = largest lattices first
int build_tiles(lb_batch *b) {
  const int TX = batch_shape_tx(b->shape), TY = batch_shape_ty(b->shape);
  std::vector<std::vector<int4>> per(b->ctxs.size());
  for (size_t l = 0; l < b->ctxs.size(); l++) {
    const lb_ctx *c = b->ctxs[l];
    for (int y0 = 0; y0 < c->ny; y0 += TY)
      for (int x0 = 0; x0 < c->nx; x0 += TX) per[l].push_back(make_int4((int)l, x0, y0, 0));
  }
  std::vector<int> idx(b->ctxs.size());
  for (size_t l = 0; l < idx.size(); l++) idx[l] = (int)l;
  if (b->order == 2)
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return per[a].size() > per[c].size(); });
  std::vector<int4> tiles;
  if (b->order == 1) {
    size_t maxn = 0;
    for (auto &v : per) maxn = std::max(maxn, v.size());
    for (size_t k = 0; k < maxn; k++)
      for (int l : idx)
        if (k < per[l].size()) tiles.push_back(per[l][k]);
  } else {
    for (int l : idx) tiles.insert(tiles.end(), per[l].begin(), per[l].end());
  }
  if (b->d_tiles) cudaFree(b->d_tiles);
  b->d_tiles = nullptr;
  BCK(cudaMalloc((void **)&b->d_tiles, tiles.size() * sizeof(int4)));
  BCK(cudaMemcpyAsync(b->d_tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream));
  b->ntiles = (int)tiles.size();
  int sms = 0;
  BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
  int occ = batch_occupancy(b->storage, b->shape);
  b->grid = std::max(1, std::min(b->ntiles, sms * std::max(occ, 1)));
  drop_graph(b);
  return LB_OK;
}

// refresh the per-lattice descriptors (a context may have been advanced on
// its own since the last batch call)
int sync_descs(lb_batch *b) {
  bool dirty = b->h_lat.empty();
  if (dirty) b->h_lat.resize(b->ctxs.size());
  for (size_t l = 0; l < b->ctxs.size(); l++) {
    lb_ctx *c = b->ctxs[l];
    BatchLat L{};
    L.nx = c->g.nx;
    L.ny = c->g.ny;
    L.pitch = c->g.pitch;
    L.mw = c->g.mw;
    L.plane = c->g.plane;
    L.buf[0] = c->fbuf[0];
    L.buf[1] = c->fbuf[1];
    L.cur = c->cur;
    L.mask = c->mask;
    L.nbc = c->nbc;
    L.rho_ref = (float)c->rho_ref[0];
    L.scale = c->scale;
    L.inv_scale = c->inv_scale;
    L.tau = (float)c->tau[0];
    L.omega = (float)(1.0 / c->tau[0]);
    L.pm = c->pm ? 1 : 0;
    L.sr = c->sr ? 1 : 0;
    L.fx = (float)c->fave[0][0];
    L.fy = (float)c->fave[0][1];
    L.ax = (float)c->acc[0][0];
    L.ay = (float)c->acc[0][1];
    if (memcmp(&L, &b->h_lat[l], sizeof L)) {
      b->h_lat[l] = L;
      dirty = true;
    }
  }
  if (dirty)
    BCK(cudaMemcpyAsync(b->d_lat, b->h_lat.data(), b->h_lat.size() * sizeof(BatchLat), cudaMemcpyHostToDevice,
                        b->stream));
  return LB_OK;
}

BatchLaunch launch_desc(lb_batch *b) {
  BatchLaunch L{};
  L.lat = b->d_lat;
  L.tiles = b->d_tiles;
  L.ntiles = b->ntiles;
  L.grid = b->grid;
  L.shape = b->shape;
  L.dynamic = b->dynamic;
  L.counters = b->d_counters;
  L.tick = b->d_tick;
  return L;
}

// LB_DEBUG_POISON on member contexts: NaN in the buffers the launch of
// this parity writes (every member's next population buffer)
int batch_poison(lb_batch *b, int parity) {
  for (lb_ctx *c : b->ctxs) {
    if (!(c->debug & LB_DEBUG_POISON)) continue;
    const int out = 1 - ((c->cur + parity) & 1);
    const cudaError_t e = cudaMemsetAsync(c->fbuf[out], 0xff, 9 * c->g.plane * storage_bytes(c->storage), b->stream);
    if (e != cudaSuccess) return batch_cuda(b, e, "poison");
  }
  return LB_OK;
}

bool batch_poisoned(const lb_batch *b) {
  for (const lb_ctx *c : b->ctxs)
    if (c->debug & LB_DEBUG_POISON) return true;
  return false;
}

int batch_direct(lb_batch *b, int parity0, int n) {
  BatchLaunch L = launch_desc(b);
  const bool poison = batch_poisoned(b);
  for (int k = 0; k < n; k++) {
    if (poison) {
      const int rc = batch_poison(b, (parity0 + k) & 1);
      if (rc != LB_OK) return rc;
    }
    if (launch_batch(b->storage, L, (parity0 + k) & 1, b->stream) < 0)
      return batch_cuda(b, cudaGetLastError(), "batch launch");
    b->launches++;
  }
  return LB_OK;
}

void batch_advance(lb_batch *b, int n) {
  for (lb_ctx *c : b->ctxs) {
    c->cur = (c->cur + n) & 1;
    c->t += n;
    c->fields_valid = false;
  }
  b->h_lat.clear();
}

constexpr int GRAPH_STEPS = 20;  // kernels per captured graph (even)

int ensure_graph(lb_batch *b) {
  if (b->gexec) return LB_OK;
  if (!b->gstream) {
    BCK(cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking));
    BCK(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
    BCK(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
  }
  cudaGraph_t graph = nullptr;
  BCK(cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeThreadLocal));
  BatchLaunch L = launch_desc(b);
  int bad = 0;
  for (int k = 0; k < GRAPH_STEPS; k++)
    if (launch_batch(b->storage, L, k & 1, b->gstream) < 0) bad = 1;
  cudaError_t e = cudaStreamEndCapture(b->gstream, &graph);
  if (bad || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return batch_cuda(b, e != cudaSuccess ? e : cudaGetLastError(), "graph capture");
  }
  e = cudaGraphInstantiate(&b->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return batch_cuda(b, e, "cudaGraphInstantiate");
  b->graph_steps = GRAPH_STEPS;
  return LB_OK;
}

}  // namespace

extern "C" {

int lb_batch_create(lb_ctx *const *ctxs, int n, lb_batch **out) {
  if (!out || !ctxs || n < 1) return LB_E_ARG;
  *out = nullptr;
  lb_batch *b = new (std::nothrow) lb_batch();
  if (!b) return LB_E_NOMEM;
  for (int k = 0; k < n; k++) {
    lb_ctx *c = ctxs[k];
    int rc = LB_OK;
    if (!c) rc = LB_E_ARG;
    else if (c->nc != 1 || c->qs || !c->open.empty() || c->sc || c->ads[0] || c->bstyle != 0 || c->rank >= 0)
      rc = c->fail(LB_E_UNSUPPORTED, "batched lattices are periodic single-component noslip lattices with body forces");
    else {
      for (int s = 0; s < c->nc && rc == LB_OK; s++)
        if (!c->painted_f[s] && !c->state_set[s]) rc = c->fail(LB_E_ORDER, "lattice %d has no initial state", k);
      if (rc == LB_OK) rc = commit(c);
    }
    if (rc == LB_OK && k > 0 && (c->device != ctxs[0]->device || c->stream != ctxs[0]->stream ||
                                 c->storage != ctxs[0]->storage))
      rc = LB_E_ARG;
    if (rc != LB_OK) {
      delete b;
      return rc;
    }
    b->ctxs.push_back(c);
  }
  b->device = ctxs[0]->device;
  b->stream = ctxs[0]->stream;
  b->storage = ctxs[0]->storage;
  if (cudaSetDevice(b->device) != cudaSuccess || cudaMalloc((void **)&b->d_lat, n * sizeof(BatchLat)) != cudaSuccess ||
      cudaMalloc((void **)&b->d_counters, 2 * sizeof(unsigned int)) != cudaSuccess ||
      cudaMemsetAsync(b->d_counters, 0, 2 * sizeof(unsigned int), b->stream) != cudaSuccess ||
      cudaMalloc((void **)&b->d_tick, 2 * sizeof(unsigned int)) != cudaSuccess ||
      cudaMemsetAsync(b->d_tick, 0, 2 * sizeof(unsigned int), b->stream) != cudaSuccess) {
    lb_batch_destroy(b);
    return LB_E_CUDA;
  }
  if (build_tiles(b) != LB_OK) {
    lb_batch_destroy(b);
    return LB_E_CUDA;
  }
  *out = b;
  return LB_OK;
}

int lb_batch_destroy(lb_batch *b) {
  if (!b) return LB_E_ARG;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  if (b->gstream) cudaStreamSynchronize(b->gstream);
  if (b->gstream) cudaStreamDestroy(b->gstream);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->d_lat) cudaFree(b->d_lat);
  if (b->d_tiles) cudaFree(b->d_tiles);
  if (b->d_counters) cudaFree(b->d_counters);
  if (b->d_tick) cudaFree(b->d_tick);
  delete b;
  return LB_OK;
}

const char *lb_batch_last_error(const lb_batch *b) { return b ? b->err.c_str() : "no batch"; }

int lb_batch_launch_count(const lb_batch *b, uint64_t *out) {
  if (!b || !out) return LB_E_ARG;
  *out = b->launches;
  return LB_OK;
}

int lb_batch_iteration(lb_batch *b, int Nt, int use_graph) {
  if (!b) return LB_E_ARG;
  NvtxRange range("lb_batch_iteration");
  if (Nt < 0) return b->fail(LB_E_ARG, "Nt must be >= 0");
  BCK(cudaSetDevice(b->device));
  int rc = sync_descs(b);
  if (rc != LB_OK) return rc;
  int done = 0;
  // poisoned members run without the graph (the poisoning is not captured)
  if (use_graph && !batch_poisoned(b)) {
    rc = ensure_graph(b);
    if (rc != LB_OK) return rc;
    if (Nt >= b->graph_steps) {
      BCK(cudaEventRecord(b->ev_in, b->stream));
      BCK(cudaStreamWaitEvent(b->gstream, b->ev_in, 0));
      while (Nt - done >= b->graph_steps) {
        BCK(cudaGraphLaunch(b->gexec, b->gstream));
        b->launches += (uint64_t)b->graph_steps;
        done += b->graph_steps;
      }
      BCK(cudaEventRecord(b->ev_out, b->gstream));
      BCK(cudaStreamWaitEvent(b->stream, b->ev_out, 0));
    }
  }
  rc = batch_direct(b, done & 1, Nt - done);
  if (rc != LB_OK) return rc;
  batch_advance(b, Nt);
  return LB_OK;
}

int lb_batch_autotune(lb_batch *b, const char *cache_json) {
  if (!b) return LB_E_ARG;
  BCK(cudaSetDevice(b->device));
  // cache key: device name, storage and the lattice shapes
  cudaDeviceProp prop;
  BCK(cudaGetDeviceProperties(&prop, b->device));
  uint64_t hsh = 1469598103934665603ULL;
  for (lb_ctx *c : b->ctxs) {
    hsh = (hsh ^ (uint64_t)c->nx) * 1099511628211ULL;
    hsh = (hsh ^ (uint64_t)c->ny) * 1099511628211ULL;
  }
  char key[512];
  snprintf(key, sizeof key, "%s|st%d|n%zu|%016llx", prop.name, b->storage, b->ctxs.size(), (unsigned long long)hsh);
  std::string cache;
  if (cache_json) {
    FILE *fp = fopen(cache_json, "rb");
    if (fp) {
      char buf[4096];
      size_t n;
      while ((n = fread(buf, 1, sizeof buf, fp)) > 0) cache.append(buf, n);
      fclose(fp);
    }
    size_t p = cache.find(std::string("\"") + key + "\"");
    if (p != std::string::npos) {
      int sh, dy, od;
      const char *q = strchr(cache.c_str() + p, '{');
      if (q && sscanf(q, "{\"shape\": %d, \"dynamic\": %d, \"order\": %d", &sh, &dy, &od) == 3 && sh >= 0 &&
          sh < BATCH_SHAPES) {
        b->shape = sh;
        b->dynamic = dy;
        b->order = od;
        return build_tiles(b);
      }
    }
  }
  // keep the lattices' states: time on them, then put the states back
  int rc = sync_descs(b);
  if (rc != LB_OK) return rc;
  std::vector<void *> saved(b->ctxs.size(), nullptr);
  std::vector<size_t> sizes(b->ctxs.size());
  for (size_t l = 0; l < b->ctxs.size(); l++) {
    lb_ctx *c = b->ctxs[l];
    sizes[l] = (size_t)9 * c->g.plane * storage_bytes(c->storage);
    BCK(cudaMalloc(&saved[l], sizes[l]));
    BCK(cudaMemcpyAsync(saved[l], c->fbuf[c->cur], sizes[l], cudaMemcpyDeviceToDevice, b->stream));
  }
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  float best = 1e30f;
  int bs = 0, bd = 1, bo = 1;
  const int reps = 6;
  for (int sh = 0; sh < BATCH_SHAPES; sh++)
    for (int dy = 0; dy < 2; dy++)
      for (int od = 0; od < 3; od++) {
        if (dy && od == 0) continue;  // dynamic hand-out makes lattice order moot
        b->shape = sh;
        b->dynamic = dy;
        b->order = od;
        rc = build_tiles(b);
        if (rc != LB_OK) return rc;
        rc = batch_direct(b, 0, 2);
        if (rc != LB_OK) return rc;
        BCK(cudaEventRecord(e0, b->stream));
        rc = batch_direct(b, 0, reps);
        if (rc != LB_OK) return rc;
        BCK(cudaEventRecord(e1, b->stream));
        BCK(cudaEventSynchronize(e1));
        float ms = 0;
        BCK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
          best = ms;
          bs = sh;
          bd = dy;
          bo = od;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // an even number of launches per candidate leaves buf[cur] the input
  for (size_t l = 0; l < b->ctxs.size(); l++) {
    lb_ctx *c = b->ctxs[l];
    BCK(cudaMemcpyAsync(c->fbuf[c->cur], saved[l], sizes[l], cudaMemcpyDeviceToDevice, b->stream));
  }
  BCK(cudaStreamSynchronize(b->stream));
  for (void *p : saved) cudaFree(p);
  b->shape = bs;
  b->dynamic = bd;
  b->order = bo;
  rc = build_tiles(b);
  if (rc != LB_OK) return rc;
  if (cache_json) {
    std::string entry = std::string("\"") + key + "\": {\"shape\": " + std::to_string(bs) +
                        ", \"dynamic\": " + std::to_string(bd) + ", \"order\": " + std::to_string(bo) +
                        ", \"ms_per_iter\": " + std::to_string(best / reps) + "}";
    std::string body;
    size_t l = cache.find('{'), r = cache.rfind('}');
    if (l != std::string::npos && r != std::string::npos && r > l) body = cache.substr(l + 1, r - l - 1);
    while (!body.empty() && isspace((unsigned char)body.back())) body.pop_back();
    std::string outs = "{" + body + (body.empty() ? "\n  " : ",\n  ") + entry + "\n}\n";
    FILE *fp = fopen(cache_json, "wb");
    if (fp) {
      fwrite(outs.data(), 1, outs.size(), fp);
      fclose(fp);
    }
  }
  return LB_OK;
}

}  // extern "C"
