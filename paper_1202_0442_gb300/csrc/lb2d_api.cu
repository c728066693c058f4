// lb2d_api.cu -- host side of the C ABI declared in include/lb2d.h.
//
// Holds the command state of one lattice (the paper's command set, Sec.
// Commands), checks command order and arguments the way the paper's module
// does (lattice before processors, boundary_style before obstacle,
// position0 before momentum0/concentration0, ...), paints the initial
// state on the host, moves it to the GPU at the first call that needs
// device memory, and then drives each iteration as a fixed sequence of
// kernel launches on the caller's stream:
//   fluid (k_fluid_local, k_fluid_sc or the fused k_fluid_solute) ->
//   gradient openings -> solute -> growth (gather, decisions and flips) ->
//   [thermo]
// Slabs and their halo exchange are in lb2d_slab.cu, snapshots in
// lb2d_state.cu, batched lattices in lb2d_batch.cu, the allocation-free
// thermo call in lb2d_static.cu, the input-data text files in lb2d_io.cu.
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

namespace {

int wall_of(const char *s) {
  if (!s) return -1;
  if (!strcmp(s, "xlo")) return 0;
  if (!strcmp(s, "xhi")) return 1;
  if (!strcmp(s, "ylo")) return 2;
  if (!strcmp(s, "yhi")) return 3;
  return -1;
}

}  // namespace

size_t storage_bytes(int st) { return st == ST_FP32 ? 4 : 2; }

namespace {

// equilibrium population i at density rho and velocity (ux, uy) (FP64,
// host side), with the density-ratio rest share of the fluids command
double feq_host(int i, double rho, double ux, double uy, double alpha) {
  const double usq = ux * ux + uy * uy, eu = EXD[i] * ux + EYD[i] * uy;
  return alpha == 4.0 / 9.0 ? W9D[i] * rho * (1 + 3 * eu + 4.5 * eu * eu - 1.5 * usq)
                            : wshare(i, alpha) * rho + W9D[i] * rho * (3 * eu + 4.5 * eu * eu - 1.5 * usq);
}

}  // namespace

int set_device(lb_ctx *ctx) {
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "cudaSetDevice");
  return LB_OK;
}

namespace {

bool fluid_ok(lb_ctx *ctx, int fluid) { return fluid >= 1 && fluid <= ctx->nc; }

int find_label(lb_ctx *ctx, const char *label, int kind, int *comp) {
  if (!label) return -1;
  for (size_t k = 0; k < ctx->open.size(); k++) {
    const Opening &o = ctx->open[k];
    if (o.kind != kind) continue;
    for (int c = 0; c < 2; c++)
      if (!o.label[c].empty() && o.label[c] == label) {
        *comp = c;
        return (int)k;
      }
  }
  return -1;
}

void node_of_open(const lb_ctx *ctx, const Opening &o, int a, int &x, int &y) {
  switch (o.wall) {
    case 0: x = 0; y = a; break;
    case 1: x = ctx->nx - 1; y = a; break;
    case 2: x = a; y = 0; break;
    default: x = a; y = ctx->ny - 1; break;
  }
}

int opening_at(const lb_ctx *ctx, int x, int y) {
  for (size_t k = 0; k < ctx->open.size(); k++) {
    const Opening &o = ctx->open[k];
    for (int a = o.a0; a <= o.a1; a++) {
      int ox, oy;
      node_of_open(ctx, o, a, ox, oy);
      if (ox == x && oy == y) return (int)k;
    }
  }
  return -1;
}

bool crosses(int wall, int ex, int ey) {
  return wall == 0 ? ex > 0 : wall == 1 ? ex < 0 : wall == 2 ? ey > 0 : ey < 0;
}

OpenDesc desc_of(const lb_ctx *ctx, const Opening &o) {
  OpenDesc d{};
  d.wall = o.wall;
  d.a0 = o.a0;
  d.a1 = o.a1;
  d.kind = o.kind;
  for (int c = 0; c < 2; c++) {
    d.style[c] = c < ctx->nc ? o.style[c] : OPEN_NONE;
    d.v[c] = (float)o.v[c];
    d.rho[c] = (float)o.rho[c];
    d.drho[c] = (float)(o.rho[c] - ctx->rho_ref[c]);
  }
  d.sstyle = o.sstyle;
  d.Cbar = (float)o.C;
  d.sv = (float)o.sv;
  return d;
}

// where the openings lie, for the membership tests in the kernels
void fill_spans(const lb_ctx *ctx, OpenSpan *sp) {
  for (size_t k = 0; k < ctx->open.size(); k++) sp[k] = {ctx->open[k].wall | ctx->open[k].a0 << 2, ctx->open[k].a1};
}

// the openings' fluid rules for the fluid kernels (the values as desc_of
// rounds them)
void fill_rules(const lb_ctx *ctx, OpenRule *r) {
  for (size_t k = 0; k < ctx->open.size(); k++) {
    const OpenDesc d = desc_of(ctx, ctx->open[k]);
    r[k].bits = d.style[0] | d.style[1] << 3 | d.kind << 6;
    for (int c = 0; c < 2; c++) r[k].val[c] = d.style[c] == OPEN_DIRICHLET ? d.drho[c] : d.v[c];
  }
}

int paint_check(lb_ctx *ctx) {
  if (!ctx->have_lattice) return ctx->fail(LB_E_ORDER, "lattice must come first");
  if (ctx->committed)
    return ctx->fail(LB_E_ORDER, "geometry and initial state are fixed after the first iteration");
  return LB_OK;
}

// the state buffers a caller may supply (lb_bind), their sizes
const char *const BUFFER_NAMES[6] = {"f0", "f1", "g0", "g1", "fields", "u"};

int buffer_index(const char *what) {
  if (!what) return -1;
  for (int k = 0; k < 6; k++)
    if (!strcmp(what, BUFFER_NAMES[k])) return k;
  return -1;
}

// ghost rows on each side of a slab: the pull reaches one row; interforce
// (the neighbours' densities after this step's streaming) and the slip
// styles (mirror sources two rows away) reach two; with surface reaction
// the two ghost rows next to the own rows are updated too (redundantly:
// the precipitation gathered by the boundary rows' solid nodes and the
// growth decisions of the solid nodes one row out come from them), which
// reach a third
int slab_halo(const lb_ctx *ctx) { return ctx->react ? 3 : (ctx->sc || ctx->bstyle != 0) ? 2 : 1; }

// ghost rows on each side that a slab updates redundantly
int slab_extra(const lb_ctx *ctx) { return ctx->rank >= 0 && ctx->react ? 2 : 0; }

// rows [y0, y0 + n) of slab `rank` out of py (sizes differ by one at most)
void slab_rows(const lb_ctx *ctx, int rank, int &y0, int &n) {
  y0 = (int)((long long)rank * ctx->ny / ctx->py);
  n = (int)((long long)(rank + 1) * ctx->ny / ctx->py) - y0;
}

// rows the context holds on the device: the lattice's, or a slab's own
// rows and its ghost rows
int held_rows(const lb_ctx *ctx) {
  if (ctx->rank < 0) return ctx->ny;
  int y0, n;
  slab_rows(ctx, ctx->rank, y0, n);
  return n + 2 * slab_halo(ctx);
}

// rows of the lattice updated here (its own rows for a slab)
int own_rows(const lb_ctx *ctx) { return ctx->committed ? ctx->g.yhi - ctx->g.ylo : ctx->ny; }

// geometry for the conversion kernels that fill every held row (ghost rows
// included)
Geometry all_rows(const Geometry &g) {
  Geometry a = g;
  a.ylo = 0;
  a.yhi = g.ny;
  return a;
}

// the held rows of a host array [planes][ny][nx] of the whole lattice, as
// [planes][held rows][nx] (held row y is lattice row y + yoff, wrapped)
const double *held_part(const lb_ctx *ctx, const double *src, int planes, std::vector<double> &buf) {
  if (!src || ctx->rank < 0) return src;
  const Geometry &g = ctx->g;
  const size_t nx = (size_t)ctx->nx, nn = nx * ctx->ny, nl = nx * g.ny;
  buf.resize((size_t)planes * nl);
  for (int q = 0; q < planes; q++)
    for (int y = 0; y < g.ny; y++) {
      const int gy = ((y + g.yoff) % ctx->ny + ctx->ny) % ctx->ny;
      memcpy(&buf[q * nl + y * nx], src + q * nn + (size_t)gy * nx, nx * sizeof(double));
    }
  return buf.data();
}

size_t buffer_bytes(const lb_ctx *ctx, int k) {
  const size_t plane = (size_t)held_rows(ctx) * (size_t)((ctx->nx + 31) / 32 * 32);
  switch (k) {
    case 0:
    case 1: return (size_t)ctx->nc * 9 * plane * storage_bytes(ctx->storage);
    case 2:
    case 3: return (size_t)ctx->qs * plane * sizeof(float);
    case 4: return (size_t)ctx->nc * NFIELD * plane * sizeof(float);
    case 5: return ctx->qs ? 2 * plane * sizeof(float) : 0;
    default: return 0;
  }
}

// LB_DEBUG_GUARDS: bytes of NaN pattern before and after each allocation
constexpr size_t GUARD_BYTES = 256 << 10;

template <class T>
int dalloc(lb_ctx *ctx, T **p, size_t n) {
  const size_t bytes = n > 0 ? n * sizeof(T) : 1;
  const bool guard = (ctx->debug & LB_DEBUG_GUARDS) != 0;
  void *raw = nullptr;
  cudaError_t e = cudaMalloc(&raw, bytes + (guard ? 2 * GUARD_BYTES : 0));
  if (e != cudaSuccess) return ctx->fail(LB_E_NOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  *p = (T *)((uint8_t *)raw + (guard ? GUARD_BYTES : 0));
  if (guard) {
    e = cudaMemsetAsync(raw, 0xff, bytes + 2 * GUARD_BYTES, ctx->stream);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "cudaMemsetAsync");
    ctx->guarded.push_back({raw, (void *)*p, bytes});
  }
  e = cudaMemsetAsync(*p, 0, n * sizeof(T), ctx->stream);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "cudaMemsetAsync");
  return LB_OK;
}

// a state buffer: the caller's (lb_bind) when bound, else allocated here;
// either way zeroed
template <class T>
int dalloc_state(lb_ctx *ctx, T **p, size_t n, int k) {
  if (!ctx->bound[k]) return dalloc(ctx, p, n);
  if (ctx->bound_bytes[k] < n * sizeof(T))
    return ctx->fail(LB_E_ARG, "bound buffer %s holds %zu bytes, the setup needs %zu", BUFFER_NAMES[k],
                     ctx->bound_bytes[k], n * sizeof(T));
  *p = (T *)ctx->bound[k];
  const cudaError_t e = cudaMemsetAsync(*p, 0, n * sizeof(T), ctx->stream);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "cudaMemsetAsync");
  return LB_OK;
}


int validate(lb_ctx *ctx) {
  const int nx = ctx->nx, ny = ctx->ny;
  if (ctx->sc && !ctx->open.empty() && ctx->rank >= 0)
    return ctx->fail(LB_E_UNSUPPORTED, "interforce with inlet/outlet openings is not built for slabs");
  for (const Opening &o : ctx->open) {
    for (int c = 0; c < ctx->nc; c++) {
      // without a momentum style the fluid stays periodic across the
      // opening's wall (boundary_style command); only a solute rule may
      // then make it an opening
      if (o.style[c] == OPEN_NONE && !(ctx->qs && o.sstyle != SOL_NONE))
        return ctx->fail(LB_E_ARG, "opening '%s' has no momentum style for fluid %d",
                         o.label[0].c_str(), c + 1);
      if ((o.style[c] == OPEN_UNIFORM || o.style[c] == OPEN_POISEUILLE) && !(std::fabs(o.v[c]) < 1.0))
        return ctx->fail(LB_E_ARG, "opening velocity must satisfy |v| < 1");
      if (o.style[c] == OPEN_DIRICHLET && !(o.rho[c] > 0.0))
        return ctx->fail(LB_E_ARG, "dirichlet density must be positive");
      if (o.style[c] == OPEN_GRADIENT) {
        int dx = o.wall == 0 ? 1 : o.wall == 1 ? -1 : 0, dy = o.wall == 2 ? 1 : o.wall == 3 ? -1 : 0;
        for (int a = o.a0; a <= o.a1; a++) {
          int x, y;
          node_of_open(ctx, o, a, x, y);
          if (ctx->solid[(size_t)y * nx + x]) continue;
          for (int k = 1; k <= 2; k++) {
            int xx = ((x + k * dx) % nx + nx) % nx, yy = ((y + k * dy) % ny + ny) % ny;
            if (ctx->solid[(size_t)yy * nx + xx])
              return ctx->fail(LB_E_ARG, "gradient opening node (%d,%d) needs two fluid nodes inside", x, y);
          }
        }
      }
    }
    if (ctx->qs && o.sstyle == SOL_NONE)
      return ctx->fail(LB_E_ARG, "opening '%s' has no solute style", o.label[0].c_str());
    if (ctx->qs && o.sstyle == SOL_FLUX) {
      const double D = (ctx->taus - 0.5) / (ctx->qs == 4 ? 2.0 : 3.0);
      if (o.kind == 1 && !(std::fabs(o.sv - D) > 1e-12))
        return ctx->fail(LB_E_ARG, "outlet flux style needs v != D = %g", D);
      if (o.kind == 0 && !(std::fabs(o.sv + D) > 1e-12))
        return ctx->fail(LB_E_ARG, "inlet flux style needs v != -D = %g", -D);
    }
  }
  if (ctx->react && ctx->t == 0) {
    // App. C rule 1: two opposite unknown modes cannot occur in the initial
    // geometry (growth can make them later; a lattice that continues a run,
    // lb_set_step t > 0, may hold them, each link then taking its own rule)
    const int q = ctx->qs;
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        if (ctx->solid[(size_t)y * nx + x]) continue;
        int k = opening_at(ctx, x, y);
        for (int i = (q == 4 ? 0 : 1); i < q; i++) {
          int ex = q == 4 ? EX4D[i] : EXD[i], ey = q == 4 ? EY4D[i] : EYD[i];
          if (k >= 0 && (crosses(ctx->open[k].wall, ex, ey) || crosses(ctx->open[k].wall, -ex, -ey)))
            continue;
          int x1 = ((x - ex) % nx + nx) % nx, y1 = ((y - ey) % ny + ny) % ny;
          int x2 = ((x + ex) % nx + nx) % nx, y2 = ((y + ey) % ny + ny) % ny;
          if (ctx->solid[(size_t)y1 * nx + x1] && ctx->solid[(size_t)y2 * nx + x2])
            return ctx->fail(LB_E_ARG,
                             "fluid node (%d,%d) has solid on two opposite sides: the surface "
                             "reaction needs a gap of at least two fluid nodes", x, y);
        }
      }
  }
  return LB_OK;
}

// allocate the device state and upload geometry and the painted state
}  // namespace

int commit(lb_ctx *ctx) {
  if (ctx->committed) return LB_OK;
  if (!ctx->have_lattice) return ctx->fail(LB_E_ORDER, "lattice must come first");
  TRY(validate(ctx));
  if (ctx->rank >= 0) {
    // a slab: which parts of the method it holds
    if (ctx->inter) return ctx->fail(LB_E_UNSUPPORTED, "intersolute on a slab is not built: run the lattice whole");
    ctx->halo = slab_halo(ctx);
    slab_rows(ctx, ctx->rank, ctx->sy0, ctx->sny);
    if (ctx->sny < std::max(3, 2 * ctx->halo))
      return ctx->fail(LB_E_ARG, "slab %d has %d rows; it needs at least %d", ctx->rank, ctx->sny,
                       std::max(3, 2 * ctx->halo));
  }
  TRY(set_device(ctx));
  Geometry &g = ctx->g;
  g.nx = ctx->nx;
  g.ny = held_rows(ctx);
  g.pitch = (ctx->nx + 31) / 32 * 32;
  g.mw = g.pitch / 32;
  g.plane = (size_t)g.ny * g.pitch;
  g.gny = ctx->ny;
  g.ylo = ctx->rank >= 0 ? ctx->halo : 0;
  g.yhi = g.ylo + (ctx->rank >= 0 ? ctx->sny : ctx->ny);
  g.yoff = ctx->rank >= 0 ? ctx->sy0 - ctx->halo : 0;
  g.clo = g.ylo - slab_extra(ctx);
  g.chi = g.yhi + slab_extra(ctx);
  const size_t sb = storage_bytes(ctx->storage);
  const size_t fbytes = (size_t)ctx->nc * 9 * g.plane * sb;
  for (int k = 0; k < 2; k++) TRY(dalloc_state(ctx, (uint8_t **)&ctx->fbuf[k], fbytes, k));
  TRY(dalloc(ctx, &ctx->mask, (size_t)g.ny * g.mw));
  TRY(dalloc(ctx, &ctx->nbc, g.plane));
  TRY(dalloc_state(ctx, &ctx->fields, (size_t)ctx->nc * NFIELD * g.plane, 4));
  if (ctx->qs) {
    TRY(dalloc_state(ctx, &ctx->u, 2 * g.plane, 5));
    for (int k = 0; k < 2; k++) TRY(dalloc_state(ctx, &ctx->gbuf[k], (size_t)ctx->qs * g.plane, 2 + k));
    if (ctx->inter) TRY(dalloc(ctx, &ctx->Cpre, g.plane));
    TRY(dalloc(ctx, &ctx->Cfield, g.plane));
    TRY(dalloc(ctx, &ctx->db, g.plane));
    TRY(dalloc(ctx, &ctx->flip, g.plane));
    TRY(dalloc(ctx, &ctx->flist, g.plane));
    TRY(dalloc(ctx, &ctx->fcount, 2));  // [0] running count, [1] last step's
    if (ctx->react && ctx->rank < 0) {
      TRY(dalloc(ctx, &ctx->slist, g.plane));
      TRY(dalloc(ctx, &ctx->scount, 1));
      TRY(dalloc(ctx, &ctx->gdone, 1));
    }
  }
  TRY(dalloc(ctx, &ctx->b, g.plane));
  TRY(dalloc(ctx, &ctx->removed, (size_t)(ctx->nc + 1) * g.plane));
  TRY(dalloc(ctx, &ctx->nflips, 1));
  TRY(dalloc(ctx, &ctx->errw, 1));
  TRY(dalloc(ctx, &ctx->d_open, MAX_OPEN));
  TRY(dalloc(ctx, &ctx->d_grad, MAX_OPEN));
  CK(cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device));
  ctx->tblocks = thermo_blocks(g, ctx->sms);
  TRY(dalloc(ctx, &ctx->partials, (size_t)ctx->tblocks * NTHERMO));
  TRY(dalloc(ctx, &ctx->tout, NTHERMO + 2));
  TRY(dalloc(ctx, &ctx->tdone, 1));

  // bit-packed mask of the held rows (held row y is lattice row y + yoff)
  auto lattice_row = [&](int y) { return ((y + g.yoff) % ctx->ny + ctx->ny) % ctx->ny; };
  std::vector<uint32_t> m((size_t)g.ny * g.mw, 0u);
  for (int y = 0; y < g.ny; y++)
    for (int x = 0; x < g.nx; x++)
      if (ctx->solid[(size_t)lattice_row(y) * g.nx + x]) m[(size_t)y * g.mw + (x >> 5)] |= 1u << (x & 31);
  CK(cudaMemcpyAsync(ctx->mask, m.data(), m.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
  LAUNCH(launch_nbcode(ctx->mask, ctx->nbc, g, ctx->stream));
  ctx->mask_host = m;
  ctx->mask_host_valid = true;
  if (ctx->slist) {
    // blocks for the growth gather over the surface list: one entry per
    // thread for the initial surface (the kernel strides over any more)
    size_t nsurf = 0;
    for (int y = 0; y < g.ny; y++)
      for (int x = 0; x < g.nx; x++) {
        if (!ctx->solid[(size_t)y * g.nx + x]) continue;
        bool wet = false;
        for (int dy = -1; dy <= 1 && !wet; dy++)
          for (int dx = -1; dx <= 1 && !wet; dx++)
            wet = !ctx->solid[(size_t)((y + dy + g.ny) % g.ny) * g.nx + (x + dx + g.nx) % g.nx];
        nsurf += wet;
      }
    ctx->sblocks = (int)std::min<size_t>((nsurf + 255) / 256 + 1, (size_t)4 * ctx->sms);
  }

  // hybrid boundary style: per-node reflection coefficients (0 on fluid
  // nodes, so nodes that grow solid later are noslip)
  if (ctx->bstyle == 3) {
    TRY(dalloc(ctx, &ctx->Rmap, (size_t)ctx->nc * g.plane));
    std::vector<float> rh((size_t)ctx->nc * g.plane, 0.0f);
    for (int c = 0; c < ctx->nc; c++)
      for (int y = 0; y < g.ny; y++)
        for (int x = 0; x < g.nx; x++) {
          const size_t n = (size_t)lattice_row(y) * g.nx + x;
          if (ctx->solid[n]) rh[(size_t)c * g.plane + (size_t)y * g.pitch + x] = ctx->Rh[c][n];
        }
    CK(cudaMemcpyAsync(ctx->Rmap, rh.data(), rh.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }

  // initial deposit b0 on every solid node (surface_reaction command)
  if (ctx->react) {
    std::vector<double> bh(g.plane, 0.0);
    for (int y = 0; y < g.ny; y++)
      for (int x = 0; x < g.nx; x++)
        if (ctx->solid[(size_t)lattice_row(y) * g.nx + x]) bh[(size_t)y * g.pitch + x] = ctx->b0;
    CK(cudaMemcpyAsync(ctx->b, bh.data(), bh.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
  }
  ctx->committed = true;

  // painted initial state (position0/momentum0/concentration0); opening
  // nodes start at the equilibrium of their opening's density and velocity
  const size_t nn = (size_t)g.nx * g.ny;
  for (int c = 0; c < ctx->nc; c++) {
    if (!ctx->painted_f[c]) continue;
    std::vector<double> f = ctx->paint_f[c];
    const std::vector<uint8_t> &base = ctx->paint_base[c];
    for (const Opening &o : ctx->open) {
      for (int a = o.a0; a <= o.a1; a++) {
        int x, y;
        node_of_open(ctx, o, a, x, y);
        // an opening node that still holds the populations read by
        // read_data keeps them (position0 does not reinitialise openings)
        if (!base.empty() && base[(size_t)y * g.nx + x]) continue;
        double v = 0.0;
        if (o.style[c] == OPEN_UNIFORM) v = o.v[c];
        if (o.style[c] == OPEN_POISEUILLE) {
          double L = o.a1 - o.a0 + 1, d = 0.5 * (2 * a - o.a1 - o.a0);
          v = 4 * o.v[c] / (L * L) * (0.25 * L * L - d * d);
        }
        double sgn = o.kind == 0 ? 1.0 : -1.0;
        double ux = 0, uy = 0;
        if (o.wall == 0) ux = sgn * v;
        if (o.wall == 1) ux = -sgn * v;
        if (o.wall == 2) uy = sgn * v;
        if (o.wall == 3) uy = -sgn * v;
        for (int i = 0; i < 9; i++)
          f[(size_t)i * nn + (size_t)y * g.nx + x] = feq_host(i, o.rho[c], ux, uy, ctx->alpha[c]);
      }
    }
    for (size_t n = 0; n < nn; n++) {
      if (ctx->solid[n]) continue;
      double r = 0;
      for (int i = 0; i < 9; i++) r += f[(size_t)i * nn + n];
      if (!(r > 0))
        return ctx->fail(LB_E_ARG, "fluid node (%zu,%zu) of fluid %d has no positive density: "
                         "initialise it with position0/momentum0 or lb_set_equilibrium",
                         n % g.nx, n / g.nx, c + 1);
    }
    int rc = lb_set_populations(ctx, c + 1, f.data());
    if (rc != LB_OK) return rc;
  }
  if (ctx->qs && ctx->painted_C) {
    int rc = lb_set_solute_equilibrium(ctx, ctx->paint_C.data(), nullptr, nullptr);
    if (rc != LB_OK) return rc;
  }
  // state read from input-data files (read_data command)
  for (int c = 0; c < ctx->nc; c++) {
    lb_ctx::ReadState &r = ctx->rf[c];
    if (r.kind == 1) TRY(lb_set_populations(ctx, c + 1, r.a.data()));
    if (r.kind == 2) TRY(lb_set_equilibrium(ctx, c + 1, r.a.data(), r.ux.data(), r.uy.data()));
    r = lb_ctx::ReadState();
  }
  if (ctx->qs && ctx->rg.kind == 1) TRY(lb_set_solute_populations(ctx, ctx->rg.a.data()));
  if (ctx->qs && ctx->rg.kind == 2)
    TRY(lb_set_solute_equilibrium(ctx, ctx->rg.a.data(), ctx->rg.ux.data(), ctx->rg.uy.data()));
  ctx->rg = lb_ctx::ReadState();
  if (!ctx->rb.empty()) {
    if (ctx->react) TRY(lb_set_precipitate(ctx, ctx->rb.data()));
    std::vector<double>().swap(ctx->rb);
  }
  return LB_OK;
}

namespace {

FluidArgs fluid_args(lb_ctx *ctx, bool fields) {
  FluidArgs a{};
  a.g = ctx->g;
  a.fin = ctx->fbuf[ctx->cur];
  a.fout = ctx->fbuf[1 - ctx->cur];
  a.mask = ctx->mask;
  a.nbc = ctx->nbc;
  a.scale = ctx->scale;
  a.inv_scale = ctx->inv_scale;
  for (int c = 0; c < 2; c++) {
    a.rho_ref[c] = (float)ctx->rho_ref[c];
    a.tau[c] = (float)ctx->tau[c];
    a.omega[c] = (float)(1.0 / ctx->tau[c]);
    a.wa[c] = (float)wshare(1, ctx->alpha[c]);
    a.wd[c] = (float)wshare(5, ctx->alpha[c]);
    a.fx[c] = (float)ctx->fave[c][0];
    a.fy[c] = (float)ctx->fave[c][1];
    a.ax[c] = (float)ctx->acc[c][0];
    a.ay[c] = (float)ctx->acc[c][1];
    a.ads[c] = ctx->ads[c] ? 1 : 0;
    a.Gads[c] = (float)ctx->Gads[c];
    a.ads_psi0[c] = (float)ctx->ads_psi0[c];
    a.ads_rho0[c] = (float)ctx->ads_rho0[c];
  }
  a.G = (float)ctx->G;
  a.psi0 = (float)ctx->psi0;
  a.sc_rho0 = (float)ctx->sc_rho0;
  a.nopen = (int)ctx->open.size();
  fill_spans(ctx, a.span);
  fill_rules(ctx, a.rule);
  a.fields = fields ? ctx->fields : nullptr;
  a.uout = ctx->qs ? ctx->u : nullptr;
  uint64_t z = (uint64_t)ctx->t * 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 31)) * 0xbf58476d1ce4e5b9ULL;
  a.step_seed = (uint32_t)(z >> 32);
  if (ctx->sr) a.sr_seed = (uint32_t)z | 1u;
  a.pm = ctx->pm ? 1 : 0;
  a.slip = ctx->bstyle != 0 ? 1 : 0;
  a.slipR[0] = a.slipR[1] = (float)(ctx->bstyle == 1 ? 1.0 : ctx->bstyle == 2 ? ctx->slipR : 0.0);
  a.Rmap = ctx->bstyle == 3 ? ctx->Rmap : nullptr;
  for (const Opening &o : ctx->open) {
    if (o.wall <= 1) a.edge_x = 1;
    else a.edge_y = 1;
  }
  return a;
}

// the thermo record of step `step` (the sums, the flip count, the TMA
// error word) into ctx->thermo; its LB_E_TIMEOUT or LB_E_NAN
int decode_thermo(lb_ctx *ctx, const double *rec, int64_t step) {
  const double *h = rec;
  unsigned long long nfl = 0;
  memcpy(&nfl, &rec[NTHERMO], sizeof nfl);
  const int errw = (int)rec[NTHERMO + 1];
  if (errw) {
    // reported once: the word is cleared for the iterations that follow
    CK(cudaMemsetAsync(ctx->errw, 0, sizeof(int), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return ctx->fail(LB_E_TIMEOUT, "a TMA pipeline wait timed out before step %lld", (long long)step);
  }
  lb_thermo_t &T = ctx->thermo;
  memset(&T, 0, sizeof T);
  T.step = step;
  T.nsolid = (int64_t)llround(h[13]);
  T.nfluid = (int64_t)llround(h[14]);
  for (int c = 0; c < ctx->nc; c++) {
    T.mass[c] = ctx->rho_ref[c] * (double)T.nfluid + h[0 + c];
    T.mass_eq[c] = ctx->rho_ref[c] * (double)T.nfluid + h[2 + c];
    T.mom_comp[c][0] = h[4 + 2 * c];
    T.mom_comp[c][1] = h[5 + 2 * c];
    T.mom[0] += h[4 + 2 * c];
    T.mom[1] += h[5 + 2 * c];
  }
  T.solute = h[8];
  T.bsum = h[9];
  T.removed[0] = h[10];
  T.removed[1] = h[11];
  T.removed_solute = h[12];
  T.flips = (int64_t)nfl;
  ctx->thermo_valid = true;
  for (int q = 0; q < NTHERMO; q++)
    if (!std::isfinite(h[q])) return ctx->fail(LB_E_NAN, "thermo sum %d is not finite at step %lld", q, (long long)step);
  return LB_OK;
}

// deferred records: read the oldest one waiting (after its copy has landed)
int read_deferred(lb_ctx *ctx) {
  const int slot = ctx->tq[0];
  ctx->tq[0] = ctx->tq[1];
  ctx->tq_n--;
  CK(cudaEventSynchronize(ctx->trec_ev[slot]));
  return decode_thermo(ctx, ctx->trec_host + (size_t)slot * (NTHERMO + 2), ctx->trec_step[slot]);
}

// ... every one waiting, in step order
}  // namespace

int read_all_deferred(lb_ctx *ctx) {
  while (ctx->tq_n) TRY(read_deferred(ctx));
  return LB_OK;
}

namespace {

int run_thermo(lb_ctx *ctx) {
  NvtxRange range("thermo");
  ThermoArgs ta{};
  ta.g = ctx->g;
  ta.mask = ctx->mask;
  ta.fields = ctx->fields;
  ta.nc = ctx->nc;
  ta.Cfield = ctx->qs ? ctx->Cfield : nullptr;
  ta.b = ctx->react ? ctx->b : nullptr;
  ta.removed = ctx->react ? ctx->removed : nullptr;
  ta.partials = ctx->partials;
  ta.out = ctx->tout;
  ta.done = ctx->tdone;
  ta.nflips = ctx->nflips;
  ta.errw = ctx->errw;
  // deferred records of earlier thermo evaluations are read first (at
  // least one thermo interval old, their copies have long landed); their
  // errors are this call's
  if (ctx->tdefer) TRY(read_all_deferred(ctx));
  LAUNCH(launch_thermo(ta, ctx->tblocks, ctx->stream));
  if (ctx->tdefer) {
    const int slot = ctx->tq_next;
    ctx->tq_next ^= 1;
    CK(cudaMemcpyAsync(ctx->trec_host + (size_t)slot * (NTHERMO + 2), ctx->tout, (NTHERMO + 2) * sizeof(double),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaEventRecord(ctx->trec_ev[slot], ctx->stream));
    ctx->trec_step[slot] = ctx->t;
    ctx->tq[ctx->tq_n++] = slot;
    return LB_OK;
  }
  double rec[NTHERMO + 2];
  CK(cudaMemcpyAsync(rec, ctx->tout, sizeof rec, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return decode_thermo(ctx, rec, ctx->t);
}

// LB_DEBUG_POISON: NaN bit patterns (all ones: NaN in FP32, FP16 and
// BF16) in every buffer the coming iteration writes
int poison_outputs(lb_ctx *ctx, int nxt, bool fields) {
  const Geometry &g = ctx->g;
  const size_t plane = g.plane;
  cudaStream_t s = ctx->stream;
  CK(cudaMemsetAsync(ctx->fbuf[nxt], 0xff, (size_t)ctx->nc * 9 * plane * storage_bytes(ctx->storage), s));
  if (ctx->qs) {
    CK(cudaMemsetAsync(ctx->gbuf[nxt], 0xff, (size_t)ctx->qs * plane * 4, s));
    CK(cudaMemsetAsync(ctx->u, 0xff, 2 * plane * 4, s));
    if (ctx->react) CK(cudaMemsetAsync(ctx->db, 0xff, plane * 4, s));
    if (ctx->inter) CK(cudaMemsetAsync(ctx->Cpre, 0xff, plane * 4, s));
    if (fields) CK(cudaMemsetAsync(ctx->Cfield, 0xff, plane * 4, s));
  }
  if (fields) CK(cudaMemsetAsync(ctx->fields, 0xff, (size_t)ctx->nc * NFIELD * plane * 4, s));
  return LB_OK;
}

// the opening descriptors in device memory (all openings; the gradient
// ones), uploaded in stream order when they differ from the last upload
int sync_openings(lb_ctx *ctx) {
  OpenDesc all[MAX_OPEN], grad[MAX_OPEN];
  int na = 0, ng = 0;
  for (const Opening &o : ctx->open) {
    all[na] = desc_of(ctx, o);
    bool gr = false;
    for (int c = 0; c < ctx->nc; c++) gr |= o.style[c] == OPEN_GRADIENT;
    if (gr) grad[ng++] = all[na];
    na++;
  }
  auto upload = [&](const OpenDesc *d, int n, std::vector<OpenDesc> &held, OpenDesc *dst) -> int {
    if ((size_t)n == held.size() && (n == 0 || !memcmp(d, held.data(), n * sizeof(OpenDesc)))) return LB_OK;
    held.assign(d, d + n);
    if (n) CK(cudaMemcpyAsync(dst, held.data(), n * sizeof(OpenDesc), cudaMemcpyHostToDevice, ctx->stream));
    return LB_OK;
  };
  TRY(upload(all, na, ctx->h_open, ctx->d_open));
  return upload(grad, ng, ctx->h_grad, ctx->d_grad);
}

int one_step(lb_ctx *ctx, bool fields) {
  NvtxRange range("step");
  TRY(sync_openings(ctx));
  cudaStream_t s = ctx->stream;
  ctx->t += 1;
  if (ctx->react) ctx->mask_host_valid = false;  // growth may change the device mask
  const int nxt = 1 - ctx->cur;
  FluidArgs fa = fluid_args(ctx, fields);
  // two components and Shan-Chen runs keep |f - w rho_ref| large: their
  // collision is the mass-exact one
  const bool mass_exact = ctx->nc == 2 || ctx->sc;
  const bool tma_ok = ctx->nc == 1 && !ctx->sc && ctx->bstyle == 0 && !ctx->pm && ctx->rank < 0 &&
                      tma_supported(ctx->storage, ctx->g);
  if (ctx->kernel == 2 && !tma_ok)
    return ctx->fail(LB_E_UNSUPPORTED, "the TMA kernel runs single-component noslip lattices without "
                     "interforce whose width is a multiple of 4 (FP32) or 8 (16-bit) nodes");
  SoluteArgs sa{};
  if (ctx->qs) {
    sa.g = ctx->g;
    sa.gin = ctx->gbuf[ctx->cur];
    sa.gout = ctx->gbuf[nxt];
    sa.mask = ctx->mask;
    sa.nbc = ctx->nbc;
    sa.u = ctx->u;
    sa.omega = (float)(1.0 / ctx->taus);
    sa.react = ctx->react ? 1 : 0;
    sa.kr = (float)ctx->kr;
    sa.Cs = (float)ctx->Cs;
    sa.rden[0] = (float)(1.0 / (ctx->kr + 2.0 * (ctx->qs == 4 ? 0.25 : 1.0 / 9.0)));
    sa.rden[1] = (float)(1.0 / (ctx->kr + 2.0 / 36.0));
    sa.db = ctx->db;
    sa.Cfield = fields ? ctx->Cfield : nullptr;
    sa.nopen = (int)ctx->open.size();
    fill_spans(ctx, sa.span);
    sa.op = ctx->d_open;
    sa.D = (float)((ctx->taus - 0.5) / (ctx->qs == 4 ? 2.0 : 3.0));
    sa.inter = ctx->inter ? 1 : 0;
    sa.isG = (float)ctx->isG;
    sa.ispsi0 = (float)ctx->ispsi0;
    sa.isC0 = (float)ctx->isC0;
    sa.taus = (float)ctx->taus;
    sa.Cpre = ctx->Cpre;
    sa.Cpre_out = ctx->Cpre;
  }
  // fluid and solute in one kernel where the solute needs nothing of other
  // nodes' fluid update (no intersolute) and the fluid kernel is the plain
  // streaming one
  const bool fuse_ok = ctx->qs && !ctx->inter && ctx->nc == 1 && !ctx->sc && !ctx->pm;
  if (ctx->kernel == 3 && !fuse_ok)
    return ctx->fail(LB_E_UNSUPPORTED, "the fused kernel runs single-component lattices with a solute, "
                     "without interforce, intersolute or exact momentum pairs");
  const bool fused = fuse_ok && (ctx->kernel == 0 || ctx->kernel == 3);
  if (ctx->debug & LB_DEBUG_POISON) TRY(poison_outputs(ctx, nxt, fields));
  if (fused) {
    // the solvent velocity stays in registers; the plane is written only
    // when the caller bound it
    fa.uout = ctx->bound[5] ? ctx->u : nullptr;
    LAUNCH(launch_fluid_solute(ctx->storage, ctx->qs, fa, sa, s));
  } else if (tma_ok && ctx->kernel == 2) {
    LAUNCH(launch_fluid_tma(ctx->storage, fa, ctx->errw, ctx->wait_limit, s, ctx->sms));
  } else {
    LAUNCH(launch_fluid(ctx->storage, ctx->nc, ctx->sc, mass_exact, fa, s));
  }
  // gradient openings
  if (!ctx->h_grad.empty()) {
    GradArgs ga{};
    ga.g = ctx->g;
    ga.f = ctx->fbuf[nxt];
    ga.fields = fields ? ctx->fields : nullptr;
    ga.mask = ctx->mask;
    ga.nc = ctx->nc;
    ga.nopen = (int)ctx->h_grad.size();
    ga.op = ctx->d_grad;
    for (const OpenDesc &o : ctx->h_grad) ga.maxlen = std::max(ga.maxlen, o.a1 - o.a0 + 1);
    ga.inv_scale = ctx->inv_scale;
    ga.scale = ctx->scale;
    LAUNCH(launch_gradient(ctx->storage, ga, s));
  }
  if (ctx->qs) {
    if (!fused) LAUNCH(launch_solute(ctx->qs, sa, s));
    if (ctx->react) {
      GrowthArgs ga2{};
      ga2.g = ctx->g;
      ga2.mask = ctx->mask;
      ga2.db = ctx->db;
      ga2.b = ctx->b;
      ga2.nbc = ctx->nbc;
      ga2.flip = ctx->flip;
      ga2.flist = ctx->flist;
      ga2.fcount = ctx->fcount;
      ga2.bmax = ctx->bmax;
      ga2.b0 = ctx->b0;
      ga2.seed = ctx->seed;
      ga2.t = ctx->t;
      // solid nodes that gather and decide: the own rows, and for a slab one
      // ghost row each side (their decisions can turn own-row nodes solid)
      ga2.rlo = ctx->rank >= 0 ? ctx->g.ylo - 1 : 0;
      ga2.rhi = ctx->rank >= 0 ? ctx->g.yhi + 1 : ctx->g.ny;
      ga2.q = ctx->qs;
      ga2.nopen = sa.nopen;
      for (int k = 0; k < sa.nopen; k++) ga2.span[k] = sa.span[k];
      ga2.f = ctx->fbuf[nxt];
      ga2.f_prev = ctx->fbuf[ctx->cur];
      ga2.nc = ctx->nc;
      ga2.rho_ref[0] = (float)ctx->rho_ref[0];
      ga2.rho_ref[1] = (float)ctx->rho_ref[1];
      ga2.inv_scale = ctx->inv_scale;
      ga2.gpop = ctx->gbuf[nxt];
      ga2.removed = ctx->removed;
      ga2.nflips = ctx->nflips;
      if (ctx->slist) {
        ga2.slist = ctx->slist;
        ga2.scount = ctx->scount;
        ga2.sblocks = ctx->sblocks;
        ga2.done = ctx->gdone;
        if (!ctx->slist_valid) {
          CK(cudaMemsetAsync(ctx->scount, 0, sizeof(unsigned int), s));
          LAUNCH(launch_surface_list(ga2, s));
          ctx->slist_valid = true;
        }
      }
      LAUNCH(launch_growth(ctx->storage, ga2, s));
    }
  }
  ctx->cur = nxt;
  return LB_OK;
}

// FP64 staging buffer on the device for host <-> device conversions
struct Stage {
  double *p = nullptr;
  ~Stage() {
    if (p) cudaFree(p);
  }
};

int stage_in(lb_ctx *ctx, Stage &st, const double *host, size_t n) {
  cudaError_t e = cudaMalloc((void **)&st.p, n * sizeof(double));
  if (e != cudaSuccess) return ctx->fail(LB_E_NOMEM, "staging cudaMalloc: %s", cudaGetErrorString(e));
  if (host) CK(cudaMemcpyAsync(st.p, host, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  return LB_OK;
}

int stage_alloc(lb_ctx *ctx, Stage &st, size_t n) { return stage_in(ctx, st, nullptr, n); }

}  // namespace

// ======================================================================
// C ABI
// ======================================================================

extern "C" {

int lb_create(int device, void *cuda_stream, lb_ctx **out) {
  if (!out) return LB_E_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return LB_E_CUDA;
  lb_ctx *ctx = new (std::nothrow) lb_ctx();
  if (!ctx) return LB_E_NOMEM;
  ctx->device = device;
  ctx->stream = (cudaStream_t)cuda_stream;
  *out = ctx;
  return LB_OK;
}

int lb_destroy(lb_ctx *ctx) {
  NEED_CTX();
  cudaSetDevice(ctx->device);
  if (ctx->committed) cudaStreamSynchronize(ctx->stream);
  void *ptrs[] = {ctx->fbuf[0], ctx->fbuf[1], ctx->mask,     ctx->fields,   ctx->u,
                  ctx->gbuf[0], ctx->gbuf[1], ctx->Cfield,   ctx->db,       ctx->b,
                  ctx->removed, ctx->flip,    ctx->nflips,   ctx->partials, ctx->tout, ctx->tdone,
                  ctx->errw,    ctx->Cpre,    ctx->Rmap,    ctx->flist,    ctx->fcount,
                  ctx->vstage,  ctx->nbc,     ctx->d_open,   ctx->d_grad,   ctx->slist,
                  ctx->scount,  ctx->gdone};
  for (void *p : ptrs) {
    bool own = p != nullptr;
    for (int k = 0; k < 6; k++) own = own && p != ctx->bound[k];
    if (!own) continue;
    for (const lb_ctx::Guarded &gd : ctx->guarded)
      if (gd.user == p) p = gd.raw;
    cudaFree(p);
  }
  for (int k = 0; k < 2; k++)
    if (ctx->trec_ev[k]) cudaEventDestroy(ctx->trec_ev[k]);
  if (ctx->trec_host) cudaFreeHost(ctx->trec_host);
  delete ctx;
  return LB_OK;
}

const char *lb_last_error(const lb_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int lb_launch_count(const lb_ctx *ctx, uint64_t *out) {
  if (!ctx || !out) return LB_E_ARG;
  *out = ctx->launches;
  return LB_OK;
}

int lb_lattice(lb_ctx *ctx, const char *style, int nx, int ny, double tau) {
  NEED_CTX();
  if (ctx->committed) return ctx->fail(LB_E_ORDER, "lattice is fixed after the first iteration");
  if (!style || strcmp(style, "d2q9")) return ctx->fail(LB_E_UNSUPPORTED, "lattice style must be d2q9");
  if (nx < 1 || ny < 1) return ctx->fail(LB_E_ARG, "bad lattice size %d x %d", nx, ny);
  // the kernels index one component's nine planes of (nx rounded up to 32)
  // x ny slots with 32-bit offsets
  if (9LL * (((long long)nx + 31) / 32 * 32) * ny > (long long)INT32_MAX)
    return ctx->fail(LB_E_UNSUPPORTED, "lattice %d x %d exceeds the 32-bit plane indexing (9 x pitch x ny < 2^31)",
                     nx, ny);
  if (!(tau > 0.5)) return ctx->fail(LB_E_ARG, "tau must exceed 1/2");
  ctx->have_lattice = true;
  ctx->nx = nx;
  ctx->ny = ny;
  ctx->tau[0] = ctx->tau[1] = tau;
  const size_t nn = (size_t)nx * ny;
  ctx->solid.assign(nn, 0);
  ctx->region.assign(nn, 0);
  // the painted initial state (position0/momentum0/concentration0) is
  // allocated by the first command that paints
  for (int c = 0; c < 2; c++) {
    ctx->paint_f[c].clear();
    ctx->paint_base[c].clear();
    ctx->painted_f[c] = false;
  }
  ctx->paint_C.clear();
  ctx->paint_base_C.clear();
  return LB_OK;
}

int lb_processors(lb_ctx *ctx, int px, int py) {
  NEED_CTX();
  if (!ctx->have_lattice) return ctx->fail(LB_E_ORDER, "processors must follow lattice");
  if (ctx->momentum_cmd)
    return ctx->fail(LB_E_ORDER, "processors must precede inlet_momentum/outlet_momentum and momentum0");
  if (px < 1 || py < 1) return ctx->fail(LB_E_ARG, "processor grid must be positive");
  if (ctx->committed) return ctx->fail(LB_E_ORDER, "processors must precede the first iteration");
  if (ctx->rank >= 0 && (px != 1 || ctx->rank >= py))
    return ctx->fail(LB_E_ARG, "rank %d does not fit the processor grid %d x %d", ctx->rank, px, py);
  ctx->px = px;
  ctx->py = py;
  return LB_OK;
}

int lb_processor_rank(lb_ctx *ctx, int rank) {
  NEED_CTX();
  if (!ctx->have_lattice) return ctx->fail(LB_E_ORDER, "the rank must follow lattice and processors");
  if (ctx->committed) return ctx->fail(LB_E_ORDER, "the rank must precede the first iteration");
  if (ctx->px != 1) return ctx->fail(LB_E_UNSUPPORTED, "slabs split the lattice along y only: processors(1, py)");
  if (rank < -1 || rank >= ctx->py) return ctx->fail(LB_E_ARG, "rank %d is outside 0..%d", rank, ctx->py - 1);
  ctx->rank = rank;
  return LB_OK;
}

int lb_fluids(lb_ctx *ctx, double tau1, double tau2, double alpha1, double alpha2) {
  NEED_CTX();
  TRY(paint_check(ctx));
  if (!(tau1 > 0.5) || !(tau2 > 0.5)) return ctx->fail(LB_E_ARG, "tau must exceed 1/2");
  // c_s^2 = (3/5)(1 - alpha) must stay positive, and A_0 = (9/4) alpha
  // must not be negative
  if (!(alpha1 >= 0.0 && alpha1 < 1.0) || !(alpha2 >= 0.0 && alpha2 < 1.0))
    return ctx->fail(LB_E_ARG, "alpha must lie in [0, 1)");
  ctx->nc = 2;
  ctx->alpha[0] = alpha1;
  ctx->alpha[1] = alpha2;
  ctx->tau[0] = tau1;
  ctx->tau[1] = tau2;
  return LB_OK;
}

int lb_solute(lb_ctx *ctx, double taus, int q) {
  NEED_CTX();
  TRY(paint_check(ctx));
  if (q != 4 && q != 9) return ctx->fail(LB_E_ARG, "solute lattice must be D2Q4 or D2Q9");
  if (!(taus > 0.5)) return ctx->fail(LB_E_ARG, "taus must exceed 1/2");
  ctx->qs = q;
  ctx->taus = taus;
  return LB_OK;
}

int lb_set_storage(lb_ctx *ctx, int storage, const double *rho_ref, double h_max) {
  NEED_CTX();
  TRY(paint_check(ctx));
  const bool sr = (storage & LB_STOCHASTIC_ROUNDING) != 0;
  const bool pm = (storage & LB_PRECISE_MOMENTUM) != 0;
  storage &= ~(LB_STOCHASTIC_ROUNDING | LB_PRECISE_MOMENTUM);
  if (storage != LB_FP32 && storage != LB_FP16 && storage != LB_BF16)
    return ctx->fail(LB_E_ARG, "unknown storage %d", storage);
  if (sr && storage == LB_FP32) return ctx->fail(LB_E_ARG, "stochastic rounding applies to 16-bit storage");
  ctx->storage = storage;
  ctx->sr = sr;
  ctx->pm = pm;
  double rmax = 0;
  for (int c = 0; c < 2; c++) {
    // a value FP32 holds exactly, so that the kernels and the FP64 host
    // conversions shift by the same reference density
    ctx->rho_ref[c] = (double)(float)(rho_ref ? rho_ref[c < ctx->nc ? c : 0] : 1.0);
    if (!(ctx->rho_ref[c] > 0)) return ctx->fail(LB_E_ARG, "rho_ref must be positive");
    rmax = std::max(rmax, ctx->rho_ref[c]);
  }
  ctx->scale = ctx->inv_scale = 1.f;
  if (storage == LB_FP16) {
    double hm = h_max > 0 ? h_max : 0.25 * rmax;
    int s = (int)std::floor(std::log2(16384.0 / hm));
    s = std::max(-14, std::min(s, 60));
    ctx->scale = (float)std::ldexp(1.0, s);
    ctx->inv_scale = (float)std::ldexp(1.0, -s);
  }
  return LB_OK;
}

int lb_boundary_style(lb_ctx *ctx, const char *style, double R) {
  NEED_CTX();
  TRY(paint_check(ctx));
  if (!style) return ctx->fail(LB_E_ARG, "no style");
  if (!strcmp(style, "noslip")) ctx->bstyle = 0;
  else if (!strcmp(style, "slip")) ctx->bstyle = 1;
  else if (!strcmp(style, "mixed")) {
    if (!(R >= 0.0 && R <= 1.0)) return ctx->fail(LB_E_ARG, "reflection coefficient must lie in [0, 1]");
    ctx->bstyle = 2;
    ctx->slipR = R;
  } else if (!strcmp(style, "hybrid")) {
    ctx->bstyle = 3;
    for (int c = 0; c < 2; c++) ctx->Rh[c].assign(ctx->solid.size(), 0.0f);
  } else {
    return ctx->fail(LB_E_ARG, "unknown boundary style '%s'", style);
  }
  ctx->have_style = true;
  return LB_OK;
}

// style name and argument of the styled obstacle calls -> R
static int style_R(lb_ctx *ctx, const char *style, double arg, float *R) {
  if (!style || !strcmp(style, "noslip")) *R = 0.0f;
  else if (!strcmp(style, "slip")) *R = 1.0f;
  else if (!strcmp(style, "mixed")) {
    if (!(arg >= 0.0 && arg <= 1.0)) return ctx->fail(LB_E_ARG, "reflection coefficient must lie in [0, 1]");
    *R = (float)arg;
  } else {
    return ctx->fail(LB_E_ARG, "obstacle style must be noslip, slip or mixed");
  }
  return LB_OK;
}

// record R1 (fluid 1) and R2 (fluid 2) on the nodes a region marks
static void paint_R(lb_ctx *ctx, const std::vector<uint8_t> &m, float R1, float R2) {
  if (ctx->bstyle != 3) return;
  for (size_t n = 0; n < m.size(); n++)
    if (m[n]) {
      ctx->Rh[0][n] = R1;
      ctx->Rh[1][n] = R2;
    }
}

static int obstacle_check(lb_ctx *ctx) {
  TRY(paint_check(ctx));
  if (!ctx->have_style) return ctx->fail(LB_E_ORDER, "obstacle must follow boundary_style");
  return LB_OK;
}

int lb_obstacle_rect_styled(lb_ctx *ctx, int x0, int x1, int y0, int y1, const char *style1, double arg1,
                            const char *style2, double arg2) {
  NEED_CTX();
  TRY(obstacle_check(ctx));
  if (x0 > x1 || y0 > y1) return ctx->fail(LB_E_ARG, "rectangle bounds must be ordered");
  float R1, R2;
  TRY(style_R(ctx, style1, arg1, &R1));
  TRY(style_R(ctx, style2 ? style2 : style1, style2 ? arg2 : arg1, &R2));
  std::vector<uint8_t> m(ctx->solid.size(), 0);
  for (int y = std::max(y0, 0); y <= std::min(y1, ctx->ny - 1); y++)
    for (int x = std::max(x0, 0); x <= std::min(x1, ctx->nx - 1); x++) m[(size_t)y * ctx->nx + x] = 1;
  for (size_t n = 0; n < m.size(); n++)
    if (m[n]) ctx->solid[n] = 1;
  paint_R(ctx, m, R1, R2);
  return LB_OK;
}

int lb_obstacle_rect(lb_ctx *ctx, int x0, int x1, int y0, int y1) {
  return lb_obstacle_rect_styled(ctx, x0, x1, y0, y1, nullptr, 0.0, nullptr, 0.0);
}

static void circle_paint(lb_ctx *ctx, std::vector<uint8_t> &m, int xc, int yc, int r, uint8_t v) {
  const int nx = ctx->nx, ny = ctx->ny;
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      int dx = x - xc, dy = y - yc;
      dx = ((dx + nx / 2) % nx + nx) % nx - nx / 2;
      dy = ((dy + ny / 2) % ny + ny) % ny - ny / 2;
      if ((long long)dx * dx + (long long)dy * dy <= (long long)r * r) m[(size_t)y * nx + x] = v;
    }
}

int lb_obstacle_circle_styled(lb_ctx *ctx, int xc, int yc, int r, const char *style1, double arg1,
                              const char *style2, double arg2) {
  NEED_CTX();
  TRY(obstacle_check(ctx));
  if (r < 0) return ctx->fail(LB_E_ARG, "negative radius");
  float R1, R2;
  TRY(style_R(ctx, style1, arg1, &R1));
  TRY(style_R(ctx, style2 ? style2 : style1, style2 ? arg2 : arg1, &R2));
  std::vector<uint8_t> m(ctx->solid.size(), 0);
  circle_paint(ctx, m, xc, yc, r, 1);
  for (size_t n = 0; n < m.size(); n++)
    if (m[n]) ctx->solid[n] = 1;
  paint_R(ctx, m, R1, R2);
  return LB_OK;
}

int lb_obstacle_circle(lb_ctx *ctx, int xc, int yc, int r) {
  return lb_obstacle_circle_styled(ctx, xc, yc, r, nullptr, 0.0, nullptr, 0.0);
}

int lb_obstacle_mask_hybrid(lb_ctx *ctx, const uint8_t *mask, const double *R) {
  NEED_CTX();
  TRY(obstacle_check(ctx));
  if (!mask) return ctx->fail(LB_E_ARG, "null mask");
  const size_t nn = ctx->solid.size();
  if (R) {
    if (ctx->bstyle != 3) return ctx->fail(LB_E_ORDER, "per-node reflection coefficients need boundary_style hybrid");
    for (size_t n = 0; n < (size_t)ctx->nc * nn; n++)
      if (mask[n % nn] && !(R[n] >= 0.0 && R[n] <= 1.0))
        return ctx->fail(LB_E_ARG, "reflection coefficient must lie in [0, 1]");
  }
  for (size_t n = 0; n < nn; n++)
    if (mask[n]) {
      ctx->solid[n] = 1;
      if (ctx->bstyle == 3) {
        ctx->Rh[0][n] = R ? (float)R[n] : 0.0f;
        ctx->Rh[1][n] = R ? (float)R[(ctx->nc > 1 ? nn : 0) + n] : 0.0f;
      }
    }
  return LB_OK;
}

int lb_obstacle_mask(lb_ctx *ctx, const uint8_t *mask) { return lb_obstacle_mask_hybrid(ctx, mask, nullptr); }

static int add_opening(lb_ctx *ctx, int kind, const char *wall, int a0, int a1, const char *l1,
                       const char *l2) {
  TRY(paint_check(ctx));
  int w = wall_of(wall);
  if (w < 0) return ctx->fail(LB_E_ARG, "wall must be xlo, xhi, ylo or yhi");
  int len = w <= 1 ? ctx->ny : ctx->nx;
  if (a0 > a1 || a0 < 0 || a1 >= len) return ctx->fail(LB_E_ARG, "opening extent %d..%d outside the wall", a0, a1);
  if (!l1 || !*l1) return ctx->fail(LB_E_ARG, "opening needs a label");
  if (ctx->nc == 2 && (!l2 || !*l2)) return ctx->fail(LB_E_ARG, "two fluids need two labels");
  if ((int)ctx->open.size() >= MAX_OPEN) return ctx->fail(LB_E_UNSUPPORTED, "at most %d openings", MAX_OPEN);
  Opening o;
  o.wall = w;
  o.a0 = a0;
  o.a1 = a1;
  o.kind = kind;
  o.label[0] = l1;
  if (l2) o.label[1] = l2;
  for (int a = a0; a <= a1; a++) {
    int x, y;
    node_of_open(ctx, o, a, x, y);
    if (opening_at(ctx, x, y) >= 0) return ctx->fail(LB_E_ARG, "node (%d,%d) already belongs to an opening", x, y);
  }
  for (const Opening &p : ctx->open)
    for (int c = 0; c < 2; c++)
      for (int d = 0; d < 2; d++)
        if (!p.label[c].empty() && !o.label[d].empty() && p.label[c] == o.label[d])
          return ctx->fail(LB_E_ARG, "label '%s' already used", o.label[d].c_str());
  ctx->open.push_back(o);
  return LB_OK;
}

int lb_inlet(lb_ctx *ctx, const char *wall, int a0, int a1, const char *l1, const char *l2) {
  NEED_CTX();
  return add_opening(ctx, 0, wall, a0, a1, l1, l2);
}

int lb_outlet(lb_ctx *ctx, const char *wall, int a0, int a1, const char *l1, const char *l2) {
  NEED_CTX();
  return add_opening(ctx, 1, wall, a0, a1, l1, l2);
}

static int set_momentum(lb_ctx *ctx, int kind, const char *label, const char *style, double v, double rho) {
  if (!ctx->have_lattice) return ctx->fail(LB_E_ORDER, "lattice must come first");
  int comp = 0;
  int k = find_label(ctx, label, kind, &comp);
  if (k < 0) return ctx->fail(LB_E_ARG, "no %s labelled '%s'", kind ? "outlet" : "inlet", label ? label : "");
  int st;
  if (!style) return ctx->fail(LB_E_ARG, "no style");
  if (!strcmp(style, "poiseuille")) st = OPEN_POISEUILLE;
  else if (!strcmp(style, "uniform")) st = OPEN_UNIFORM;
  else if (!strcmp(style, "dirichlet")) st = OPEN_DIRICHLET;
  else if (!strcmp(style, "gradient")) st = OPEN_GRADIENT;
  else return ctx->fail(LB_E_ARG, "unknown momentum style '%s'", style);
  if (!(rho > 0)) return ctx->fail(LB_E_ARG, "opening density must be positive");
  if ((st == OPEN_UNIFORM || st == OPEN_POISEUILLE) && !(std::fabs(v) < 1.0))
    return ctx->fail(LB_E_ARG, "opening velocity must satisfy |v| < 1");
  if (ctx->committed && st != ctx->open[k].style[comp] &&
      (st == OPEN_GRADIENT || ctx->open[k].style[comp] == OPEN_GRADIENT))
    return ctx->fail(LB_E_ORDER, "gradient style cannot be switched after the first iteration");
  ctx->open[k].style[comp] = st;
  ctx->open[k].v[comp] = v;
  ctx->open[k].rho[comp] = rho;
  ctx->momentum_cmd = true;
  return LB_OK;
}

int lb_inlet_momentum(lb_ctx *ctx, const char *label, const char *style, double v, double rho) {
  NEED_CTX();
  return set_momentum(ctx, 0, label, style, v, rho);
}

int lb_outlet_momentum(lb_ctx *ctx, const char *label, const char *style, double v, double rho) {
  NEED_CTX();
  return set_momentum(ctx, 1, label, style, v, rho);
}

static int set_solute_open(lb_ctx *ctx, int kind, const char *label, const char *style, double C,
                           double v) {
  if (!ctx->qs) return ctx->fail(LB_E_ORDER, "inlet_solute/outlet_solute need the solute command");
  int comp = 0;
  int k = find_label(ctx, label, kind, &comp);
  if (k < 0) return ctx->fail(LB_E_ARG, "no %s labelled '%s'", kind ? "outlet" : "inlet", label ? label : "");
  if (!style) return ctx->fail(LB_E_ARG, "no style");
  if (!strcmp(style, "dirichlet")) ctx->open[k].sstyle = SOL_DIRICHLET;
  else if (!strcmp(style, "adiabatic")) ctx->open[k].sstyle = SOL_ADIABATIC;
  else if (!strcmp(style, "flux")) ctx->open[k].sstyle = SOL_FLUX;
  else return ctx->fail(LB_E_ARG, "unknown solute style '%s'", style);
  ctx->open[k].C = C;
  ctx->open[k].sv = v;
  return LB_OK;
}

int lb_inlet_solute(lb_ctx *ctx, const char *label, const char *style, double C, double v) {
  NEED_CTX();
  return set_solute_open(ctx, 0, label, style, C, v);
}

int lb_outlet_solute(lb_ctx *ctx, const char *label, const char *style, double C, double v) {
  NEED_CTX();
  return set_solute_open(ctx, 1, label, style, C, v);
}

int lb_intersolute(lb_ctx *ctx, double G, double psi0, double C0) {
  NEED_CTX();
  TRY(paint_check(ctx));
  if (!ctx->qs) return ctx->fail(LB_E_ORDER, "intersolute needs the solute command");
  if (!std::isfinite(G) || !std::isfinite(psi0) || !std::isfinite(C0))
    return ctx->fail(LB_E_ARG, "intersolute parameters must be finite");
  ctx->inter = true;
  ctx->isG = G;
  ctx->ispsi0 = psi0;
  ctx->isC0 = C0;
  return LB_OK;
}

int lb_surface_reaction(lb_ctx *ctx, double kr, double Cs, const char *style, double b0, double bmax,
                        uint64_t seed) {
  NEED_CTX();
  TRY(paint_check(ctx));
  if (!ctx->qs) return ctx->fail(LB_E_ORDER, "surface_reaction needs the solute command");
  if (!style || strcmp(style, "growth")) return ctx->fail(LB_E_ARG, "surface_reaction style must be growth");
  if (!(kr >= 0)) return ctx->fail(LB_E_ARG, "kr must be >= 0");
  ctx->react = true;
  ctx->kr = kr;
  ctx->Cs = Cs;
  ctx->b0 = b0;
  ctx->bmax = bmax;
  ctx->seed = seed;
  return LB_OK;
}

int lb_position0_rect(lb_ctx *ctx, int x0, int x1, int y0, int y1) {
  NEED_CTX();
  TRY(paint_check(ctx));
  if (x0 > x1 || y0 > y1) return ctx->fail(LB_E_ARG, "rectangle bounds must be ordered");
  std::fill(ctx->region.begin(), ctx->region.end(), 0);
  for (int y = std::max(y0, 0); y <= std::min(y1, ctx->ny - 1); y++)
    for (int x = std::max(x0, 0); x <= std::min(x1, ctx->nx - 1); x++) ctx->region[(size_t)y * ctx->nx + x] = 1;
  ctx->have_region = true;
  return LB_OK;
}

int lb_position0_circle(lb_ctx *ctx, int xc, int yc, int r) {
  NEED_CTX();
  TRY(paint_check(ctx));
  if (r < 0) return ctx->fail(LB_E_ARG, "negative radius");
  std::fill(ctx->region.begin(), ctx->region.end(), 0);
  circle_paint(ctx, ctx->region, xc, yc, r, 1);
  ctx->have_region = true;
  return LB_OK;
}

int lb_momentum0(lb_ctx *ctx, int mode, double value, int fluid) {
  NEED_CTX();
  TRY(paint_check(ctx));
  if (!ctx->have_region) return ctx->fail(LB_E_ORDER, "momentum0 must follow position0");
  if (mode < 0 || mode > 8 || !fluid_ok(ctx, fluid)) return ctx->fail(LB_E_ARG, "bad mode or fluid");
  const size_t nn = ctx->region.size();
  const int c = fluid - 1;
  std::vector<double> &f = ctx->paint_f[c];
  std::vector<uint8_t> &base = ctx->paint_base[c];
  if (f.empty()) {
    // after read_data the painting starts from the state read: only the
    // nodes position0 marks are reinitialised (the first momentum0 that
    // reaches a node clears the populations read there)
    lb_ctx::ReadState &r = ctx->rf[c];
    f.assign(9 * nn, 0.0);
    base.clear();
    if (r.kind) base.assign(nn, 1);
    if (r.kind == 1) f = r.a;
    if (r.kind == 2)
      for (size_t n = 0; n < nn; n++)
        for (int i = 0; i < 9; i++) f[(size_t)i * nn + n] = feq_host(i, r.a[n], r.ux[n], r.uy[n], ctx->alpha[c]);
    r = lb_ctx::ReadState();
  }
  for (size_t n = 0; n < nn; n++)
    if (ctx->region[n]) {
      if (!base.empty() && base[n]) {
        for (int i = 0; i < 9; i++) f[(size_t)i * nn + n] = 0.0;
        base[n] = 0;
      }
      f[(size_t)mode * nn + n] += value;
    }
  ctx->painted_f[c] = true;
  ctx->momentum_cmd = true;
  return LB_OK;
}

int lb_concentration0(lb_ctx *ctx, double value) {
  NEED_CTX();
  TRY(paint_check(ctx));
  if (!ctx->have_region) return ctx->fail(LB_E_ORDER, "concentration0 must follow position0");
  if (!ctx->qs) return ctx->fail(LB_E_ORDER, "concentration0 needs the solute command");
  const size_t nn = ctx->region.size();
  std::vector<uint8_t> &base = ctx->paint_base_C;
  if (ctx->paint_C.empty()) {
    // after read_data the painting starts from the concentrations read (the
    // solute then starts at their equilibrium at rest)
    lb_ctx::ReadState &r = ctx->rg;
    ctx->paint_C.assign(nn, 0.0);
    base.clear();
    if (r.kind) base.assign(nn, 1);
    if (r.kind == 1)
      for (size_t n = 0; n < nn; n++)
        for (int i = 0; i < ctx->qs; i++) ctx->paint_C[n] += r.a[(size_t)i * nn + n];
    if (r.kind == 2) ctx->paint_C = r.a;
    r = lb_ctx::ReadState();
  }
  for (size_t n = 0; n < nn; n++)
    if (ctx->region[n]) {
      if (!base.empty() && base[n]) {
        ctx->paint_C[n] = 0.0;
        base[n] = 0;
      }
      ctx->paint_C[n] += value;
    }
  ctx->painted_C = true;
  return LB_OK;
}

int lb_set_equilibrium(lb_ctx *ctx, int fluid, const double *rho, const double *ux, const double *uy) {
  NEED_CTX();
  ctx->fields_step = -1;  // the live state no longer matches the field planes
  if (!ctx->have_lattice) return ctx->fail(LB_E_ORDER, "lattice must come first");
  if (!fluid_ok(ctx, fluid) || !rho) return ctx->fail(LB_E_ARG, "bad fluid or null rho");
  const size_t nn = (size_t)ctx->nx * ctx->ny;
  for (size_t n = 0; n < nn; n++)
    if (!ctx->solid[n] && !(rho[n] > 0))
      return ctx->fail(LB_E_ARG, "density must be positive on fluid node (%zu,%zu)", n % ctx->nx, n / ctx->nx);
  ctx->painted_f[fluid - 1] = false;
  TRY(commit(ctx));
  // a slab takes its rows and ghost rows of the lattice's arrays
  std::vector<double> br, bu, bv;
  const size_t nl = (size_t)ctx->nx * ctx->g.ny;
  Stage r, u, v;
  TRY(stage_in(ctx, r, held_part(ctx, rho, 1, br), nl));
  if (ux) TRY(stage_in(ctx, u, held_part(ctx, ux, 1, bu), nl));
  if (uy) TRY(stage_in(ctx, v, held_part(ctx, uy, 1, bv), nl));
  const size_t sb = storage_bytes(ctx->storage);
  void *dst = (uint8_t *)ctx->fbuf[ctx->cur] + (size_t)(fluid - 1) * 9 * ctx->g.plane * sb;
  LAUNCH(launch_equilibrium(ctx->storage, r.p, u.p, v.p, dst, ctx->mask, all_rows(ctx->g),
                            (float)ctx->rho_ref[fluid - 1], ctx->scale, ctx->alpha[fluid - 1], ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->state_set[fluid - 1] = true;
  return LB_OK;
}

int lb_set_solute_equilibrium(lb_ctx *ctx, const double *C, const double *ux, const double *uy) {
  NEED_CTX();
  ctx->fields_step = -1;  // the live state no longer matches the field planes
  if (!ctx->qs) return ctx->fail(LB_E_ORDER, "no solute");
  if (!C) return ctx->fail(LB_E_ARG, "null C");
  ctx->painted_C = false;
  TRY(commit(ctx));
  std::vector<double> bc, bu, bv;
  const size_t nl = (size_t)ctx->nx * ctx->g.ny;
  Stage c, u, v;
  TRY(stage_in(ctx, c, held_part(ctx, C, 1, bc), nl));
  if (ux) TRY(stage_in(ctx, u, held_part(ctx, ux, 1, bu), nl));
  if (uy) TRY(stage_in(ctx, v, held_part(ctx, uy, 1, bv), nl));
  LAUNCH(launch_solute_equilibrium(ctx->qs, c.p, u.p, v.p, ctx->gbuf[ctx->cur], ctx->mask, all_rows(ctx->g),
                                   ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->solute_set = true;
  return LB_OK;
}

int lb_set_populations(lb_ctx *ctx, int fluid, const double *f) {
  NEED_CTX();
  ctx->fields_step = -1;  // the live state no longer matches the field planes
  if (!ctx->have_lattice) return ctx->fail(LB_E_ORDER, "lattice must come first");
  if (!fluid_ok(ctx, fluid) || !f) return ctx->fail(LB_E_ARG, "bad fluid or null array");
  if (!ctx->committed) ctx->painted_f[fluid - 1] = false;
  TRY(commit(ctx));
  std::vector<double> bf;
  const size_t nl = (size_t)ctx->nx * ctx->g.ny;
  Stage st;
  TRY(stage_in(ctx, st, held_part(ctx, f, 9, bf), 9 * nl));
  const size_t sb = storage_bytes(ctx->storage);
  void *dst = (uint8_t *)ctx->fbuf[ctx->cur] + (size_t)(fluid - 1) * 9 * ctx->g.plane * sb;
  LAUNCH(launch_import_pops(ctx->storage, st.p, dst, ctx->mask, all_rows(ctx->g), 9, (float)ctx->rho_ref[fluid - 1],
                            ctx->scale, true, ctx->alpha[fluid - 1], ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->state_set[fluid - 1] = true;
  return LB_OK;
}

int lb_set_solute_populations(lb_ctx *ctx, const double *g) {
  NEED_CTX();
  ctx->fields_step = -1;  // the live state no longer matches the field planes
  if (!ctx->qs) return ctx->fail(LB_E_ORDER, "no solute");
  if (!g) return ctx->fail(LB_E_ARG, "null array");
  ctx->painted_C = false;
  TRY(commit(ctx));
  std::vector<double> bg;
  const size_t nl = (size_t)ctx->nx * ctx->g.ny;
  Stage st;
  TRY(stage_in(ctx, st, held_part(ctx, g, ctx->qs, bg), (size_t)ctx->qs * nl));
  LAUNCH(launch_import_pops(ST_FP32, st.p, ctx->gbuf[ctx->cur], ctx->mask, all_rows(ctx->g), ctx->qs, 0.f, 1.f, false,
                            4.0 / 9.0, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->solute_set = true;
  return LB_OK;
}

int lb_set_precipitate(lb_ctx *ctx, const double *b) {
  NEED_CTX();
  ctx->fields_step = -1;  // the live state no longer matches the field planes
  if (!b) return ctx->fail(LB_E_ARG, "null array");
  TRY(commit(ctx));
  std::vector<double> bb;
  Stage st;
  TRY(stage_in(ctx, st, held_part(ctx, b, 1, bb), (size_t)ctx->nx * ctx->g.ny));
  LAUNCH(launch_import_plane_f64(st.p, all_rows(ctx->g), ctx->b, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return LB_OK;
}

static int add_vec(lb_ctx *ctx, double (*dst)[2], int mode, double value, int fluid) {
  if (!ctx->have_lattice) return ctx->fail(LB_E_ORDER, "force commands must follow lattice or fluids");
  if (mode < 0 || mode > 8 || !fluid_ok(ctx, fluid)) return ctx->fail(LB_E_ARG, "bad mode or fluid");
  dst[fluid - 1][0] += value * EXD[mode];
  dst[fluid - 1][1] += value * EYD[mode];
  return LB_OK;
}

int lb_aveforce(lb_ctx *ctx, int mode, double value, int fluid) {
  NEED_CTX();
  return add_vec(ctx, ctx->fave, mode, value, fluid);
}

int lb_aveforce_xy(lb_ctx *ctx, double fx, double fy, int fluid) {
  NEED_CTX();
  if (!ctx->have_lattice) return ctx->fail(LB_E_ORDER, "force commands must follow lattice or fluids");
  if (!fluid_ok(ctx, fluid)) return ctx->fail(LB_E_ARG, "bad fluid");
  ctx->fave[fluid - 1][0] += fx;
  ctx->fave[fluid - 1][1] += fy;
  return LB_OK;
}

int lb_aveacceleration(lb_ctx *ctx, int mode, double value, int fluid) {
  NEED_CTX();
  return add_vec(ctx, ctx->acc, mode, value, fluid);
}

int lb_aveacceleration_xy(lb_ctx *ctx, double ax, double ay, int fluid) {
  NEED_CTX();
  if (!ctx->have_lattice) return ctx->fail(LB_E_ORDER, "force commands must follow lattice or fluids");
  if (!fluid_ok(ctx, fluid)) return ctx->fail(LB_E_ARG, "bad fluid");
  ctx->acc[fluid - 1][0] += ax;
  ctx->acc[fluid - 1][1] += ay;
  return LB_OK;
}

int lb_interforce(lb_ctx *ctx, double G, double psi0, double rho0) {
  NEED_CTX();
  if (!ctx->have_lattice) return ctx->fail(LB_E_ORDER, "interforce must follow lattice or fluids");
  if (ctx->nc == 1 && G != 0.0 && !(rho0 > 0 || rho0 < 0 || psi0 == 0))
    return ctx->fail(LB_E_ARG, "interforce needs rho0 for one component");
  ctx->sc = (G != 0.0);
  ctx->G = G;
  ctx->psi0 = psi0;
  ctx->sc_rho0 = rho0;
  if (ctx->committed && ctx->sc && !ctx->open.empty() && ctx->rank >= 0)
    return ctx->fail(LB_E_UNSUPPORTED, "interforce with inlet/outlet openings is not built for slabs");
  return LB_OK;
}

int lb_adhesiveforce(lb_ctx *ctx, double G, double psi0, double rho0, int fluid) {
  NEED_CTX();
  if (!ctx->have_lattice) return ctx->fail(LB_E_ORDER, "adhesiveforce must follow lattice or fluids");
  if (!fluid_ok(ctx, fluid)) return ctx->fail(LB_E_ARG, "bad fluid");
  ctx->ads[fluid - 1] = (G != 0.0);
  ctx->Gads[fluid - 1] = G;
  ctx->ads_psi0[fluid - 1] = psi0;
  ctx->ads_rho0[fluid - 1] = rho0;
  return LB_OK;
}

int lb_set_kernel(lb_ctx *ctx, const char *name) {
  NEED_CTX();
  if (!name) return ctx->fail(LB_E_ARG, "no kernel name");
  if (!strcmp(name, "auto")) ctx->kernel = 0;
  else if (!strcmp(name, "streaming")) ctx->kernel = 1;
  else if (!strcmp(name, "tma")) ctx->kernel = 2;
  else if (!strcmp(name, "fused")) ctx->kernel = 3;
  else return ctx->fail(LB_E_ARG, "kernel must be auto, streaming, tma or fused");
  return LB_OK;
}

int lb_set_wait_limit(lb_ctx *ctx, int64_t cycles) {
  NEED_CTX();
  ctx->wait_limit = cycles < 0 ? -1 : (long long)cycles;
  return LB_OK;
}

int lb_set_debug(lb_ctx *ctx, int flags) {
  NEED_CTX();
  if (flags & ~(LB_DEBUG_POISON | LB_DEBUG_GUARDS)) return ctx->fail(LB_E_ARG, "unknown debug flags 0x%x", flags);
  ctx->debug = flags;
  return LB_OK;
}

int lb_debug_check(lb_ctx *ctx, int64_t *bad) {
  NEED_CTX();
  if (!bad) return ctx->fail(LB_E_ARG, "null output");
  TRY(set_device(ctx));
  CK(cudaStreamSynchronize(ctx->stream));
  std::vector<uint8_t> h(GUARD_BYTES);
  int64_t n = 0;
  for (const lb_ctx::Guarded &gd : ctx->guarded) {
    for (int side = 0; side < 2; side++) {
      const uint8_t *src = side ? (const uint8_t *)gd.user + gd.bytes : (const uint8_t *)gd.raw;
      CK(cudaMemcpy(h.data(), src, GUARD_BYTES, cudaMemcpyDeviceToHost));
      for (uint8_t v : h) n += v != 0xff;
    }
  }
  *bad = n;
  return LB_OK;
}

int lb_output(lb_ctx *ctx, int Nf) {
  NEED_CTX();
  if (Nf < 0) return ctx->fail(LB_E_ARG, "Nf must be >= 0");
  ctx->nout = Nf;
  return LB_OK;
}

int lb_thermo(lb_ctx *ctx, int Nf) {
  NEED_CTX();
  if (Nf < 0) return ctx->fail(LB_E_ARG, "Nf must be >= 0");
  ctx->nf = Nf;
  return LB_OK;
}

int lb_thermo_deferred(lb_ctx *ctx, int on) {
  NEED_CTX();
  if (on != 0 && on != 1) return ctx->fail(LB_E_ARG, "on must be 0 or 1");
  if (on && !ctx->trec_host) {
    TRY(set_device(ctx));
    CK(cudaHostAlloc((void **)&ctx->trec_host, 2 * (NTHERMO + 2) * sizeof(double), cudaHostAllocDefault));
    for (int k = 0; k < 2; k++) CK(cudaEventCreateWithFlags(&ctx->trec_ev[k], cudaEventDisableTiming));
  }
  if (!on && ctx->tq_n) {
    TRY(set_device(ctx));
    TRY(read_all_deferred(ctx));
  }
  ctx->tdefer = on != 0;
  return LB_OK;
}

int lb_iteration(lb_ctx *ctx, int Nt) {
  NEED_CTX();
  NvtxRange range("lb_iteration");
  if (Nt < 0) return ctx->fail(LB_E_ARG, "Nt must be >= 0");
  if (!ctx->have_lattice) return ctx->fail(LB_E_ORDER, "lattice must come first");
  for (int c = 0; c < ctx->nc; c++)
    if (!ctx->painted_f[c] && !ctx->state_set[c] && !ctx->rf[c].kind)
      return ctx->fail(LB_E_ORDER, "fluid %d has no initial state (position0/momentum0, read_data or "
                       "lb_set_equilibrium)", c + 1);
  if (ctx->qs && !ctx->painted_C && !ctx->solute_set && !ctx->rg.kind)
    return ctx->fail(LB_E_ORDER, "solute has no initial state (concentration0, read_data or "
                     "lb_set_solute_equilibrium)");
  TRY(commit(ctx));
  TRY(set_device(ctx));
  // a slab reads its ghost rows every iteration: with other slabs they are
  // filled between calls (lb_exchange or lb_halo_pack/unpack); a single slab
  // (processors 1 x 1) is its own neighbour and refills them itself
  if (ctx->rank >= 0 && ctx->py > 1 && Nt > 1)
    return ctx->fail(LB_E_ORDER, "a slab of a lattice split into %d advances one iteration per call, its halo "
                     "rows exchanged between calls", ctx->py);
  for (int k = 1; k <= Nt; k++) {
    const bool thermo = ctx->nf > 0 ? ((ctx->t + 1) % ctx->nf == 0) : (k == Nt);
    const bool out = ctx->nout > 0 && (ctx->t + 1) % ctx->nout == 0;
    TRY(one_step(ctx, thermo || out));
    if (ctx->rank >= 0 && ctx->py == 1) TRY(exchange_slabs(&ctx, 1));
    if (out && !thermo) {
      ctx->fields_valid = true;
      ctx->fields_step = ctx->t;
    }
    if (thermo) {
      ctx->fields_valid = true;
      ctx->fields_step = ctx->t;
      TRY(run_thermo(ctx));
    }
    ctx->iterated = true;
    // write_restart: the state after this iteration, "<file>.<t>"
    if (ctx->restart_nf > 0 && ctx->t % ctx->restart_nf == 0)
      TRY(write_data_files(ctx, ctx->restart_file + "." + std::to_string((long long)ctx->t)));
  }
  return LB_OK;
}

int lb_get_thermo(lb_ctx *ctx, lb_thermo_t *out) {
  NEED_CTX();
  if (!out) return ctx->fail(LB_E_ARG, "null output");
  if (ctx->tq_n) {
    TRY(set_device(ctx));
    TRY(read_all_deferred(ctx));
  }
  if (!ctx->thermo_valid) return ctx->fail(LB_E_ORDER, "no thermo record yet: call lb_iteration first");
  *out = ctx->thermo;
  return LB_OK;
}

int lb_get_fields(lb_ctx *ctx, int fluid, double *rho, double *px, double *py, double *rho_eq) {
  NEED_CTX();
  if (!ctx->fields_valid) return ctx->fail(LB_E_ORDER, "no fields yet: call lb_iteration first");
  if (!fluid_ok(ctx, fluid)) return ctx->fail(LB_E_ARG, "bad fluid");
  TRY(set_device(ctx));
  const size_t nn = (size_t)ctx->nx * own_rows(ctx);  // a slab: its own rows
  Stage st;
  TRY(stage_alloc(ctx, st, 4 * nn));
  LAUNCH(launch_export_fields(ctx->fields, fluid - 1, ctx->mask, ctx->g, (float)ctx->rho_ref[fluid - 1], st.p,
                              st.p + nn, st.p + 2 * nn, st.p + 3 * nn, ctx->stream));
  double *outs[4] = {rho, px, py, rho_eq};
  for (int k = 0; k < 4; k++)
    if (outs[k]) CK(cudaMemcpyAsync(outs[k], st.p + k * nn, nn * 8, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return LB_OK;
}

// a host buffer the device addresses directly (page-locked, mapped, with the
// same address on both sides), else nullptr
static float *device_view(float *h) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, h) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return (at.type == cudaMemoryTypeHost && at.devicePointer == (void *)h) ? h : nullptr;
}

int lb_get_velocity_f32(lb_ctx *ctx, float *rho, float *ux, float *uy) {
  NEED_CTX();
  if (!ctx->fields_valid) return ctx->fail(LB_E_ORDER, "no fields yet: call lb_iteration first");
  if (!rho || !ux || !uy) return ctx->fail(LB_E_ARG, "null output");
  TRY(set_device(ctx));
  const size_t nn = (size_t)ctx->nx * own_rows(ctx);  // a slab: its own rows
  float rr[2] = {(float)ctx->rho_ref[0], (float)ctx->rho_ref[1]};
  if (device_view(rho) && device_view(ux) && device_view(uy)) {
    // page-locked outputs: the export kernel writes them over the host link
    // itself, with no staging buffer and no separate copies
    int n = launch_export_velocity(ctx->fields, ctx->nc, ctx->mask, ctx->g, rr, rho, ux, uy, ctx->stream);
    cudaError_t e = n < 0 ? cudaGetLastError() : cudaSuccess;
    if (n > 0) ctx->launches += n;
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "velocity export");
    return LB_OK;
  }
  // a staging buffer kept for the context's life: an allocation per call
  // costs more than the copies
  if (!ctx->vstage) TRY(dalloc(ctx, &ctx->vstage, 3 * nn));
  float *st = ctx->vstage;
  int n = launch_export_velocity(ctx->fields, ctx->nc, ctx->mask, ctx->g, rr, st, st + nn, st + 2 * nn,
                                 ctx->stream);
  cudaError_t e = n < 0 ? cudaGetLastError() : cudaSuccess;
  if (n > 0) ctx->launches += n;
  if (e == cudaSuccess) e = cudaMemcpyAsync(rho, st, nn * 4, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ux, st + nn, nn * 4, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(uy, st + 2 * nn, nn * 4, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return ctx->cuda_fail(e, "velocity export");
  return LB_OK;
}

int lb_get_populations(lb_ctx *ctx, int fluid, double *f) {
  NEED_CTX();
  if (!ctx->committed) return ctx->fail(LB_E_ORDER, "no device state yet");
  if (!fluid_ok(ctx, fluid) || !f) return ctx->fail(LB_E_ARG, "bad fluid or null array");
  TRY(set_device(ctx));
  const size_t nn = (size_t)ctx->nx * own_rows(ctx);  // a slab: its own rows
  Stage st;
  TRY(stage_alloc(ctx, st, 9 * nn));
  const size_t sb = storage_bytes(ctx->storage);
  const void *src = (const uint8_t *)ctx->fbuf[ctx->cur] + (size_t)(fluid - 1) * 9 * ctx->g.plane * sb;
  LAUNCH(launch_export_pops(ctx->storage, src, st.p, ctx->mask, ctx->g, 9, (float)ctx->rho_ref[fluid - 1],
                            ctx->inv_scale, true, ctx->alpha[fluid - 1], ctx->stream));
  CK(cudaMemcpyAsync(f, st.p, 9 * nn * 8, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return LB_OK;
}

int lb_get_solute(lb_ctx *ctx, double *g, double *C, double *b) {
  NEED_CTX();
  if (!ctx->committed) return ctx->fail(LB_E_ORDER, "no device state yet");
  TRY(set_device(ctx));
  const size_t nn = (size_t)ctx->nx * own_rows(ctx);  // a slab: its own rows
  if (g) {
    if (!ctx->qs) return ctx->fail(LB_E_ORDER, "no solute");
    Stage st;
    TRY(stage_alloc(ctx, st, (size_t)ctx->qs * nn));
    LAUNCH(launch_export_pops(ST_FP32, ctx->gbuf[ctx->cur], st.p, ctx->mask, ctx->g, ctx->qs, 0.f, 1.f, false,
                              4.0 / 9.0, ctx->stream));
    CK(cudaMemcpyAsync(g, st.p, (size_t)ctx->qs * nn * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  if (C) {
    if (!ctx->qs) return ctx->fail(LB_E_ORDER, "no solute");
    if (!ctx->fields_valid) return ctx->fail(LB_E_ORDER, "no fields yet: call lb_iteration first");
    Stage st;
    TRY(stage_alloc(ctx, st, nn));
    LAUNCH(launch_export_plane_f32(ctx->Cfield, ctx->mask, ctx->g, st.p, ctx->stream));
    CK(cudaMemcpyAsync(C, st.p, nn * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  if (b) {
    Stage st;
    TRY(stage_alloc(ctx, st, nn));
    LAUNCH(launch_export_plane_f64(ctx->b, ctx->g, st.p, ctx->stream));
    CK(cudaMemcpyAsync(b, st.p, nn * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return LB_OK;
}

int lb_get_mask(lb_ctx *ctx, uint8_t *mask) {
  NEED_CTX();
  if (!mask) return ctx->fail(LB_E_ARG, "null output");
  if (!ctx->committed) {
    int y0 = 0, n = ctx->ny;
    if (ctx->rank >= 0) slab_rows(ctx, ctx->rank, y0, n);
    memcpy(mask, ctx->solid.data() + (size_t)y0 * ctx->nx, (size_t)n * ctx->nx);
    return LB_OK;
  }
  TRY(set_device(ctx));
  std::vector<uint32_t> m((size_t)ctx->g.ny * ctx->g.mw);
  CK(cudaMemcpyAsync(m.data(), ctx->mask, m.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  // the updated rows (a slab's own rows)
  for (int y = ctx->g.ylo; y < ctx->g.yhi; y++)
    for (int x = 0; x < ctx->nx; x++)
      mask[(size_t)(y - ctx->g.ylo) * ctx->nx + x] = (m[(size_t)y * ctx->g.mw + (x >> 5)] >> (x & 31)) & 1u;
  return LB_OK;
}

int lb_set_step(lb_ctx *ctx, int64_t t) {
  NEED_CTX();
  if (t < 0) return ctx->fail(LB_E_ARG, "t must be >= 0");
  ctx->t = t;
  return LB_OK;
}

int lb_buffer_size(lb_ctx *ctx, const char *what, size_t *bytes) {
  NEED_CTX();
  const int k = buffer_index(what);
  if (k < 0 || !bytes) return ctx->fail(LB_E_ARG, "unknown buffer name or null output");
  if (!ctx->have_lattice) return ctx->fail(LB_E_ORDER, "lattice must come first");
  *bytes = buffer_bytes(ctx, k);
  return LB_OK;
}

int lb_bind(lb_ctx *ctx, const char *what, void *dev, size_t bytes) {
  NEED_CTX();
  const int k = buffer_index(what);
  if (k < 0) return ctx->fail(LB_E_ARG, "unknown buffer name");
  if (!ctx->have_lattice) return ctx->fail(LB_E_ORDER, "lattice must come first");
  if (ctx->committed) return ctx->fail(LB_E_ORDER, "buffers are fixed after the first iteration");
  if (!dev) {
    ctx->bound[k] = nullptr;
    ctx->bound_bytes[k] = 0;
    return LB_OK;
  }
  if ((uintptr_t)dev % 256 != 0) return ctx->fail(LB_E_ARG, "bound buffer must be 256-byte aligned");
  if (bytes < buffer_bytes(ctx, k))
    return ctx->fail(LB_E_ARG, "buffer %s needs %zu bytes, got %zu", what, buffer_bytes(ctx, k), bytes);
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, dev) != cudaSuccess) {
    cudaGetLastError();
    return ctx->fail(LB_E_ARG, "not a device pointer");
  }
  if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != ctx->device)
    return ctx->fail(LB_E_ARG, "buffer %s is not device memory of device %d", what, ctx->device);
  for (int j = 0; j < 6; j++)
    if (j != k && ctx->bound[j] == dev) return ctx->fail(LB_E_ARG, "one buffer bound twice");
  ctx->bound[k] = dev;
  ctx->bound_bytes[k] = bytes;
  return LB_OK;
}

int lb_current_buffer(lb_ctx *ctx, int *index) {
  NEED_CTX();
  if (!index) return ctx->fail(LB_E_ARG, "null output");
  *index = ctx->cur;
  return LB_OK;
}

int lb_get_flips(lb_ctx *ctx, int64_t *idx, int cap, int *count) {
  NEED_CTX();
  if (!count || cap < 0 || (cap > 0 && !idx)) return ctx->fail(LB_E_ARG, "bad output");
  *count = 0;
  if (!ctx->committed || !ctx->react) return LB_OK;
  TRY(set_device(ctx));
  unsigned int n = 0;
  CK(cudaMemcpyAsync(&n, ctx->fcount + 1, sizeof n, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  std::vector<unsigned int> off(n);
  if (n) {
    CK(cudaMemcpyAsync(off.data(), ctx->flist, n * sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  std::vector<int64_t> node(n);
  for (unsigned int k = 0; k < n; k++) {
    const int64_t y = off[k] / ctx->g.pitch, x = off[k] - y * ctx->g.pitch;
    node[k] = (y - ctx->g.ylo) * ctx->nx + x;  // in the own rows (a slab's)
  }
  std::sort(node.begin(), node.end());
  for (int k = 0; k < (int)n && k < cap; k++) idx[k] = node[k];
  *count = (int)n;
  return LB_OK;
}


}  // extern "C"
