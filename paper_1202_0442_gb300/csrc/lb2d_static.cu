// lb2d_static.cu -- lb_thermo_static, the thermo record recomputed without
// allocating anything (its partial sums in a fixed device array).
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
// thermo sums without allocation
//
// Some callers cannot let a library call cudaMalloc/cudaFree: applications
// whose device memory is already handed out by a framework's caching
// allocator (a fresh cudaMalloc can fail even though the framework has free
// memory in its pool), loops that must not pay for an allocation or the
// device-wide synchronisation cudaFree can imply, and programs that forbid
// allocating once they are initialised.  lb_thermo_static serves them: its
// FP64 partial sums live in the fixed array below instead of the context's
// own buffer, so the call allocates nothing.
// ======================================================================

namespace {

// room for the per-block partial sums of up to STATIC_THERMO_BLOCKS blocks
// plus the final record (NTHERMO sums, flip count, error word) and the
// blocks-finished counter: (1024 + 1) * 16 + 2 doubles and 4 bytes =
// 131,220 bytes, held by every GPU that loads the library until the
// process exits.  The thermo grid has at most THERMO_BLOCKS_PER_SM blocks
// per SM, so 1024 blocks cover GPUs of up to 256 SMs.
constexpr int STATIC_THERMO_BLOCKS = 1024;
static_assert(STATIC_THERMO_BLOCKS >= THERMO_BLOCKS_PER_SM * 256, "static thermo scratch below 256 SMs");
static __device__ __align__(256) double g_thermo_scratch[(STATIC_THERMO_BLOCKS + 1) * NTHERMO + 2];
static __device__ unsigned int g_thermo_done;

// device address of g_thermo_scratch per device, looked up once per device
// (the host-side name of a __device__ array is not a device address)
constexpr int STATIC_MAX_DEVICES = 64;
double *g_thermo_scratch_dev[STATIC_MAX_DEVICES] = {};
unsigned int *g_thermo_done_dev[STATIC_MAX_DEVICES] = {};
std::mutex g_thermo_scratch_mu;

}  // namespace

extern "C" int lb_thermo_static(lb_ctx *ctx, lb_thermo_t *out) {
  NEED_CTX();
  if (!out) return ctx->fail(LB_E_ARG, "null output");
  if (ctx->tq_n) {
    TRY(set_device(ctx));
    TRY(read_all_deferred(ctx));
  }
  if (!ctx->fields_valid || !ctx->thermo_valid) return ctx->fail(LB_E_ORDER, "no fields yet: call lb_iteration first");
  // the field planes must describe the live state: written by the last
  // iteration executed, with no state replaced and no step count set since
  // (mask, deposits and removed mass are read live)
  if (ctx->fields_step != ctx->t || ctx->thermo.step != ctx->t)
    return ctx->fail(LB_E_ORDER, "the node fields are not those of the current state (step %lld): the "
                     "record can be recomputed only after an iteration whose last step is a thermo step",
                     (long long)ctx->t);
  if (ctx->device < 0 || ctx->device >= STATIC_MAX_DEVICES)
    return ctx->fail(LB_E_UNSUPPORTED, "device %d is beyond the %d devices the static scratch serves",
                     ctx->device, STATIC_MAX_DEVICES);
  if (ctx->tblocks > STATIC_THERMO_BLOCKS)
    return ctx->fail(LB_E_ARG, "lattice needs %d blocks of partial sums; the static scratch holds %d",
                     ctx->tblocks, STATIC_THERMO_BLOCKS);
  TRY(set_device(ctx));
  double *scratch = nullptr;
  unsigned int *done = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_thermo_scratch_mu);
    if (!g_thermo_scratch_dev[ctx->device]) {
      cudaError_t e = cudaGetSymbolAddress((void **)&g_thermo_scratch_dev[ctx->device], g_thermo_scratch);
      if (e == cudaSuccess) e = cudaGetSymbolAddress((void **)&g_thermo_done_dev[ctx->device], g_thermo_done);
      if (e != cudaSuccess) {
        g_thermo_scratch_dev[ctx->device] = nullptr;
        g_thermo_done_dev[ctx->device] = nullptr;
        return ctx->cuda_fail(e, "cudaGetSymbolAddress(g_thermo_scratch)");
      }
    }
    scratch = g_thermo_scratch_dev[ctx->device];
    done = g_thermo_done_dev[ctx->device];
  }
  // every slot the kernels read is written by the same call first, so the
  // contents a previous call left behind need no clearing
  ThermoArgs ta{};
  ta.g = ctx->g;
  ta.mask = ctx->mask;
  ta.fields = ctx->fields;
  ta.nc = ctx->nc;
  ta.Cfield = ctx->qs ? ctx->Cfield : nullptr;
  ta.b = ctx->react ? ctx->b : nullptr;
  ta.removed = ctx->react ? ctx->removed : nullptr;
  ta.partials = scratch;
  ta.out = scratch + (size_t)STATIC_THERMO_BLOCKS * NTHERMO;
  ta.done = done;  // zero at load; the last block of every call resets it
  ta.nflips = ctx->nflips;
  ta.errw = ctx->errw;
  LAUNCH(launch_thermo(ta, ctx->tblocks, ctx->stream));
  double rec[NTHERMO + 2];
  CK(cudaMemcpyAsync(rec, ta.out, sizeof rec, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const double *h = rec;
  unsigned long long nfl = 0;
  memcpy(&nfl, &rec[NTHERMO], sizeof nfl);
  if ((int)rec[NTHERMO + 1]) {
    CK(cudaMemsetAsync(ctx->errw, 0, sizeof(int), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return ctx->fail(LB_E_TIMEOUT, "a TMA pipeline wait timed out before step %lld", (long long)ctx->t);
  }
  lb_thermo_t T;
  memset(&T, 0, sizeof T);
  T.step = ctx->t;
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
  *out = T;
  for (int q = 0; q < NTHERMO; q++)
    if (!std::isfinite(h[q])) return ctx->fail(LB_E_NAN, "thermo sum %d is not finite", q);
  return LB_OK;
}
