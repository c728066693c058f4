// lbctx.h -- the command state and device state of one lattice (the
// lb_ctx behind the C ABI of include/lb2d.h), shared by the host-side
// translation units: lb2d_api.cu (commands, device state, iteration) and
// lb2d_io.cu (input-data and restart text files).
#pragma once

#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "lb2d.h"
#include "lbint.h"

// an inlet or outlet opening (inlet/outlet command) with its momentum
// style per fluid (inlet_momentum/outlet_momentum) and solute style
// (inlet_solute/outlet_solute)
struct Opening {
  int wall = 0, a0 = 0, a1 = 0, kind = 0;
  std::string label[2];
  int style[2] = {lbk::OPEN_NONE, lbk::OPEN_NONE};
  double v[2] = {0, 0}, rho[2] = {1, 1};
  int sstyle = lbk::SOL_NONE;
  double C = 0, sv = 0;  // dirichlet C or flux C0; flux velocity
};

struct lb_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  uint64_t launches = 0;

  // command state
  bool have_lattice = false, have_style = false, have_region = false;
  bool momentum_cmd = false, committed = false;
  bool iterated = false;  // an iteration has run (write_restart must come first)
  int nx = 0, ny = 0, nc = 1;
  double tau[2] = {1, 1};
  double alpha[2] = {4.0 / 9.0, 4.0 / 9.0};  // fluids command, density-ratio parameter
  int qs = 0;
  double taus = 1.0;
  int storage = lbk::ST_FP32;
  bool sr = false;
  bool pm = false;  // LB_PRECISE_MOMENTUM
  double rho_ref[2] = {1, 1};
  float scale = 1.f, inv_scale = 1.f;
  std::vector<uint8_t> solid, region;
  // boundary_style: 0 noslip, 1 slip, 2 mixed (slipR), 3 hybrid (Rh per
  // solid node and component, from the styled obstacle calls)
  int bstyle = 0;
  double slipR = 0.0;
  std::vector<float> Rh[2];
  float *Rmap = nullptr;
  // opening descriptors the kernels read (all openings; the gradient
  // ones), uploaded when they change, and the host copies last uploaded
  lbk::OpenDesc *d_open = nullptr, *d_grad = nullptr;
  std::vector<lbk::OpenDesc> h_open, h_grad;
  std::vector<double> paint_f[2], paint_C;
  // nodes whose painted values are still those read by read_data (cleared
  // by the first momentum0 / concentration0 that reaches them)
  std::vector<uint8_t> paint_base[2], paint_base_C;
  bool painted_f[2] = {false, false}, painted_C = false;
  bool state_set[2] = {false, false}, solute_set = false;
  double fave[2][2] = {{0, 0}, {0, 0}}, acc[2][2] = {{0, 0}, {0, 0}};
  bool ads[2] = {false, false};
  double Gads[2] = {0, 0}, ads_psi0[2] = {0, 0}, ads_rho0[2] = {0, 0};
  bool sc = false;
  double G = 0, psi0 = 0, sc_rho0 = 0;
  std::vector<Opening> open;
  bool react = false;
  double kr = 0, Cs = 0, b0 = 0, bmax = 0;
  bool inter = false;  // intersolute command
  double isG = 0, ispsi0 = 0, isC0 = 0;
  uint64_t seed = 0;
  int nf = 0;
  int nout = 0;  // output command: node fields every nout iterations (0: off)
  // processors command: a px x py grid of processes; a context given a
  // rank (lb_processor_rank) holds one y slab of the lattice: rows
  // [sy0, sy0 + sny) and `halo` ghost rows on each side
  int px = 1, py = 1;
  int rank = -1;  // -1: the whole lattice
  int halo = 0, sy0 = 0, sny = 0;

  // device state
  lbk::Geometry g{};
  void *fbuf[2] = {nullptr, nullptr};
  int cur = 0;
  uint32_t *mask = nullptr;
  float *fields = nullptr, *u = nullptr, *gbuf[2] = {nullptr, nullptr};
  float *Cfield = nullptr, *db = nullptr, *Cpre = nullptr;
  float *vstage = nullptr;  // lb_get_velocity_f32 staging (3 planes, kept)
  double *b = nullptr, *removed = nullptr;
  unsigned int *flip = nullptr, *flist = nullptr, *fcount = nullptr;
  // surface list of the growth gather (whole lattice with surface reaction):
  // rebuilt at the next step whenever the device mask is replaced
  unsigned int *slist = nullptr, *scount = nullptr, *gdone = nullptr;
  bool slist_valid = false;
  int sblocks = 0;
  uint16_t *nbc = nullptr;  // per-node neighbour codes of the streaming kernel
  // host copy of the device mask words while the two are known to agree
  // (lost once growth may have changed the device mask)
  std::vector<uint32_t> mask_host;
  bool mask_host_valid = false;
  // caller-owned device buffers (lb_bind): f0, f1, g0, g1, fields, u
  void *bound[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  size_t bound_bytes[6] = {0, 0, 0, 0, 0, 0};
  unsigned long long *nflips = nullptr;
  double *partials = nullptr, *tout = nullptr;
  unsigned int *tdone = nullptr;  // thermo blocks finished (reset by the last)
  int tblocks = 0;
  int64_t t = 0;
  int debug = 0;          // LB_DEBUG_* flags (lb_set_debug)
  // LB_DEBUG_GUARDS: allocations made with guard zones (raw block, the
  // pointer handed out, its size)
  struct Guarded {
    void *raw, *user;
    size_t bytes;
  };
  std::vector<Guarded> guarded;
  int kernel = 0;        // 0 auto (streaming), 1 streaming (k_fluid_local), 2 TMA pipeline,
                         // 3 fused fluid-solute
  int *errw = nullptr;   // device error word of the TMA kernel
  long long wait_limit = -1;  // TMA kernel's wait limit in clock cycles (-1: its default)
  int sms = 0;
  bool fields_valid = false;
  int64_t fields_step = -1;  // iteration whose end state the field planes hold
  lb_thermo_t thermo{};
  bool thermo_valid = false;
  // lb_thermo_deferred: records copied to page-locked host memory in stream
  // order (two slots, an event after each copy) and read, oldest first,
  // when a call needs them
  bool tdefer = false;
  double *trec_host = nullptr;  // [2][NTHERMO + 2]
  cudaEvent_t trec_ev[2] = {nullptr, nullptr};
  int64_t trec_step[2] = {0, 0};
  int tq[2] = {0, 0}, tq_n = 0, tq_next = 0;

  // read_data command: the state read from input-data files, applied when
  // the device state is created (kind 1: populations a; kind 2: the
  // equilibrium of the density or concentration a at velocity (ux, uy))
  struct ReadState {
    int kind = 0;
    std::vector<double> a, ux, uy;
  };
  ReadState rf[2], rg;
  std::vector<double> rb;  // deposits b read (empty: b0 on every solid node)
  // write_restart command: the state written every restart_nf iterations
  std::string restart_file;
  int restart_nf = 0;

  int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    err = buf;
    return code;
  }
  int cuda_fail(cudaError_t e, const char *what) {
    return fail(LB_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
  }
};

#define CK(call)                                                   \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return ctx->cuda_fail(e_, #call);       \
  } while (0)

#define LAUNCH(expr)                                                              \
  do {                                                                            \
    int n_ = (expr);                                                              \
    if (n_ < 0) return ctx->cuda_fail(cudaGetLastError(), "kernel launch");       \
    ctx->launches += (uint64_t)n_;                                                \
  } while (0)

#define NEED_CTX()                              \
  do {                                          \
    if (!ctx) return LB_E_ARG;                  \
  } while (0)

#define TRY(x)               \
  do {                       \
    int r_ = (x);            \
    if (r_ != LB_OK) return r_; \
  } while (0)

// an NVTX range over a scope: the library's phases show up by name in
// Nsight Systems timelines and can select kernels in Nsight Compute
// (--nvtx --nvtx-include "lb_iteration/"); without a tool attached a push
// or pop costs a pointer test
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// write the state of `ctx` as input-data text files named base (one
// fluid), base.fluid1 / base.fluid2 (two) and base.solute (write_restart
// command); lb2d_io.cu
int write_data_files(lb_ctx *ctx, const std::string &base);
