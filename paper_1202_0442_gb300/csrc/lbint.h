// lbint.h -- internal interface between the host orchestration and the
// kernels: argument structs (passed by value to the kernels) and the
// launch functions each kernel file exports.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace lbk {

enum { ST_FP32 = 0, ST_FP16 = 1, ST_BF16 = 2 };
enum { OPEN_NONE = 0, OPEN_POISEUILLE = 1, OPEN_UNIFORM = 2, OPEN_DIRICHLET = 3,
       OPEN_GRADIENT = 4 };
enum { SOL_NONE = 0, SOL_DIRICHLET = 1, SOL_ADIABATIC = 2, SOL_FLUX = 3 };

constexpr int MAX_OPEN = 8;
constexpr int NFIELD = 4;   // per component: drho, px, py, drho_eq
constexpr int NTHERMO = 16; // FP64 thermo partial sums per block

struct OpenDesc {
  int wall;      // 0 xlo, 1 xhi, 2 ylo, 3 yhi
  int a0, a1;    // extent along the wall
  int kind;      // 0 inlet, 1 outlet
  int style[2];  // OPEN_* per component
  float v[2];    // speed (uniform) or v_max (poiseuille)
  float rho[2];  // density held by dirichlet
  float drho[2]; // that density minus the component's rho_ref (from FP64)
  int sstyle;    // SOL_* for the solute
  float Cbar;    // dirichlet concentration, or C0 of the flux style
  float sv;      // velocity v of the flux style
};

// where an opening lies on the lattice border: wall | a0 << 2, and a1.
// Kept in the launch parameters for the membership tests, which every
// border node makes; the full descriptor (64 B) is read from device memory
// only by the opening's own nodes.
struct OpenSpan {
  int wa0;
  int a1;
};

// the fluid rule of an opening, in the launch parameters of the fluid
// kernels (its own nodes read it in every iteration; from the constant bank
// it costs no registers): styles and kind packed, and one value per
// component, the speed (uniform) or v_max (poiseuille), or for dirichlet the
// density minus rho_ref (a velocity rule does not use that difference)
struct OpenRule {
  int bits;      // style[0] | style[1] << 3 | kind << 6
  float val[2];
};

struct Geometry {
  int nx, ny, pitch, mw;  // ny: rows held (a slab: its own rows and its
                          // ghost rows); mw = pitch / 32 mask words per row
  size_t plane;           // ny * pitch
  // own rows [ylo, yhi) (every row of a whole lattice): the rows a
  // context updates for good, sums (thermo) and reads out; computed rows
  // [clo, chi) (the own rows, and for a slab with surface reaction also
  // the two ghost rows on each side next to them, updated redundantly so
  // that the precipitation and growth of the boundary rows need no
  // exchange within the iteration); local row y is row y + yoff of the
  // whole lattice of gny rows (yoff = 0, gny = ny for a whole lattice)
  int ylo, yhi, clo, chi, yoff, gny;
};

// one iteration of the fluid lattice(s)
// rest-state share s_i = w_i A_i of population i under the fluids
// command's density-ratio parameter alpha (Eq. (2) weights at alpha = 4/9)
#ifdef __CUDACC__
__host__ __device__
#endif
inline double wshare(int i, double alpha) {
  if (alpha == 4.0 / 9.0) return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  return i == 0 ? alpha : (i < 5 ? (1.0 - alpha) / 5.0 : (1.0 - alpha) / 20.0);
}

struct FluidArgs {
  Geometry g;
  const void *fin;        // populations before the step [nc][9][plane]
  void *fout;             // populations after the step
  const uint32_t *mask;
  const uint16_t *nbc;    // per node slot [plane]: the solid bits of its 3 x 3
                          // neighbourhood (NBPOS layout, periodic wrap);
                          // slots past nx read as solid
  float rho_ref[2];
  float scale, inv_scale; // storage scale 2^s and 2^-s (FP16), else 1
  float tau[2], omega[2];
  float wa[2], wd[2];     // rest-state shares s_1..4, s_5..8 (fluids alpha)
  float fx[2], fy[2];     // aveforce
  float ax[2], ay[2];     // aveacceleration
  int ads[2];             // adhesiveforce on/off per component
  float Gads[2], ads_psi0[2], ads_rho0[2];
  float G, psi0, sc_rho0; // interforce
  int nopen;
  OpenSpan span[MAX_OPEN];
  OpenRule rule[MAX_OPEN];
  float *fields;          // [nc][NFIELD][plane] or nullptr
  float *uout;            // [2][plane] solvent velocity or nullptr
  uint32_t sr_seed;       // 16-bit stores: 0 = round to nearest, else the
                          // step's seed of the stochastic-rounding dither
  uint32_t step_seed;     // per-iteration seed of the mass-exact collision
  // boundary_style slip/mixed/hybrid: reflection coefficient R of the solid
  // nodes, uniform (slipR) or per node (Rmap [nc][plane], read on solid
  // nodes); edge_x/edge_y: the x/y edge carries an opening (not periodic)
  int pm;                 // momentum as an exact hi + lo sum (LB_PRECISE_MOMENTUM)
  int slip;
  float slipR[2];
  const float *Rmap;
  int edge_x, edge_y;
};

// gradient openings (after collision)
struct GradArgs {
  Geometry g;
  void *f;                // populations after the step
  float *fields;          // or nullptr
  const uint32_t *mask;
  int nc;
  int nopen;
  const OpenDesc *op;     // [nopen] descriptors in device memory (the
                          // launch parameters stay small: launch latency)
  int maxlen;             // nodes of the longest of these openings
  float inv_scale, scale;
};

// one iteration of the solute lattice
struct SoluteArgs {
  Geometry g;
  const float *gin;       // [q][plane]
  float *gout;
  const uint32_t *mask;
  const uint16_t *nbc;    // neighbour codes (as FluidArgs::nbc)
  const float *u;         // [2][plane] solvent velocity of this step
  float omega;
  int react;
  float kr, Cs;
  float rden[2];          // 1 / (kr + 2 w) for the axis (D2Q4: all) and diagonal weights
  float *db;              // deposit share per fluid node
  float *Cfield;          // or nullptr
  int nopen;
  OpenSpan span[MAX_OPEN];
  const OpenDesc *op;     // [nopen] descriptors in device memory (the
                          // launch parameters stay small: launch latency)
  float D;                // diffusion coefficient (tau_s - 1/2)/2 or /3
  // intersolute: concentrations after streaming and the opening rules,
  // written by a first pass (Cpre_out) and read by the update (Cpre)
  int inter;
  float isG, ispsi0, isC0, taus;
  const float *Cpre;
  float *Cpre_out;
};

// precipitation gather and growth decisions / flips
struct GrowthArgs {
  Geometry g;
  uint32_t *mask;
  const float *db;
  double *b;
  uint16_t *nbc;          // neighbour codes, refreshed around every flip
  unsigned int *flip;     // per node: chosen to turn solid this step
  unsigned int *flist;    // the chosen nodes (plane offsets), *fcount of them
  unsigned int *fcount;
  double bmax, b0;
  uint64_t seed;
  int64_t t;              // 1-based iteration number
  int rlo, rhi;           // rows whose solid nodes gather and decide (a
                          // slab: its own rows and one ghost row each side;
                          // only own-row nodes are turned solid)
  unsigned int *slist;    // whole lattice: the solid nodes that had a fluid
  unsigned int *scount;   // neighbour when listed (plane offsets, *scount of
                          // them; flipped nodes are appended), or nullptr:
                          // the rows [rlo, rhi) are scanned
  int sblocks;            // blocks of the launch over the list
  unsigned int *done;     // CTAs of that launch finished (0 between launches)
  int q;
  int nopen;
  OpenSpan span[MAX_OPEN];
  // flip application
  void *f;                // fluid populations after the step [nc][9][plane]
  void *f_prev;           // the other population buffer
  int nc;
  float rho_ref[2];
  float inv_scale;
  float *gpop;            // solute populations after the step
  double *removed;        // [nc + 1][plane] booked mass of flipped nodes
  unsigned long long *nflips;
};

// thermo reduction over the node fields
struct ThermoArgs {
  Geometry g;
  const uint32_t *mask;
  const float *fields;    // [nc][NFIELD][plane]
  int nc;
  const float *Cfield;    // or nullptr
  const double *b;        // or nullptr
  const double *removed;  // [nc + 1][plane] or nullptr
  double *partials;       // [nblocks][NTHERMO]
  double *out;            // [NTHERMO + 2]: the sums, then the flip count
                          // (its 64 bits) and the TMA error word
  unsigned int *done;     // blocks finished (0 between calls): the last
                          // block reduces the partial sums
  const unsigned long long *nflips;  // or nullptr
  const int *errw;        // or nullptr
};

// device-to-device copies of up to MAX_RUNS contiguous runs in one launch
constexpr int MAX_RUNS = 128;
struct CopyRuns {
  int n;
  const void *src[MAX_RUNS];
  void *dst[MAX_RUNS];
  unsigned bytes[MAX_RUNS];
};

// launchers (return the kernel count launched, or -1 on a launch error)
int launch_fluid(int storage, int nc, bool sc, bool mass_exact, const FluidArgs &a, cudaStream_t s);
int launch_gradient(int storage, const GradArgs &a, cudaStream_t s);
// fluid and solute iteration in one kernel (one component, no interforce,
// no intersolute, no exact momentum pairs, streaming kernel)
int launch_fluid_solute(int storage, int q, const FluidArgs &a, const SoluteArgs &sa, cudaStream_t s);
// neighbour codes of every node slot from the mask (after any mask upload)
// (rows [r0, r1) only, r1 < 0: to the last row)
int launch_nbcode(const uint32_t *mask, uint16_t *nbc, const Geometry &g, cudaStream_t s, int r0 = 0,
                  int r1 = -1);
// persistent TMA-pipelined single-component kernel (k_tma.cu); err is a
// device word the kernel sets when an mbarrier wait runs past `limit`
// clock cycles (negative: the default, about two seconds)
bool tma_supported(int storage, const Geometry &g);
int launch_fluid_tma(int storage, const FluidArgs &a, int *err, long long limit, cudaStream_t s, int sms);
// one solute iteration (two kernels with intersolute: concentrations, then the update)
int launch_solute(int q, const SoluteArgs &a, cudaStream_t s);
int launch_surface_list(const GrowthArgs &a, cudaStream_t s);
// a growth step (gather, decisions and flips): one or two launches
int launch_growth(int storage, const GrowthArgs &a, cudaStream_t s);
// thermo grid: one block per row, at most THERMO_BLOCKS_PER_SM per SM
constexpr int THERMO_BLOCKS_PER_SM = 4;
int thermo_blocks(const Geometry &g, int sms);
int launch_thermo(const ThermoArgs &a, int nblocks, cudaStream_t s);
int launch_copy_runs(const CopyRuns &r, cudaStream_t s);

// state conversion between FP64 host-layout arrays [q][ny][nx] and storage
int launch_import_pops(int storage, const double *src, void *dst, const uint32_t *mask,
                       Geometry g, int q, float rho_ref, float scale, bool shift,
                       double alpha, cudaStream_t s);
int launch_export_pops(int storage, const void *src, double *dst, const uint32_t *mask,
                       Geometry g, int q, float rho_ref, float inv_scale, bool shift,
                       double alpha, cudaStream_t s);
int launch_equilibrium(int storage, const double *rho, const double *ux, const double *uy,
                       void *dst, const uint32_t *mask, Geometry g, float rho_ref,
                       float scale, double alpha, cudaStream_t s);
int launch_solute_equilibrium(int q, const double *C, const double *ux, const double *uy,
                              float *dst, const uint32_t *mask, Geometry g, cudaStream_t s);
int launch_export_fields(const float *fields, int comp, const uint32_t *mask, Geometry g,
                         float rho_ref, double *rho, double *px, double *py, double *req,
                         cudaStream_t s);
int launch_export_velocity(const float *fields, int nc, const uint32_t *mask, Geometry g,
                           const float *rho_ref, float *rho, float *ux, float *uy,
                           cudaStream_t s);
int launch_export_plane_f32(const float *src, const uint32_t *mask, Geometry g, double *dst,
                            cudaStream_t s);
int launch_export_plane_f64(const double *src, Geometry g, double *dst, cudaStream_t s);
int launch_import_plane_f64(const double *src, Geometry g, double *dst, cudaStream_t s);

}  // namespace lbk
