/*
 * lb2d.h -- C ABI of the GB300 lattice Boltzmann library.
 *
 * One call per command of the paper's command set (arXiv:1202.0442,
 * "Introduction to Perl module lb2d.pm 0.1", Sec. Commands): set up a
 * lattice with lb_lattice, geometry, openings, forces and initial state,
 * then advance it with lb_iteration and read the thermo record and fields.
 * All per-iteration work runs in the library's CUDA kernels for sm_103a.
 *
 * Conventions
 *   - Every call returns int: LB_OK (0) or a negative LB_E_* code;
 *     lb_last_error() gives the message of the last failure on a context.
 *   - Nodes are (x, y), 0 <= x < nx, 0 <= y < ny.  A paper script's
 *     lattice(N_x, N_y) has nx = N_x + 1, ny = N_y + 1 (lattice command:
 *     the sites run from 0 to N_x).  Node arrays passed in or out
 *     are dense row-major [ny][nx] (x fastest); population arrays are
 *     [q][ny][nx] with the D2Q9 numbering e0=(0,0) e1=(1,0) e2=(0,1)
 *     e3=(-1,0) e4=(0,-1) e5=(1,1) e6=(-1,1) e7=(-1,-1) e8=(1,-1) and the
 *     D2Q4 numbering g1..g4 = +x,+y,-x,-y at index 0..3.
 *   - Host pointers are borrowed for the duration of the call; the library
 *     copies what it needs.  Pinned host memory makes the copies faster
 *     but is not required.  Device memory is owned by the library and
 *     released by lb_destroy, except state buffers the caller supplies
 *     with lb_bind (the caller's to free, after lb_destroy).
 *   - Calls on one context run on the CUDA stream given to lb_create, in
 *     order; calls that return host data synchronise that stream.  A
 *     context is not thread safe.
 *   - Fluid components are numbered 1 and 2 as in the paper's commands
 *     (the "fluid" argument); 1 is the only one of a single-component run.
 */
#ifndef LB2D_H
#define LB2D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LB_OK 0
#define LB_E_ORDER (-1)       /* command out of the required order */
#define LB_E_ARG (-2)         /* invalid argument or inconsistent setup */
#define LB_E_UNSUPPORTED (-3) /* valid in the paper, not built here */
#define LB_E_CUDA (-4)        /* CUDA runtime error (message has details) */
#define LB_E_NAN (-5)         /* thermo found a non-finite sum */
#define LB_E_NOMEM (-6)       /* device or host allocation failed */
#define LB_E_TIMEOUT (-7)     /* a bounded wait inside a kernel gave up */

/* population storage (lb_set_storage) */
#define LB_FP32 0 /* f_i - w_i rho_ref in FP32 */
#define LB_FP16 1 /* (f_i - w_i rho_ref) * 2^s in IEEE binary16 */
#define LB_BF16 2 /* f_i - w_i rho_ref in bfloat16 */
/* OR'd into LB_FP16 / LB_BF16: round stores stochastically (a dither drawn
 * from a hash of node, direction and iteration; reproducible) instead of
 * to nearest even */
#define LB_STOCHASTIC_ROUNDING 0x100
/* OR'd into any storage: form the momentum sum_i e_i f_i of single-component
 * lattices as an exact FP32 pair (error-free additions).  A rounded moment
 * feeds its rounding error back as a spurious force; in slow force-driven
 * flows (|j| much larger than the force per step) that biases u by up to
 * ~2e-5 relative in FP32.  Costs about 3 % (4096^2) to 9 % (1024^2) of the
 * streaming kernel's time; applies to the streaming and batched kernels. */
#define LB_PRECISE_MOMENTUM 0x200

typedef struct lb_ctx lb_ctx;
typedef struct lb_batch lb_batch;

/* thermo record (thermo command): FP64 sums over the state at the end of
 * the last iteration.  mass = sum of rho over fluid nodes; mom = sum of
 * the physical momentum j + F/2 (Eq. (4)); mass_eq = sum of the
 * equilibrium densities; solute = sum of C over fluid nodes; bsum = sum of
 * the precipitate b over solid nodes; removed* = fluid and solute mass of
 * nodes that surface growth turned solid. */
typedef struct {
  int64_t step;
  double mass[2];
  double mom[2];       /* x, y: mixture */
  double mom_comp[2][2];
  double mass_eq[2];
  double solute;
  double bsum;
  double removed[2];
  double removed_solute;
  int64_t nsolid;
  int64_t nfluid;
  int64_t flips; /* growth events since the start */
} lb_thermo_t;

/* ---- context --------------------------------------------------------- */

/* Create a context on CUDA device `device`, issuing all work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).  The
 * stream stays owned by the caller and must outlive the context. */
int lb_create(int device, void *cuda_stream, lb_ctx **out);
/* Free every device and host buffer of the context. */
int lb_destroy(lb_ctx *ctx);
/* Message of the last failing call on ctx (never NULL). */
const char *lb_last_error(const lb_ctx *ctx);
/* Number of kernels the context has launched so far (graph replays count
 * their kernel nodes). */
int lb_launch_count(const lb_ctx *ctx, uint64_t *out);

/* ---- initialization commands ---------------------------------------- */

/* lattice command: style "d2q9", nx x ny nodes, relaxation time tau > 1/2.
 * Must come first.  Boundaries are periodic until openings or obstacles
 * say otherwise.  Any nx, ny >= 1 up to 9 x round_up(nx, 32) x ny < 2^31
 * (about 238 M nodes; LB_E_UNSUPPORTED beyond: the kernels index a
 * component's planes with 32-bit offsets). */
int lb_lattice(lb_ctx *ctx, const char *style, int nx, int ny, double tau);

/* processors command (Sec. Commands, processors; Sec. Parallelization): the
 * px x py grid of processes the lattice is split over.  After lb_lattice
 * (LB_E_ORDER before it, as in the paper) and before the first iteration.
 * On its own it changes nothing: the context still holds the whole lattice.
 * With lb_processor_rank the context holds one piece of it; pieces are y
 * slabs, so px must be 1. */
int lb_processors(lb_ctx *ctx, int px, int py);

/* Make the context hold slab `rank` (0 <= rank < py) of a lattice split by
 * lb_processors(ctx, 1, py) into py y slabs: lattice rows [y0, y0 + n),
 * y0 = floor(rank ny / py), n = floor((rank + 1) ny / py) - y0, plus `halo`
 * ghost rows on each side (1; 2 with interforce or a slip, mixed or hybrid
 * boundary style; 3 with surface_reaction, whose slab also updates the two
 * ghost rows next to its own rows, redundantly, so that precipitation and
 * growth at its edges need nothing from its neighbours within an
 * iteration) that hold the neighbouring slabs' rows (periodic in y: slab
 * py - 1 and slab 0 are neighbours).  rank -1 returns to the whole
 * lattice.  After lb_processors, before the first iteration.
 * Every command of the setup is issued as for the whole lattice (node
 * coordinates, obstacle masks and initial-state arrays [..][ny][nx] of the
 * whole lattice); the context keeps the rows it holds.  The read-out calls
 * (lb_get_fields, lb_get_velocity_f32, lb_get_populations, lb_get_solute,
 * lb_get_mask) return the slab's own rows, arrays [..][n][nx]; lb_get_thermo
 * sums over the slab's own nodes (the lattice's record is the sum over the
 * slabs; lb_get_flips gives indices into the slab's own rows).  Each slab
 * draws the same random numbers for a node as the whole lattice does (the
 * growth pick included), so after every iteration followed by a halo
 * exchange the slabs hold, bit for bit, the rows of the whole lattice.
 * A slab of a lattice split into py > 1 advances one iteration per
 * lb_iteration call (LB_E_ORDER for Nt > 1): exchange halos between calls.
 * Not built for slabs (LB_E_UNSUPPORTED at the first iteration):
 * intersolute, the TMA kernel, batches.  A slab needs at least
 * max(3, 2 halo) rows (LB_E_ARG). */
int lb_processor_rank(lb_ctx *ctx, int rank);

/* The data the processes of a split lattice exchange after every iteration
 * (processors command, Sec. Parallelization; the paper does not fix its
 * form): lb_halo_size, lb_halo_pack, lb_halo_unpack, lb_exchange.
 *
 * Bytes of one halo message of a slab (either face; the same for every
 * slab of a lattice).  With one ghost row a face carries the populations
 * the pull takes across it: fluid directions 2, 5, 6 (moving to +y) or
 * 4, 7, 8 (to -y) of each component and the solute's (+y or -y) ones, one
 * row each; with two or three ghost rows every population of that many
 * rows, and with surface_reaction also those rows of the solid mask and
 * of the FP64 deposits.  Layout: planes in order (component, direction;
 * then solute direction; then mask words, deposits), each `halo` rows of
 * round_up(nx, 32) values of the storage type, every part starting at a
 * multiple of 16 bytes.  After the device state exists (LB_E_ORDER
 * before). */
int lb_halo_size(lb_ctx *ctx, size_t *bytes);

/* Copy the slab's own rows that its neighbour across face `face` (0: the
 * low-y side, the slab rank - 1; 1: the high-y side, rank + 1) needs into
 * the device buffer `buf` (lb_halo_size bytes, 16-byte aligned, on the
 * context's device); queued on the context's stream.  After an iteration,
 * the buffer of face 1 goes to slab rank + 1 and that of face 0 to rank - 1
 * (e.g. by NCCL), which unpack them into their face 0 and face 1. */
int lb_halo_pack(lb_ctx *ctx, int face, void *buf);

/* Fill the slab's ghost rows on face `face` (0: low y, from slab rank - 1's
 * face-1 message; 1: high y, from rank + 1's face-0 message) from the
 * device buffer `buf`; queued on the context's stream. */
int lb_halo_unpack(lb_ctx *ctx, int face, const void *buf);

/* The halo exchange of all n slabs of one lattice held in one process on
 * one device and stream (ctxs[r] holds slab r of n): each slab's first and
 * last own rows go to its neighbours' ghost rows, device to device, in one
 * launch on that stream.  Call after every iteration of the slabs (all at
 * the same step).  LB_E_ARG if the contexts are not the slabs of one
 * lattice at one step, LB_E_UNSUPPORTED if they do not share the device
 * and stream. */
int lb_exchange(lb_ctx *const *ctxs, int n);

/* fluids command: two components with relaxation times tau1, tau2 and
 * density-ratio parameters alpha1, alpha2 in [0, 1) (LB_E_ARG otherwise).
 * Component s then relaxes to f_eq,i = w_i rho [A_i + 3 e.u + 9/2 (e.u)^2
 * - 3/2 u.u] with A_0 = (9/4) alpha_s, A_{1..8} = (9/5)(1 - alpha_s), so its
 * sound speed squared is (3/5)(1 - alpha_s); alpha = 4/9 is Eq. (2).  Must
 * follow lb_lattice and precede openings, initial state and forces. */
int lb_fluids(lb_ctx *ctx, double tau1, double tau2, double alpha1,
              double alpha2);

/* solute command: one solute on a D2Q4 (q = 4, the paper's lattice) or
 * D2Q9 (q = 9) lattice with relaxation time taus > 1/2; D = (taus-1/2)/2
 * on D2Q4, (taus-1/2)/3 on D2Q9. */
int lb_solute(lb_ctx *ctx, double taus, int q);

/* Population storage: LB_FP32, LB_FP16 or LB_BF16 (the 16-bit ones
 * optionally | LB_STOCHASTIC_ROUNDING; any | LB_PRECISE_MOMENTUM).
 * Populations are kept
 * as deviations f_i - w_i rho_ref[c] from the rest state of reference
 * density rho_ref[c] (one per component; NULL = 1.0); FP16 stores them
 * multiplied by the power of two 2^s with s the largest integer such that
 * h_max * 2^s <= 2^14, h_max being the largest |f_i - w_i rho_ref| the
 * run will see (<= 0 picks 0.25 * max rho_ref); a deviation beyond the
 * format's range (about 4 h_max) is stored as infinite by the stochastic
 * and nearest roundings (the next thermo evaluation then returns
 * LB_E_NAN; the mass-exact collision of two components clamps it), so
 * h_max must bound the run.  Arithmetic is FP32 in all three.  Before the
 * first lb_iteration only. */
int lb_set_storage(lb_ctx *ctx, int storage, const double *rho_ref,
                   double h_max);

/* boundary_style command: how fluid populations meet solid nodes.
 *   "noslip": half-way bounce-back.
 *   "slip": mirror reflection at flat walls (Fig. slip).  A diagonal mode
 *     (a, b) of node x whose source x - (a, b) is solid arrives instead from
 *     x - (2a, 0) as mode (a, -b) when x - (0, b), x - (2a, b) are solid and
 *     x - (a, 0), x - (2a, 0) fluid (a wall along x), or from x - (0, 2b) as
 *     mode (-a, b) when x - (a, 0), x - (a, 2b) are solid and x - (0, b),
 *     x - (0, 2b) fluid (a wall along y); every other case, the axis modes,
 *     and paths across an edge of the lattice that carries an opening are
 *     bounced back.  Each reflection pairs with its reverse, so mass is kept.
 *   "mixed": a fraction R (0 <= R <= 1) slips, 1 - R bounces back.
 *   "hybrid": R per solid node and fluid, from lb_obstacle_*_styled or
 *     lb_obstacle_mask_hybrid (plain obstacle calls give noslip nodes;
 *     nodes that turn solid by growth are noslip).
 * R is read by "mixed" only.  The solute always bounces back (or reacts).
 * Must precede obstacles.  Slip styles run on the streaming kernels and
 * are not available to batched lattices. */
int lb_boundary_style(lb_ctx *ctx, const char *style, double R);

/* obstacle command: mark nodes solid.  Rectangle with inclusive bounds;
 * circle (x-xc)^2 + (y-yc)^2 <= r^2 with periodic distance; mask: nx*ny
 * bytes, nonzero = solid (for generated media).  After lb_boundary_style
 * (LB_E_ORDER otherwise).  Solid overrides openings and initial state. */
int lb_obstacle_rect(lb_ctx *ctx, int x0, int x1, int y0, int y1);
int lb_obstacle_circle(lb_ctx *ctx, int xc, int yc, int r);
int lb_obstacle_mask(lb_ctx *ctx, const uint8_t *mask);

/* obstacle command with the hybrid style's extra arguments: style1 for
 * fluid 1 and style2 for fluid 2 ("noslip", "slip" or "mixed" with its
 * coefficient arg; NULL style2 repeats style1; NULL style1 is noslip).
 * Outside the hybrid style the styles are checked and otherwise ignored. */
int lb_obstacle_rect_styled(lb_ctx *ctx, int x0, int x1, int y0, int y1,
                            const char *style1, double arg1,
                            const char *style2, double arg2);
int lb_obstacle_circle_styled(lb_ctx *ctx, int xc, int yc, int r,
                              const char *style1, double arg1,
                              const char *style2, double arg2);
/* mask form: R, if not NULL, holds [ncomp][ny][nx] reflection
 * coefficients in [0, 1] read on the masked nodes (needs the hybrid
 * style; LB_E_ORDER otherwise); NULL makes them noslip. */
int lb_obstacle_mask_hybrid(lb_ctx *ctx, const uint8_t *mask, const double *R);

/* inlet/outlet commands: an opening on wall "xlo", "xhi", "ylo" or "yhi"
 * spanning a0..a1 along it (y for x-walls, x for y-walls).  label1 names
 * it for fluid 1 (and the solute), label2 for fluid 2 (NULL with one
 * component).  Openings on one wall may not overlap; two walls may not
 * both have an opening on a shared corner node.  At most 8 openings per
 * lattice (LB_E_UNSUPPORTED beyond: where each lies and its fluid rule
 * travel in the kernels' launch parameters). */
int lb_inlet(lb_ctx *ctx, const char *wall, int a0, int a1,
             const char *label1, const char *label2);
int lb_outlet(lb_ctx *ctx, const char *wall, int a0, int a1,
              const char *label1, const char *label2);

/* inlet_momentum/outlet_momentum commands (App. A): style "poiseuille"
 * (v = v_max of the profile), "uniform" (v = speed, into the domain for
 * an inlet and out of it for an outlet), "dirichlet" (rho held), or
 * "gradient" (extrapolation after collision).  rho is the opening's
 * density (held by dirichlet; initial value for the others).  |v| < 1. */
int lb_inlet_momentum(lb_ctx *ctx, const char *label, const char *style,
                      double v, double rho);
int lb_outlet_momentum(lb_ctx *ctx, const char *label, const char *style,
                       double v, double rho);

/* inlet_solute/outlet_solute commands (App. B): "dirichlet" (C held at C),
 * "adiabatic" (zero flux; C is the initial value) or "flux" (C is the
 * injected concentration C0, v its velocity: after streaming the opening
 * node takes C = (v C0 + D C1)/(D + v) on an inlet, (v C0 - D C1)/(v - D)
 * on an outlet, C1 the streamed concentration of the nearest inner node,
 * D = (tau_s - 1/2)/2 on D2Q4 or /3 on D2Q9, and every mode is set to
 * g_eq(C, u); v = D on an outlet is LB_E_ARG at the first iteration).  v
 * is ignored by the other styles.  Every opening needs a solute style when
 * a solute is on; an opening with a solute style but no momentum style
 * leaves the fluid periodic across its wall. */
int lb_inlet_solute(lb_ctx *ctx, const char *label, const char *style,
                    double C, double v);
int lb_outlet_solute(lb_ctx *ctx, const char *label, const char *style,
                     double C, double v);

/* surface_reaction command: rate kr >= 0, saturation Cs, style "growth",
 * initial deposit b0 on every solid node, growth threshold bmax.  seed
 * selects the growth choices (SplitMix64 of seed ^ (t*nx*ny + node)).
 * After lb_solute. */
int lb_surface_reaction(lb_ctx *ctx, double kr, double Cs,
                        const char *style, double b0, double bmax,
                        uint64_t seed);

/* position0 command: select the region the next momentum0 /
 * concentration0 calls fill (rectangle inclusive, circle as obstacle). */
int lb_position0_rect(lb_ctx *ctx, int x0, int x1, int y0, int y1);
int lb_position0_circle(lb_ctx *ctx, int xc, int yc, int r);

/* momentum0 command: add value to population `mode` (0..8) of fluid
 * `fluid` on the fluid nodes of the last position0 region (values of
 * repeated calls add up; negative values subtract).  LB_E_ORDER without a
 * preceding position0. */
int lb_momentum0(lb_ctx *ctx, int mode, double value, int fluid);

/* concentration0 command: add value to the concentration of the last
 * position0 region (populations at equilibrium with the fluid at rest). */
int lb_concentration0(lb_ctx *ctx, double value);

/* read_data "equilibrium" analogue: populations of fluid `fluid` become
 * f_eq(rho, u) of Eq. (2) on fluid nodes.  rho, ux, uy: host [ny][nx]
 * FP64 (ux/uy may be NULL = 0).  Allowed before or after iterations. */
int lb_set_equilibrium(lb_ctx *ctx, int fluid, const double *rho,
                       const double *ux, const double *uy);
/* Same for the solute: g = g_eq(C, u) of Eq. (3) (D2Q9: w_i C(1+3e.u)). */
int lb_set_solute_equilibrium(lb_ctx *ctx, const double *C,
                              const double *ux, const double *uy);
/* Set every population of fluid `fluid` (host [9][ny][nx] FP64). */
int lb_set_populations(lb_ctx *ctx, int fluid, const double *f);
/* Set every solute population (host [q][ny][nx] FP64). */
int lb_set_solute_populations(lb_ctx *ctx, const double *g);
/* Set the precipitate b of every node (host [ny][nx] FP64; only solid
 * nodes' values are used). */
int lb_set_precipitate(lb_ctx *ctx, const double *b);

/* ---- force fields ---------------------------------------------------- */

/* aveforce / aveacceleration commands: add value * e_mode (mode 0..8) to
 * the force per fluid node (or acceleration; force = rho a) of `fluid`.
 * The _xy forms add (fx, fy) directly. */
int lb_aveforce(lb_ctx *ctx, int mode, double value, int fluid);
int lb_aveforce_xy(lb_ctx *ctx, double fx, double fy, int fluid);
int lb_aveacceleration(lb_ctx *ctx, int mode, double value, int fluid);
int lb_aveacceleration_xy(lb_ctx *ctx, double ax, double ay, int fluid);

/* interforce command: one component F = -G psi(x) sum_i w_i psi(x+e_i) e_i
 * with psi = psi0 exp(-rho0/rho); two components F_s = -G rho_s(x)
 * sum_i w_i rho_sbar(x+e_i) e_i (psi0, rho0 ignored).  psi = 0 on solid
 * nodes.  With inlet/outlet openings the densities are those after the
 * opening rules of the same iteration, and the sums wrap periodically
 * across every wall, as the domain's boundaries do; not built for slabs
 * (LB_E_UNSUPPORTED at the first iteration). */
int lb_interforce(lb_ctx *ctx, double G, double psi0, double rho0);

/* adhesiveforce command: F = -G psi(x) sum_i w_i s(x+e_i) e_i, s = 1 on
 * solid nodes; one component psi = psi0 exp(-rho0/rho), two components
 * psi = rho_fluid. */
int lb_adhesiveforce(lb_ctx *ctx, double G, double psi0, double rho0,
                     int fluid);

/* intersolute command: interfaces for the solute.  The solute collision
 * relaxes to g_eq(C, u + tau_s F / C) with F = -G psi(x) sum_{i=1..4}
 * psi(x + e_i) e_i over the D2Q4 neighbours, psi = psi0 exp(-C0 / C) of
 * the concentrations after this step's streaming and opening rules (0 on
 * solid nodes and where C <= 0).  Needs lb_solute; adds one pass over the
 * solute lattice per iteration. */
int lb_intersolute(lb_ctx *ctx, double G, double psi0, double C0);

/* ---- output and action ----------------------------------------------- */

/* thermo command: evaluate the thermo record and the node fields every Nf
 * iterations (Nf > 0), or at the end of every lb_iteration call (Nf = 0,
 * the default).  Evaluating them reads the record back to the host, so it
 * synchronises the stream. */
int lb_thermo(lb_ctx *ctx, int Nf);

/* output command: produce the node fields (each component's density and
 * momentum j + F/2, read by lb_get_fields and lb_get_velocity_f32) every Nf
 * iterations (Nf > 0) without the thermo sums; Nf = 0 (the default) leaves
 * them to the thermo steps.  The paper's command prints them to a file;
 * here the caller reads them from the library.  No synchronisation. */
int lb_output(lb_ctx *ctx, int Nf);

/* Fluid kernel for single-component lattices without interforce:
 * "streaming" (one thread per node, loads straight from HBM; the fastest
 * on GB300), "tma" (a persistent kernel that streams 128 x 4 tiles into
 * shared memory with bulk asynchronous copies; same results bit for bit,
 * needs the width to be a multiple of 4 nodes for FP32 or 8 for 16-bit
 * storage), "fused" (with a solute and without intersolute or exact
 * momentum pairs: the fluid and the solute update in one kernel, the
 * solvent velocity kept in registers; same results bit for bit) or "auto"
 * (fused where it applies, else streaming; the default).  Other lattices
 * always use the streaming kernels.  A timed-out wait inside the TMA kernel
 * is reported as LB_E_TIMEOUT at the next thermo evaluation; a kernel that
 * does not apply to the setup fails the iteration with LB_E_UNSUPPORTED. */
int lb_set_kernel(lb_ctx *ctx, const char *name);

/* Clock cycles an mbarrier wait of the TMA kernel may take before the kernel
 * gives up (failure detection; the paper has no counterpart).  A wait that
 * runs out sets the context's error word; the CTA then lets the copies it
 * has already issued land (waiting up to the default limit, about two
 * seconds at 2 GHz) and returns, so no asynchronous copy is in flight when
 * it exits.  The next thermo evaluation returns LB_E_TIMEOUT and clears the
 * word; the state of that iteration is not valid (restore a snapshot).
 * cycles < 0 restores the default; 0 makes every CTA give up at its first
 * wait (a test of the give-up path).  Any time. */
int lb_set_wait_limit(lb_ctx *ctx, int64_t cycles);

/* Checking aid in place of a memory sanitizer: with LB_DEBUG_POISON set,
 * every iteration first fills the buffers it is about to write (the
 * populations and solute populations of the next state, the deposit
 * shares, the solvent-velocity and concentration planes, and on thermo or
 * output steps the node-field planes) with NaN bit patterns.  A kernel
 * that read a slot no kernel of the iteration wrote (a solid slot, a row
 * padding lane, a plane it does not own) would carry the NaN into the fluid
 * state, the exports or the thermo sums; with correct kernels the results
 * equal those of a run without the flag bit for bit.  Costs a memset of
 * those buffers per iteration; a batch with a poisoned member poisons its
 * population buffers before every launch and runs without its graph.
 * flags: any of LB_DEBUG_POISON and LB_DEBUG_GUARDS. */
#define LB_DEBUG_POISON 0x1
/* LB_DEBUG_GUARDS: every device buffer the library allocates after the
 * flag is set (set it before the first iteration or state upload) gets a
 * 256 KB zone of NaN bit patterns on each side.  A read past a buffer's
 * end (or before its start) within that distance carries NaN into the
 * results; lb_debug_check counts the guard bytes that no longer hold the
 * pattern (a write out of bounds) into *bad.  Buffers bound with lb_bind
 * have no guards. */
#define LB_DEBUG_GUARDS 0x2
int lb_set_debug(lb_ctx *ctx, int flags);
int lb_debug_check(lb_ctx *ctx, int64_t *bad);

/* iteration command: advance Nt iterations.  The first call validates the
 * setup (LB_E_ARG with a message if it is inconsistent) and moves the
 * state to the GPU.  Returns LB_E_NAN if a thermo sum is not finite. */
int lb_iteration(lb_ctx *ctx, int Nt);

/* Thermo record of the last thermo evaluation. */
int lb_get_thermo(lb_ctx *ctx, lb_thermo_t *out);

/* Thermo evaluations that do not stop the host (no counterpart in the
 * paper, whose thermo command prints at once).  By default (on = 0) every
 * thermo evaluation copies its record to the host and waits for it, so
 * lb_iteration returns LB_E_NAN or LB_E_TIMEOUT from the iteration that
 * found it.  With on = 1 the record is copied, in stream order, to
 * page-locked host memory of the context (allocated by the first such
 * call) and read later, without the host waiting for the GPU to catch up:
 * by the next thermo evaluation before it runs (the record is then a
 * thermo interval old), by lb_get_thermo and lb_thermo_static, and by
 * lb_thermo_deferred(ctx, 0).  Those calls then return the record's
 * LB_E_NAN or LB_E_TIMEOUT: the error of a thermo step reaches the caller
 * with the next of them, after the iterations queued since have run.  The
 * records and the thermo kernel are the same in both modes, bit for bit.
 * LB_E_ARG unless on is 0 or 1. */
int lb_thermo_deferred(lb_ctx *ctx, int on);

/* Recompute the thermo record of the context's last thermo evaluation
 * without allocating anything.  The paper has no counterpart: this is for
 * callers that cannot let the library allocate device memory -- when a
 * framework's caching allocator already holds the free device memory, when
 * a loop cannot afford an allocation or the device-wide synchronisation a
 * cudaFree may imply, or when a program forbids allocation after start-up.
 * The FP64 partial sums go to one fixed device array of the library (room
 * for 1024 blocks of partial sums, 131,220 bytes, kept by every GPU that
 * loads the library until the process exits) instead of a buffer of the
 * context; the result is the same, bit for bit, as lb_get_thermo's.
 * Inputs: ctx (its fields, mask and deposits on the device); output: *out
 * (host).  The thermo kernel takes one block per lattice row, at most four
 * per SM, so the array serves every lattice on GPUs of up to 256 SMs;
 * a lattice that would need more than 1024 blocks gets LB_E_ARG.  Returns
 * LB_E_ORDER unless the last iteration executed ended with a thermo step
 * and no state was replaced since (lb_set_populations, lb_set_equilibrium,
 * lb_set_solute_*, lb_set_precipitate, lb_load_state, lb_set_step): the
 * field planes then describe the live mask and deposits the kernel also
 * reads.  Returns LB_E_TIMEOUT, like lb_iteration, if a TMA pipeline wait
 * gave up.  Synchronises ctx's stream.  The first call on a device looks up the
 * array's device address (once per device, with that device current);
 * make that first call before any stream capture.  All calls share the
 * one array: calls whose kernels overlap on a GPU (different streams,
 * contexts or threads) race and must be serialised by the caller.  Every
 * value the kernels read is written earlier in the same call, so what a
 * previous call left in the array does not matter. */
int lb_thermo_static(lb_ctx *ctx, lb_thermo_t *out);

/* Node fields of the last thermo evaluation for fluid `fluid` (host
 * [ny][nx] FP64, any pointer may be NULL): density, physical momentum
 * density j + F/2 and equilibrium density; zero on solid nodes. */
int lb_get_fields(lb_ctx *ctx, int fluid, double *rho, double *px,
                  double *py, double *rho_eq);
/* Total density and solvent velocity u = sum(j + F/2)/sum(rho) (Eq. (4))
 * of the last thermo evaluation as FP32 host [ny][nx] arrays (zero on
 * solid nodes).  Page-locked outputs (cudaHostAlloc, or pinned torch
 * tensors) are written by the export kernel directly; other host memory
 * through a staging buffer and copies.  Synchronises the stream. */
int lb_get_velocity_f32(lb_ctx *ctx, float *rho, float *ux, float *uy);
/* Current populations of fluid `fluid` (host [9][ny][nx] FP64). */
int lb_get_populations(lb_ctx *ctx, int fluid, double *f);
/* Current solute populations (host [q][ny][nx]), concentration of the
 * last thermo evaluation and current precipitate (host [ny][nx]); NULL
 * skips. */
int lb_get_solute(lb_ctx *ctx, double *g, double *C, double *b);
/* Solid mask (host [ny][nx] bytes, 1 = solid). */
int lb_get_mask(lb_ctx *ctx, uint8_t *mask);
/* Set the count of iterations done to t >= 0 (any time).  The growth
 * rule's random pick (seed and step, App. C) and the thermo schedule read
 * it, so a state taken from another run at step t (with lb_set_populations,
 * lb_set_solute_populations, lb_set_precipitate) continues with that run's
 * decisions.  Called with t > 0 before the device state exists, it also
 * admits a geometry that growth has made: fluid nodes with reactive links
 * on two opposite sides, which a fresh lb_surface_reaction setup refuses
 * (App. C rule 1), each link then taking the link rule on its own. */
int lb_set_step(lb_ctx *ctx, int64_t t);
/* Nodes that surface growth turned solid in the last iteration executed
 * (the last of the Nt steps of lb_iteration; growth rule of App. C):
 * *count = their number, and the first min(count, cap) node indices
 * y*nx + x, ascending, go to idx (cap = 0 with idx = NULL only counts).
 * Without surface_reaction, before the first iteration and right after
 * lb_load_state, *count = 0.  Synchronises the context's stream. */
int lb_get_flips(lb_ctx *ctx, int64_t *idx, int cap, int *count);

/* ---- caller-owned device buffers ------------------------------------- */

/* The state buffers a caller may supply instead of the library allocating
 * them, by name:
 *   "f0", "f1"  the two population buffers, [nc][9][ny][pitch] elements of
 *               the storage type (FP32, or binary16 / bfloat16), each the
 *               deviation h_i = f_i - s_i rho_ref of Eq. (2)'s rest state
 *               (rho_ref as lb_set_storage holds it, rounded to FP32;
 *               times 2^s for FP16); pitch = nx rounded up to 32; slots of
 *               solid nodes and past nx are unspecified
 *   "g0", "g1"  the two solute population buffers, [q][ny][pitch] FP32
 *   "fields"    node fields of the last thermo step, [nc][4][ny][pitch]
 *               FP32: rho - rho_ref, the physical momentum x and y
 *               (j + F/2, Eq. (4)), sum of the equilibrium deviations
 *   "u"         solvent velocity of the last step (with lb_solute),
 *               [2][ny][pitch] FP32 (the fused kernel writes it only
 *               when it is bound)
 * lb_buffer_size gives the bytes the current setup needs (0 for "u" without
 * lb_solute).  lb_bind, after lb_lattice and before the first iteration,
 * makes the library use dev (device memory of the context's device, 256-byte
 * aligned, at least that many bytes) for the named buffer; dev = NULL
 * unbinds.  The library zeroes and writes it but never frees it; the caller
 * keeps it alive until lb_destroy.  A setup changed after binding
 * (storage, fluids, solute) is checked against the bound size when the
 * device state is created (first iteration or state upload: LB_E_ARG).  lb_current_buffer gives k such that f<k>
 * and g<k> hold the current state (it alternates every iteration). */
int lb_buffer_size(lb_ctx *ctx, const char *what, size_t *bytes);
int lb_bind(lb_ctx *ctx, const char *what, void *dev, size_t bytes);
int lb_current_buffer(lb_ctx *ctx, int *index);

/* Raw state snapshot (checkpoint/resume): populations in their storage
 * format, mask, solute, step counter and, with surface_reaction, the
 * precipitate, removed-mass tallies and flip count.  lb_state_size gives the byte count; save/load copy to/from a
 * host buffer of that size (pinned memory gives full copy bandwidth).
 * Loading a snapshot of the same setup resumes bit for bit. */
int lb_state_size(lb_ctx *ctx, size_t *bytes);
int lb_save_state(lb_ctx *ctx, void *host, size_t bytes);
int lb_load_state(lb_ctx *ctx, const void *host, size_t bytes);

/* ---- input-data and restart text files ------------------------------- */

/* write_restart command (Sec. Commands, write_restart; the file layout is
 * the input-data format of the read_data command): after every iteration
 * whose step t is a multiple of Nf, lb_iteration writes the state as text
 * files named "<file>.<t>" (one fluid), "<file>.<t>.fluid1" and
 * "<file>.<t>.fluid2" (two fluids) and "<file>.<t>.solute" (solute).  A
 * fluid file holds the sections relaxation_time (tau; with two fluids also
 * the density-ratio alpha), domain
 * (Nx Ny: sites 0..Nx, 0..Ny), processors, inlet/outlet (wall x0 x1 label
 * style arguments), boundary, field (force/acceleration as e1/e2 values,
 * interforce, adhesiveforce), density (x y rho style; rho = -11 on solid
 * sites) and momentum (x y f0 .. f8, the full populations, zero on solid
 * sites); a solute file holds relaxation_time, inlet/outlet, reaction
 * (surface kr Cs growth bmax b0 seed), field (intersolute), concentration
 * (x y C [b]) and solute_modes (x y g_1 .. g_q).  Numbers are written with
 * 17 significant digits.  As in the paper, the command precedes the
 * iteration command (LB_E_ORDER once an iteration has run, except Nf = 0,
 * which stops writing).  file is copied.  Errors: LB_E_ARG (Nf < 0,
 * no name; a file that cannot be written is reported by lb_iteration),
 * LB_E_ORDER, LB_E_UNSUPPORTED (a slab). */
int lb_write_restart(lb_ctx *ctx, const char *file, int Nf);
/* The same files for the current state, now, named "<file>" (one fluid),
 * "<file>.fluid1"/".fluid2" and "<file>.solute".  Errors: LB_E_ORDER (no
 * device state yet), LB_E_ARG (cannot write), LB_E_UNSUPPORTED (a slab). */
int lb_write_data(lb_ctx *ctx, const char *file);
/* read_data command (Sec. Commands, read_data): sets up the lattice from
 * input-data files before the first iteration.  args: NULL or a comma- or
 * space-separated subset of "fluids" (two fluids: read "<file>.fluid1" and
 * "<file>.fluid2" instead of "<file>"), "solute" (also read
 * "<file>.solute") and "equilibrium" (start from the equilibrium of the
 * densities and velocities read instead of the populations).  The sections
 * may come in any order but domain before processors, field after
 * relaxation_time, processors before density and momentum, boundary before
 * density, reaction before concentration.  A domain section (re)defines
 * the lattice (as lb_lattice; its relaxation time from the file); the
 * density section's solid sites replace the mask; openings listed are added
 * (or, where an opening already lies at the same place, relabelled) and
 * given their styles; force/acceleration items add to the body forces,
 * interforce/adhesiveforce/intersolute/reaction items set them; the state
 * read is applied when the device state is created (a later
 * position0/momentum0/concentration0 replaces it).  Every site must be
 * listed in density and, when present, momentum, concentration and
 * solute_modes; a file without a momentum (solute_modes) section starts at
 * the equilibrium of its densities (concentrations) at rest.  Errors:
 * LB_E_ARG (unreadable file, a malformed or misplaced section or line, with
 * the file and line in lb_last_error), LB_E_ORDER (after the first
 * iteration; no domain section and no lattice), LB_E_UNSUPPORTED (a slab),
 * and those of the commands it applies. */
int lb_read_data(lb_ctx *ctx, const char *file, const char *args);
/* The lattice as the commands (or read_data) have set it up: nodes nx x ny,
 * fluid components, solute lattice (0 none, 4 or 9), processor grid.  Any
 * output pointer may be NULL.  Errors: LB_E_ORDER (no lattice yet). */
int lb_lattice_info(lb_ctx *ctx, int *nx, int *ny, int *ncomp, int *q, int *px, int *py);

/* ---- batched lattices ------------------------------------------------ */

/* Group n committed single-component contexts of one device and stream
 * (periodic, no openings, no solute, same storage) so that lb_batch_iteration
 * advances all of them with one kernel launch per iteration.  The contexts
 * stay owned by the caller and must outlive the batch. */
int lb_batch_create(lb_ctx *const *ctxs, int n, lb_batch **out);
int lb_batch_destroy(lb_batch *b);
/* Advance every lattice of the batch Nt iterations; use_graph != 0
 * captures the launches in a CUDA graph and replays it. */
int lb_batch_iteration(lb_batch *b, int Nt, int use_graph);
/* Time the candidate tile shapes and work schedules and keep the fastest;
 * cache_json (may be NULL) is a file that stores the choice keyed by
 * device, shapes and storage. */
int lb_batch_autotune(lb_batch *b, const char *cache_json);
const char *lb_batch_last_error(const lb_batch *b);
/* Number of kernels the batch has launched (graph replays count their
 * kernel nodes). */
int lb_batch_launch_count(const lb_batch *b, uint64_t *out);

#ifdef __cplusplus
}
#endif
#endif
