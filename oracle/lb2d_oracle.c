/*
 * lb2d_oracle.c -- FP64 CPU oracle for the lattice Boltzmann update of
 * arXiv:1202.0442 ("Introduction to Perl module lb2d.pm 0.1").
 *
 * TEST INFRASTRUCTURE ONLY: the checker the GPU library is compared
 * against.  Nothing in the product path links or calls this file.
 *
 * The method is a time-stepping scheme with no shortcut, so the oracle is
 * the algorithm itself, one plain loop per step, in the order of Fig. 1 of
 * the paper (initial populations -> [stream with boundary handling ->
 * equilibrium -> collision] repeated), with the extra steps of the command
 * descriptions placed where those descriptions put them:
 *
 *   1. streaming with half-way bounce-back at solid nodes (Fig. 1, Eq. (1),
 *      boundary_style noslip)
 *   2. inlet/outlet openings after streaming (inlet_momentum/outlet_momentum
 *      commands, App. A)
 *   3. moments rho, j (Sec. Model and algorithm)
 *   4. forces: aveforce, aveacceleration, interforce, adhesiveforce
 *   5. equilibrium velocity (velocity-shift forcing; fluids command for two
 *      components) and 6. BGK collision with Eq. (2) / the fluids-command
 *      equilibrium
 *   7. gradient openings after collision (inlet_momentum/outlet_momentum)
 *   8. node fields: density and physical momentum j + F/2 (Eq. (4), output
 *      command)
 *   9. solute on D2Q4 (solute command, Eq. (3)) or D2Q9: streaming,
 *      bounce-back or surface reaction (surface_reaction command, App. C),
 *      inlet_solute/outlet_solute rules (dirichlet, adiabatic, flux;
 *      App. B), BGK collision, with the intersolute force in the
 *      equilibrium velocity
 *  10. precipitation after collision and 11. surface growth
 *      (surface_reaction command, App. C)
 *  12. thermo sums over the final state (thermo command)
 *
 * Everything is FP64, single-threaded, unblocked.  Arrays are AoS inside
 * (population i of node n at [n*Q + i]); the interface is SoA.
 *
 * Readings where the paper is silent or ambiguous (each one is listed in
 * the design notes of the repository):
 *   - D2Q9 numbering e1=(1,0) e2=(0,1) e3=(-1,0) e4=(0,-1) e5=(1,1)
 *     e6=(-1,1) e7=(-1,-1) e8=(1,-1), as the unknown sets of the opening
 *     rules require; D2Q4 g1..g4 = +x,+y,-x,-y.
 *   - all domain edges wrap periodically; on an opening node the modes that
 *     cross the opening's wall are replaced by the opening rule.
 *   - forcing by velocity shift u_eq = u + tau F / rho; physical momentum
 *     j + F/2 (Eq. (4)).
 *   - Shan-Chen sums use the D2Q9 weights and take psi = 0 on solid nodes;
 *     neighbour densities are those of the same step after streaming.
 *   - surface reaction on link i: C_i = (2 g_out + kr Cs)/(kr + 2 w_i),
 *     g_in = -g_out + 2 w_i C_i (w_i = 1/4 on D2Q4 gives App. C exactly);
 *     the node concentration used by the collision is the sum of the
 *     populations; the wall concentration is the mean of the C_i.
 *   - precipitation dB = kr (C_w - Cs) if > 0, taken in equal parts from
 *     the incoming modes after collision and credited in equal parts to
 *     the solid nodes behind them.
 *   - solute flux openings: C1 is the inner neighbour's concentration
 *     right after streaming (before its own opening rule); intersolute
 *     uses the concentrations after streaming and the opening rules of the
 *     same step, psi = 0 on solid nodes and where C <= 0.
 *   - growth: a solid node with b > bmax turns one fluid 4-neighbour (not
 *     an opening node) to solid; the choice is SplitMix64(seed ^ (t*nx*ny
 *     + node)) mod (number of candidates), candidates in the order
 *     +x, +y, -x, -y; all decisions use the state before any flip.
 */
#include "lb2d_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* D2Q9 velocity set and weights (Eq. (2) and the text below it). */
static const int EX9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W9[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                             1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int OPP9[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

/* index of the D2Q9 direction (ex, ey) */
static int dir9(int ex, int ey) {
  for (int i = 0; i < 9; i++)
    if (EX9[i] == ex && EY9[i] == ey) return i;
  return -1;
}

/* D2Q4 solute lattice (solute command): g1=+x, g2=+y, g3=-x, g4=-y at
 * storage index 0..3. */
static const int EX4[4] = {1, 0, -1, 0};
static const int EY4[4] = {0, 1, 0, -1};
static const double W4[4] = {0.25, 0.25, 0.25, 0.25};
static const int OPP4[4] = {2, 3, 0, 1};

#define MAXOPEN 16

typedef struct {
  int wall, a0, a1, kind;
  int style[2];
  double v[2], rho[2];
  int sstyle;
  double Cbar, sv;
} opening_t;

struct orc {
  int nx, ny, nc, qs;
  long t;
  double tau[2], alpha[2], taus;
  uint8_t *solid;
  double *f[2], *ft[2];
  double *rho[2], *jx[2], *jy[2], *Fx[2], *Fy[2];
  double *px[2], *py[2], *meq[2];
  double fave[2][2], acc[2][2];
  int sc_on;
  double G, psi0, rho0;
  int ads_on[2];
  double Gads[2], ads_psi0[2], ads_rho0[2];
  int nopen;
  opening_t op[MAXOPEN];
  int *open_id;
  double *g, *gt, *C, *b, *db, *Cw;
  double *Cst, *Cpre; /* solute: C after streaming; after the opening rules */
  double slipR[2];    /* boundary_style slip/mixed: R of every solid node */
  double *Rmap[2];    /* hybrid: R per node (NULL: slipR) */
  int is_on;          /* intersolute */
  double isG, ispsi0, isC0;
  int *nU, *Ubits;
  int react_on;
  double kr, Cs, b0, bmax;
  uint64_t seed;
  uint8_t *flip;
  double removed[2], removed_solute;
  long nflips_last;
  /* growth decisions taken within margin_eps * bmax of the threshold in
   * the last iteration (trigger node, b - bmax) */
  double margin_eps;
  int nmargin, capmargin;
  int64_t *margin_node;
  double *margin_val;
  double thermo[ORC_T_COUNT];
};

static int wrap(int a, int n) { return ((a % n) + n) % n; }

/* ------------------------------------------------------------------ */
/* creation and state access                                           */
/* ------------------------------------------------------------------ */

orc_t *orc_create(int nx, int ny, int ncomp, int solute_q) {
  if (nx < 1 || ny < 1 || (ncomp != 1 && ncomp != 2)) return NULL;
  if (solute_q != 0 && solute_q != 4 && solute_q != 9) return NULL;
  orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
  if (!o) return NULL;
  size_t nn = (size_t)nx * ny;
  o->nx = nx;
  o->ny = ny;
  o->nc = ncomp;
  o->qs = solute_q;
  for (int s = 0; s < 2; s++) {
    o->tau[s] = 1.0;
    o->alpha[s] = 4.0 / 9.0;
  }
  o->taus = 1.0;
  o->solid = (uint8_t *)calloc(nn, 1);
  o->open_id = (int *)malloc(nn * sizeof(int));
  o->flip = (uint8_t *)calloc(nn, 1);
  for (size_t n = 0; n < nn; n++) o->open_id[n] = -1;
  for (int s = 0; s < ncomp; s++) {
    o->f[s] = (double *)calloc(nn * 9, sizeof(double));
    o->ft[s] = (double *)calloc(nn * 9, sizeof(double));
    o->rho[s] = (double *)calloc(nn, sizeof(double));
    o->jx[s] = (double *)calloc(nn, sizeof(double));
    o->jy[s] = (double *)calloc(nn, sizeof(double));
    o->Fx[s] = (double *)calloc(nn, sizeof(double));
    o->Fy[s] = (double *)calloc(nn, sizeof(double));
    o->px[s] = (double *)calloc(nn, sizeof(double));
    o->py[s] = (double *)calloc(nn, sizeof(double));
    o->meq[s] = (double *)calloc(nn, sizeof(double));
  }
  if (solute_q) {
    o->g = (double *)calloc(nn * solute_q, sizeof(double));
    o->gt = (double *)calloc(nn * solute_q, sizeof(double));
    o->C = (double *)calloc(nn, sizeof(double));
    o->db = (double *)calloc(nn, sizeof(double));
    o->Cw = (double *)calloc(nn, sizeof(double));
    o->Cst = (double *)calloc(nn, sizeof(double));
    o->Cpre = (double *)calloc(nn, sizeof(double));
    o->nU = (int *)calloc(nn, sizeof(int));
    o->Ubits = (int *)calloc(nn, sizeof(int));
  }
  o->b = (double *)calloc(nn, sizeof(double));
  return o;
}

void orc_destroy(orc_t *o) {
  if (!o) return;
  for (int s = 0; s < o->nc; s++) {
    free(o->f[s]); free(o->ft[s]); free(o->rho[s]); free(o->jx[s]);
    free(o->jy[s]); free(o->Fx[s]); free(o->Fy[s]); free(o->px[s]);
    free(o->py[s]); free(o->meq[s]);
  }
  free(o->g); free(o->gt); free(o->C); free(o->db); free(o->b);
  free(o->Cw); free(o->nU); free(o->Ubits);
  free(o->Cst); free(o->Cpre);
  free(o->margin_node); free(o->margin_val);
  free(o->Rmap[0]); free(o->Rmap[1]);
  free(o->solid); free(o->open_id); free(o->flip);
  free(o);
}

int orc_set_tau(orc_t *o, int comp, double tau) {
  if (comp < 0 || comp >= o->nc || !(tau > 0.5)) return -1;
  o->tau[comp] = tau;
  return 0;
}

int orc_set_alpha(orc_t *o, int comp, double alpha) {
  if (comp < 0 || comp >= o->nc) return -1;
  o->alpha[comp] = alpha;
  return 0;
}

int orc_set_taus(orc_t *o, double taus) {
  if (!(taus > 0.5)) return -1;
  o->taus = taus;
  return 0;
}

int orc_set_solid(orc_t *o, const uint8_t *mask) {
  size_t nn = (size_t)o->nx * o->ny;
  for (size_t n = 0; n < nn; n++) o->solid[n] = mask[n] ? 1 : 0;
  return 0;
}

int orc_get_solid(const orc_t *o, uint8_t *mask) {
  memcpy(mask, o->solid, (size_t)o->nx * o->ny);
  return 0;
}

static int set_pops(double *dst, const double *src, int q, size_t nn) {
  for (int i = 0; i < q; i++)
    for (size_t n = 0; n < nn; n++) dst[n * q + i] = src[i * nn + n];
  return 0;
}

static int get_pops(const double *src, double *dst, int q, size_t nn) {
  for (int i = 0; i < q; i++)
    for (size_t n = 0; n < nn; n++) dst[i * nn + n] = src[n * q + i];
  return 0;
}

int orc_set_f(orc_t *o, int comp, const double *f) {
  if (comp < 0 || comp >= o->nc) return -1;
  return set_pops(o->f[comp], f, 9, (size_t)o->nx * o->ny);
}

int orc_get_f(const orc_t *o, int comp, double *f) {
  if (comp < 0 || comp >= o->nc) return -1;
  return get_pops(o->f[comp], f, 9, (size_t)o->nx * o->ny);
}

int orc_set_g(orc_t *o, const double *g) {
  if (!o->qs) return -1;
  return set_pops(o->g, g, o->qs, (size_t)o->nx * o->ny);
}

int orc_get_g(const orc_t *o, double *g) {
  if (!o->qs) return -1;
  return get_pops(o->g, g, o->qs, (size_t)o->nx * o->ny);
}

int orc_set_b(orc_t *o, const double *b) {
  memcpy(o->b, b, (size_t)o->nx * o->ny * sizeof(double));
  return 0;
}

int orc_get_b(const orc_t *o, double *b) {
  memcpy(b, o->b, (size_t)o->nx * o->ny * sizeof(double));
  return 0;
}

/* ------------------------------------------------------------------ */
/* equilibria                                                          */
/* ------------------------------------------------------------------ */

/* Eq. (2) generalised by the fluids command:
 * f_i^eq = w_i rho [A_i + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u],
 * A_0 = (9/4) alpha, A_{1..8} = (9/5)(1 - alpha); alpha = 4/9 gives
 * A_i = 1, i.e. Eq. (2) with c_s^2 = 1/3. */
void orc_feq(double rho, double ux, double uy, double alpha, double *feq) {
  double uu = ux * ux + uy * uy;
  for (int i = 0; i < 9; i++) {
    double A = (i == 0) ? 2.25 * alpha : 1.8 * (1.0 - alpha);
    double eu = EX9[i] * ux + EY9[i] * uy;
    feq[i] = W9[i] * rho * (A + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
  }
}

int orc_set_equilibrium(orc_t *o, int comp, const double *rho,
                        const double *ux, const double *uy) {
  if (comp < 0 || comp >= o->nc) return -1;
  size_t nn = (size_t)o->nx * o->ny;
  for (size_t n = 0; n < nn; n++) {
    double feq[9];
    if (o->solid[n]) {
      for (int i = 0; i < 9; i++) o->f[comp][n * 9 + i] = 0.0;
      continue;
    }
    orc_feq(rho[n], ux[n], uy[n], o->alpha[comp], feq);
    for (int i = 0; i < 9; i++) o->f[comp][n * 9 + i] = feq[i];
  }
  return 0;
}

/* Eq. (3) on D2Q4: g_i^eq = C/4 [1 + 2 e_i.u]; on D2Q9 the same linear
 * advection-diffusion equilibrium with the D2Q9 weights and c_s^2 = 1/3:
 * g_i^eq = w_i C [1 + 3 e_i.u]. */
/* solvent velocity of Eq. (4) at node n: sum of the physical momenta
 * (j + F/2) over the sum of the densities of the fluid components */
static void solvent_velocity(const orc_t *o, size_t n, double *u) {
  double rs = 0.0, pxs = 0.0, pys = 0.0;
  for (int s = 0; s < o->nc; s++) {
    rs += o->rho[s][n];
    pxs += o->px[s][n];
    pys += o->py[s][n];
  }
  u[0] = pxs / rs;
  u[1] = pys / rs;
}

static void solute_geq(int q, double C, double ux, double uy, double *geq) {
  if (q == 4) {
    for (int i = 0; i < 4; i++)
      geq[i] = 0.25 * C * (1.0 + 2.0 * (EX4[i] * ux + EY4[i] * uy));
  } else {
    for (int i = 0; i < 9; i++)
      geq[i] = W9[i] * C * (1.0 + 3.0 * (EX9[i] * ux + EY9[i] * uy));
  }
}

int orc_set_solute_equilibrium(orc_t *o, const double *C, const double *ux,
                               const double *uy) {
  if (!o->qs) return -1;
  size_t nn = (size_t)o->nx * o->ny;
  for (size_t n = 0; n < nn; n++) {
    double geq[9];
    if (o->solid[n]) {
      for (int i = 0; i < o->qs; i++) o->g[n * o->qs + i] = 0.0;
      continue;
    }
    solute_geq(o->qs, C[n], ux[n], uy[n], geq);
    for (int i = 0; i < o->qs; i++) o->g[n * o->qs + i] = geq[i];
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* commands                                                            */
/* ------------------------------------------------------------------ */

int orc_set_aveforce(orc_t *o, int comp, double fx, double fy) {
  if (comp < 0 || comp >= o->nc) return -1;
  o->fave[comp][0] = fx;
  o->fave[comp][1] = fy;
  return 0;
}

int orc_set_aveacceleration(orc_t *o, int comp, double ax, double ay) {
  if (comp < 0 || comp >= o->nc) return -1;
  o->acc[comp][0] = ax;
  o->acc[comp][1] = ay;
  return 0;
}

int orc_set_interforce(orc_t *o, double G, double psi0, double rho0) {
  o->sc_on = (G != 0.0);
  o->G = G;
  o->psi0 = psi0;
  o->rho0 = rho0;
  return 0;
}

int orc_set_adhesiveforce(orc_t *o, int comp, double G, double psi0,
                          double rho0) {
  if (comp < 0 || comp >= o->nc) return -1;
  o->ads_on[comp] = (G != 0.0);
  o->Gads[comp] = G;
  o->ads_psi0[comp] = psi0;
  o->ads_rho0[comp] = rho0;
  return 0;
}

int orc_set_slip(orc_t *o, int comp, double R_all, const double *R_map) {
  if (comp < 0 || comp >= o->nc || R_all < 0.0 || R_all > 1.0) return -1;
  size_t nn = (size_t)o->nx * o->ny;
  o->slipR[comp] = R_all;
  free(o->Rmap[comp]);
  o->Rmap[comp] = NULL;
  if (R_map) {
    o->Rmap[comp] = (double *)calloc(nn, sizeof(double));
    for (size_t n = 0; n < nn; n++)
      o->Rmap[comp][n] = o->solid[n] ? R_map[n] : 0.0;
  }
  return 0;
}

/* inlet/outlet commands: an opening spans coordinates a0..a1 along its
 * wall (y for xlo/xhi, x for ylo/yhi). */
int orc_add_opening(orc_t *o, int wall, int a0, int a1, int kind) {
  if (o->nopen >= MAXOPEN || wall < 0 || wall > 3 || a0 > a1) return -1;
  int len = (wall <= ORC_XHI) ? o->ny : o->nx;
  if (a0 < 0 || a1 >= len) return -1;
  int id = o->nopen;
  for (int a = a0; a <= a1; a++) {
    int x, y;
    if (wall == ORC_XLO) { x = 0; y = a; }
    else if (wall == ORC_XHI) { x = o->nx - 1; y = a; }
    else if (wall == ORC_YLO) { x = a; y = 0; }
    else { x = a; y = o->ny - 1; }
    if (o->open_id[y * o->nx + x] >= 0) return -1;
  }
  for (int a = a0; a <= a1; a++) {
    int x, y;
    if (wall == ORC_XLO) { x = 0; y = a; }
    else if (wall == ORC_XHI) { x = o->nx - 1; y = a; }
    else if (wall == ORC_YLO) { x = a; y = 0; }
    else { x = a; y = o->ny - 1; }
    o->open_id[y * o->nx + x] = id;
  }
  opening_t *p = &o->op[id];
  memset(p, 0, sizeof(*p));
  p->wall = wall;
  p->a0 = a0;
  p->a1 = a1;
  p->kind = kind;
  o->nopen++;
  return id;
}

int orc_set_opening_momentum(orc_t *o, int opening, int comp, int style,
                             double v, double rho) {
  if (opening < 0 || opening >= o->nopen || comp < 0 || comp >= o->nc)
    return -1;
  o->op[opening].style[comp] = style;
  o->op[opening].v[comp] = v;
  o->op[opening].rho[comp] = rho;
  return 0;
}

int orc_set_opening_solute(orc_t *o, int opening, int style, double Cbar,
                           double v) {
  if (opening < 0 || opening >= o->nopen) return -1;
  o->op[opening].sstyle = style;
  o->op[opening].Cbar = Cbar;
  o->op[opening].sv = v;
  return 0;
}

int orc_set_intersolute(orc_t *o, double G, double psi0, double C0) {
  if (!o->qs) return -1;
  o->is_on = 1;
  o->isG = G;
  o->ispsi0 = psi0;
  o->isC0 = C0;
  return 0;
}

int orc_set_reaction(orc_t *o, double kr, double Cs, double b0, double bmax,
                     uint64_t seed) {
  if (!o->qs) return -1;
  o->react_on = 1;
  o->kr = kr;
  o->Cs = Cs;
  o->b0 = b0;
  o->bmax = bmax;
  o->seed = seed;
  return 0;
}

long orc_time(const orc_t *o) { return o->t; }

/* the step counter (a run resumed from a restart file continues its count) */
int orc_set_time(orc_t *o, long t) {
  if (t < 0) return -1;
  o->t = t;
  return 0;
}

/* ------------------------------------------------------------------ */
/* inlet/outlet rules (inlet_momentum/outlet_momentum commands, App. A) */
/* ------------------------------------------------------------------ */

/* Poiseuille inlet profile (inlet_momentum command):
 * v(y) = 4 vmax/(y1-y0+1)^2 [((y1-y0+1)/2)^2 - ((2y-y1-y0)/2)^2]. */
double orc_poiseuille_v(double vmax, int a0, int a1, int coord) {
  double L = (double)(a1 - a0 + 1);
  double h = 0.5 * L;
  double d = 0.5 * (double)(2 * coord - a1 - a0);
  return 4.0 * vmax / (L * L) * (h * h - d * d);
}

/* Zou-He rules, written wall by wall as printed.  f holds the populations
 * after streaming and bounce-back; the three modes that crossed the wall
 * are overwritten.  Velocity styles: v is the imposed speed, positive into
 * the domain for an inlet and out of it for an outlet; returns the node
 * density in *out_rho.  Dirichlet: rho is imposed; returns the signed
 * velocity component normal to the wall (+x or +y) in *out_v. */
int orc_zouhe(int wall, int kind, int style, double v, double rho,
              double *f, double *out_rho, double *out_v) {
  double r, vx;
  if (style == ORC_M_POISEUILLE || style == ORC_M_UNIFORM) {
    if (kind == ORC_INLET) {
      switch (wall) {
        case ORC_XLO: /* inlet_momentum command, main text */
          r = (f[0] + f[2] + f[4] + 2.0 * (f[3] + f[6] + f[7])) / (1.0 - v);
          f[1] = f[3] + 2.0 / 3.0 * r * v;
          f[5] = f[7] - 0.5 * (f[2] - f[4]) + 1.0 / 6.0 * r * v;
          f[8] = f[6] + 0.5 * (f[2] - f[4]) + 1.0 / 6.0 * r * v;
          break;
        case ORC_XHI: /* App. A, inlet, xhi */
          r = (f[0] + f[2] + f[4] + 2.0 * (f[1] + f[5] + f[8])) / (1.0 - v);
          f[3] = f[1] + 2.0 / 3.0 * r * v;
          f[6] = f[8] + 0.5 * (f[4] - f[2]) + 1.0 / 6.0 * r * v;
          f[7] = f[5] - 0.5 * (f[4] - f[2]) + 1.0 / 6.0 * r * v;
          break;
        case ORC_YHI: /* App. A, inlet, yhi */
          r = (f[0] + f[1] + f[3] + 2.0 * (f[2] + f[5] + f[6])) / (1.0 - v);
          f[4] = f[2] + 2.0 / 3.0 * r * v;
          f[7] = f[5] + 0.5 * (f[1] - f[3]) + 1.0 / 6.0 * r * v;
          f[8] = f[6] - 0.5 * (f[1] - f[3]) + 1.0 / 6.0 * r * v;
          break;
        case ORC_YLO: /* App. A, inlet, ylo */
          r = (f[0] + f[1] + f[3] + 2.0 * (f[4] + f[7] + f[8])) / (1.0 - v);
          f[2] = f[4] + 2.0 / 3.0 * r * v;
          f[5] = f[7] + 0.5 * (f[3] - f[1]) + 1.0 / 6.0 * r * v;
          f[6] = f[8] - 0.5 * (f[3] - f[1]) + 1.0 / 6.0 * r * v;
          break;
        default:
          return -1;
      }
    } else {
      switch (wall) {
        case ORC_XHI: /* App. A, outlet, xhi */
          r = (f[0] + f[2] + f[4] + 2.0 * (f[1] + f[5] + f[8])) / (1.0 + v);
          f[3] = f[1] - 2.0 / 3.0 * r * v;
          f[6] = f[8] + 0.5 * (f[4] - f[2]) - 1.0 / 6.0 * r * v;
          f[7] = f[5] - 0.5 * (f[4] - f[2]) - 1.0 / 6.0 * r * v;
          break;
        case ORC_XLO: /* App. A, outlet, xlo */
          r = (f[0] + f[2] + f[4] + 2.0 * (f[3] + f[6] + f[7])) / (1.0 + v);
          f[1] = f[3] - 2.0 / 3.0 * r * v;
          f[5] = f[7] - 0.5 * (f[2] - f[4]) - 1.0 / 6.0 * r * v;
          f[8] = f[6] + 0.5 * (f[2] - f[4]) - 1.0 / 6.0 * r * v;
          break;
        case ORC_YHI: /* App. A, outlet, yhi */
          r = (f[0] + f[1] + f[3] + 2.0 * (f[2] + f[5] + f[6])) / (1.0 + v);
          f[4] = f[2] - 2.0 / 3.0 * r * v;
          f[7] = f[5] + 0.5 * (f[1] - f[3]) - 1.0 / 6.0 * r * v;
          f[8] = f[6] - 0.5 * (f[1] - f[3]) - 1.0 / 6.0 * r * v;
          break;
        case ORC_YLO: /* App. A, outlet, ylo */
          r = (f[0] + f[1] + f[3] + 2.0 * (f[4] + f[7] + f[8])) / (1.0 + v);
          f[2] = f[4] - 2.0 / 3.0 * r * v;
          f[5] = f[7] + 0.5 * (f[3] - f[1]) - 1.0 / 6.0 * r * v;
          f[6] = f[8] - 0.5 * (f[3] - f[1]) - 1.0 / 6.0 * r * v;
          break;
        default:
          return -1;
      }
    }
    if (out_rho) *out_rho = r;
    if (out_v) *out_v = v;
    return 0;
  }
  if (style == ORC_M_DIRICHLET) {
    r = rho;
    switch (wall) {
      case ORC_XHI: /* inlet_momentum command, dirichlet, main text */
        vx = (f[0] + f[2] + f[4] + 2.0 * (f[1] + f[5] + f[8])) / r - 1.0;
        f[3] = f[1] - 2.0 / 3.0 * r * vx;
        f[6] = f[8] + 0.5 * (f[4] - f[2]) - 1.0 / 6.0 * r * vx;
        f[7] = f[5] - 0.5 * (f[4] - f[2]) - 1.0 / 6.0 * r * vx;
        break;
      case ORC_XLO: /* App. A, dirichlet, xlo */
        vx = 1.0 - (f[0] + f[2] + f[4] + 2.0 * (f[3] + f[6] + f[7])) / r;
        f[1] = f[3] + 2.0 / 3.0 * r * vx;
        f[5] = f[7] - 0.5 * (f[2] - f[4]) + 1.0 / 6.0 * r * vx;
        f[8] = f[6] + 0.5 * (f[2] - f[4]) + 1.0 / 6.0 * r * vx;
        break;
      case ORC_YHI: /* App. A, dirichlet, yhi */
        vx = (f[0] + f[1] + f[3] + 2.0 * (f[2] + f[5] + f[6])) / r - 1.0;
        f[4] = f[2] - 2.0 / 3.0 * r * vx;
        f[7] = f[5] + 0.5 * (f[1] - f[3]) - 1.0 / 6.0 * r * vx;
        f[8] = f[6] - 0.5 * (f[1] - f[3]) - 1.0 / 6.0 * r * vx;
        break;
      case ORC_YLO: /* App. A, dirichlet, ylo */
        vx = 1.0 - (f[0] + f[1] + f[3] + 2.0 * (f[4] + f[7] + f[8])) / r;
        f[2] = f[4] + 2.0 / 3.0 * r * vx;
        f[5] = f[7] + 0.5 * (f[3] - f[1]) + 1.0 / 6.0 * r * vx;
        f[6] = f[8] - 0.5 * (f[3] - f[1]) + 1.0 / 6.0 * r * vx;
        break;
      default:
        return -1;
    }
    if (out_rho) *out_rho = r;
    if (out_v) *out_v = vx;
    return 0;
  }
  return -1;
}

/* Does mode (ex, ey) arriving at a node of this wall come from outside
 * the domain through the wall? */
static int crosses(int wall, int ex, int ey) {
  switch (wall) {
    case ORC_XLO: return ex > 0;
    case ORC_XHI: return ex < 0;
    case ORC_YLO: return ey > 0;
    case ORC_YHI: return ey < 0;
  }
  return 0;
}

/* coordinate of a node along its opening's wall */
static int along(int wall, int x, int y) {
  return (wall == ORC_XLO || wall == ORC_XHI) ? y : x;
}

/* ------------------------------------------------------------------ */
/* surface reaction (surface_reaction command, App. C)                 */
/* ------------------------------------------------------------------ */

/* One reactive link.  g_out is the post-collision mode of the fluid node
 * that headed into the solid; returns the link concentration C_i and the
 * incoming mode g_in.  With the D2Q4 weight 2 w_i = 1/2 this is
 * C = (2 g + kr Cs)/(kr + 1/2), g_i = -g + C/2 of the surface_reaction
 * command. */
void orc_reaction_link(int q, int i, double g_out, double kr, double Cs,
                       double *C_i, double *g_in) {
  double w = (q == 4) ? W4[i] : W9[i];
  double c = (2.0 * g_out + kr * Cs) / (kr + 2.0 * w);
  *C_i = c;
  *g_in = -g_out + 2.0 * w * c;
}

/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): one step of the
 * generator whose state is x, i.e. the finaliser applied to x + gamma. */
uint64_t orc_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/* ------------------------------------------------------------------ */
/* one iteration                                                       */
/* ------------------------------------------------------------------ */

static double psi_sc(const orc_t *o, double rho) {
  /* interforce command: psi = psi0 exp(-rho0/rho) */
  return o->psi0 * exp(-o->rho0 / rho);
}

/* An edge of the domain is no longer periodic when an opening lies on
 * either of its two walls (the x edge for xlo/xhi, the y edge for
 * ylo/yhi); the slip rule must not reach across it. */
static int edge_open(const orc_t *o, int xedge) {
  for (int k = 0; k < o->nopen; k++)
    if ((o->op[k].wall <= ORC_XHI) == (xedge != 0)) return 1;
  return 0;
}

/* solid test of node (x, y) given in unwrapped coordinates: 1 if solid,
 * 0 if fluid, -1 if it lies across an edge that has an opening */
static int solid_u(const orc_t *o, int x, int y) {
  if (((x < 0 || x >= o->nx) && edge_open(o, 1)) || ((y < 0 || y >= o->ny) && edge_open(o, 0)))
    return -1;
  return o->solid[(size_t)wrap(y, o->ny) * o->nx + wrap(x, o->nx)] ? 1 : 0;
}

/* boundary_style slip (Fig. slip): the diagonal mode i = (a, b) arriving at
 * fluid node y = (x, y) whose source y - (a, b) is solid comes by mirror
 * reflection from a wall of that source.  Horizontal wall (the nodes
 * y - (0, b) and y - (2a, b) solid, y - (a, 0) and y - (2a, 0) fluid): the
 * mode (a, -b) emitted by y - (2a, 0), as in f8(i+2, j) = f5(i, j).
 * Vertical wall (y - (a, 0) and y - (a, 2b) solid, y - (0, b) and
 * y - (0, 2b) fluid): the mode (-a, b) emitted by y - (0, 2b), as in
 * f6(i, j+2) = f5(i, j).  The two arrangements exclude each other and
 * each reflection maps onto its reverse, so every emitted population is
 * used exactly once.  Returns 0 (bounce-back) in every other case,
 * including a path across a wall with an opening. */
static int slip_source(const orc_t *o, int s, int x, int y, int i, double *fs) {
  const int a = EX9[i], b = EY9[i];
  int s1 = solid_u(o, x, y - b), s2 = solid_u(o, x - 2 * a, y - b);
  int f1 = solid_u(o, x - a, y), f2 = solid_u(o, x - 2 * a, y);
  if (s1 == 1 && s2 == 1 && f1 == 0 && f2 == 0) {
    int m = dir9(a, -b);
    size_t ne = (size_t)wrap(y, o->ny) * o->nx + wrap(x - 2 * a, o->nx);
    *fs = o->f[s][ne * 9 + m];
    return 1;
  }
  s1 = solid_u(o, x - a, y);
  s2 = solid_u(o, x - a, y - 2 * b);
  f1 = solid_u(o, x, y - b);
  f2 = solid_u(o, x, y - 2 * b);
  if (s1 == 1 && s2 == 1 && f1 == 0 && f2 == 0) {
    int m = dir9(-a, b);
    size_t ne = (size_t)wrap(y - 2 * b, o->ny) * o->nx + wrap(x, o->nx);
    *fs = o->f[s][ne * 9 + m];
    return 1;
  }
  return 0;
}

int orc_step(orc_t *o) {
  const int nx = o->nx, ny = o->ny, nc = o->nc;
  const size_t nn = (size_t)nx * ny;
  o->t += 1;

  /* 1. streaming with half-way bounce-back (Fig. 1; noslip style):
   * f~_i(x) = f*_i(x - e_i), or f*_opp(i)(x) when x - e_i is solid. */
  for (int s = 0; s < nc; s++) {
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        size_t n = (size_t)y * nx + x;
        double *ft = &o->ft[s][n * 9];
        if (o->solid[n]) {
          for (int i = 0; i < 9; i++) ft[i] = 0.0;
          continue;
        }
        for (int i = 0; i < 9; i++) {
          int xs = wrap(x - EX9[i], nx), ys = wrap(y - EY9[i], ny);
          size_t ns = (size_t)ys * nx + xs;
          if (o->solid[ns]) {
            ft[i] = o->f[s][n * 9 + OPP9[i]];
            double R = o->Rmap[s] ? o->Rmap[s][ns] : o->slipR[s];
            if (R > 0.0 && i >= 5) {
              double fs;
              if (slip_source(o, s, x, y, i, &fs))
                ft[i] = R * fs + (1.0 - R) * ft[i];
            }
          } else {
            ft[i] = o->f[s][ns * 9 + i];
          }
        }
      }
  }

  /* 2. openings after streaming: velocity and dirichlet styles
   * (inlet_momentum/outlet_momentum commands, App. A). */
  for (int s = 0; s < nc; s++) {
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        size_t n = (size_t)y * nx + x;
        int id = o->open_id[n];
        if (id < 0 || o->solid[n]) continue;
        const opening_t *p = &o->op[id];
        int st = p->style[s];
        if (st == ORC_M_POISEUILLE || st == ORC_M_UNIFORM) {
          double v = (st == ORC_M_UNIFORM)
                         ? p->v[s]
                         : orc_poiseuille_v(p->v[s], p->a0, p->a1,
                                            along(p->wall, x, y));
          orc_zouhe(p->wall, p->kind, st, v, 0.0, &o->ft[s][n * 9], NULL,
                    NULL);
        } else if (st == ORC_M_DIRICHLET) {
          orc_zouhe(p->wall, p->kind, st, 0.0, p->rho[s], &o->ft[s][n * 9],
                    NULL, NULL);
        }
      }
  }

  /* 3. moments: rho = sum f, j = sum f e (Sec. Model and algorithm) */
  for (int s = 0; s < nc; s++)
    for (size_t n = 0; n < nn; n++) {
      double r = 0.0, jx = 0.0, jy = 0.0;
      if (!o->solid[n]) {
        for (int i = 0; i < 9; i++) {
          double fi = o->ft[s][n * 9 + i];
          r += fi;
          jx += fi * EX9[i];
          jy += fi * EY9[i];
        }
      }
      o->rho[s][n] = r;
      o->jx[s][n] = jx;
      o->jy[s][n] = jy;
    }

  /* 4. forces.  aveforce: F per fluid node; aveacceleration: rho a;
   * interforce: F = -G psi(x) sum_i w_i psi(x+e_i) e_i (one component,
   * psi = psi0 exp(-rho0/rho)) or F_s = -G rho_s(x) sum_i w_i
   * rho_sbar(x+e_i) e_i (two components); adhesiveforce: the same with
   * s(x+e_i) = 1 on solid nodes, 0 on fluid nodes. */
  for (int s = 0; s < nc; s++)
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        size_t n = (size_t)y * nx + x;
        double Fx = 0.0, Fy = 0.0;
        if (!o->solid[n]) {
          double r = o->rho[s][n];
          Fx = o->fave[s][0] + r * o->acc[s][0];
          Fy = o->fave[s][1] + r * o->acc[s][1];
          if (o->sc_on) {
            double sx = 0.0, sy = 0.0;
            int other = (nc == 2) ? 1 - s : s;
            for (int i = 1; i < 9; i++) {
              size_t nb = (size_t)wrap(y + EY9[i], ny) * nx +
                          wrap(x + EX9[i], nx);
              double pn = 0.0;
              if (!o->solid[nb])
                pn = (nc == 2) ? o->rho[other][nb] : psi_sc(o, o->rho[s][nb]);
              sx += W9[i] * pn * EX9[i];
              sy += W9[i] * pn * EY9[i];
            }
            double pself = (nc == 2) ? r : psi_sc(o, r);
            Fx += -o->G * pself * sx;
            Fy += -o->G * pself * sy;
          }
          if (o->ads_on[s]) {
            double sx = 0.0, sy = 0.0;
            for (int i = 1; i < 9; i++) {
              size_t nb = (size_t)wrap(y + EY9[i], ny) * nx +
                          wrap(x + EX9[i], nx);
              double sn = o->solid[nb] ? 1.0 : 0.0;
              sx += W9[i] * sn * EX9[i];
              sy += W9[i] * sn * EY9[i];
            }
            double pself = (nc == 2)
                               ? r
                               : o->ads_psi0[s] * exp(-o->ads_rho0[s] / r);
            Fx += -o->Gads[s] * pself * sx;
            Fy += -o->Gads[s] * pself * sy;
          }
        }
        o->Fx[s][n] = Fx;
        o->Fy[s][n] = Fy;
      }

  /* 5-6. equilibrium velocity and BGK collision, Eq. (1):
   * f* = f~ - (f~ - f^eq(rho, u_eq))/tau.
   * One component: u_eq = (j + tau F)/rho.  Two components (fluids
   * command and its references): u' = sum_s (j_s/tau_s) / sum_s
   * (rho_s/tau_s), u_eq,s = u' + tau_s F_s / rho_s. */
  for (size_t n = 0; n < nn; n++) {
    if (o->solid[n]) {
      for (int s = 0; s < nc; s++) {
        for (int i = 0; i < 9; i++) o->f[s][n * 9 + i] = 0.0;
        o->meq[s][n] = 0.0;
      }
      continue;
    }
    double upx = 0.0, upy = 0.0;
    if (nc == 2) {
      double num_x = 0.0, num_y = 0.0, den = 0.0;
      for (int s = 0; s < 2; s++) {
        num_x += o->jx[s][n] / o->tau[s];
        num_y += o->jy[s][n] / o->tau[s];
        den += o->rho[s][n] / o->tau[s];
      }
      upx = num_x / den;
      upy = num_y / den;
    }
    for (int s = 0; s < nc; s++) {
      double r = o->rho[s][n], tau = o->tau[s];
      double uex, uey;
      if (nc == 1) {
        uex = (o->jx[s][n] + tau * o->Fx[s][n]) / r;
        uey = (o->jy[s][n] + tau * o->Fy[s][n]) / r;
      } else {
        uex = upx + tau * o->Fx[s][n] / r;
        uey = upy + tau * o->Fy[s][n] / r;
      }
      double feq[9], se = 0.0;
      orc_feq(r, uex, uey, o->alpha[s], feq);
      for (int i = 0; i < 9; i++) {
        double fi = o->ft[s][n * 9 + i];
        o->f[s][n * 9 + i] = fi - (fi - feq[i]) / tau;
        se += feq[i];
      }
      o->meq[s][n] = se;
    }
  }

  /* 8. node fields: density and physical momentum j + F/2 (Eq. (4)) */
  for (int s = 0; s < nc; s++)
    for (size_t n = 0; n < nn; n++) {
      o->px[s][n] = o->jx[s][n] + 0.5 * o->Fx[s][n];
      o->py[s][n] = o->jy[s][n] + 0.5 * o->Fy[s][n];
    }

  /* 7. gradient openings after collision: f_i(wall) = 2 f_i(wall+1n) -
   * f_i(wall+2n), n the inward normal (inlet_momentum command, gradient
   * style).  The node fields are extrapolated the same way. */
  for (int s = 0; s < nc; s++)
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        size_t n = (size_t)y * nx + x;
        int id = o->open_id[n];
        if (id < 0 || o->solid[n] || o->op[id].style[s] != ORC_M_GRADIENT)
          continue;
        int dx = 0, dy = 0;
        switch (o->op[id].wall) {
          case ORC_XLO: dx = 1; break;
          case ORC_XHI: dx = -1; break;
          case ORC_YLO: dy = 1; break;
          case ORC_YHI: dy = -1; break;
        }
        size_t n1 = (size_t)wrap(y + dy, ny) * nx + wrap(x + dx, nx);
        size_t n2 = (size_t)wrap(y + 2 * dy, ny) * nx + wrap(x + 2 * dx, nx);
        for (int i = 0; i < 9; i++)
          o->f[s][n * 9 + i] =
              2.0 * o->f[s][n1 * 9 + i] - o->f[s][n2 * 9 + i];
        o->rho[s][n] = 2.0 * o->rho[s][n1] - o->rho[s][n2];
        o->px[s][n] = 2.0 * o->px[s][n1] - o->px[s][n2];
        o->py[s][n] = 2.0 * o->py[s][n1] - o->py[s][n2];
        o->meq[s][n] = 2.0 * o->meq[s][n1] - o->meq[s][n2];
      }

  /* 9. solute transport (solute command, Eq. (3), Eq. (4)) */
  if (o->qs) {
    const int q = o->qs;
    const int *EX = (q == 4) ? EX4 : EX9;
    const int *EY = (q == 4) ? EY4 : EY9;
    const double *W = (q == 4) ? W4 : W9;
    const int *OPP = (q == 4) ? OPP4 : OPP9;
    /* 9a. streaming of every node first (the sources must still hold the
     * previous post-collision state); bounce-back or the reaction rule at
     * solid sources */
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        size_t n = (size_t)y * nx + x;
        double *gt = &o->gt[n * q];
        o->nU[n] = 0;
        o->Ubits[n] = 0;
        o->Cw[n] = 0.0;
        if (o->solid[n]) {
          for (int i = 0; i < q; i++) gt[i] = 0.0;
          continue;
        }
        int id = o->open_id[n];
        const opening_t *p = (id >= 0) ? &o->op[id] : NULL;
        for (int i = 0; i < q; i++) {
          if (p && crosses(p->wall, EX[i], EY[i])) {
            gt[i] = 0.0; /* filled by the opening rule below */
            continue;
          }
          int xs = wrap(x - EX[i], nx), ys = wrap(y - EY[i], ny);
          size_t ns = (size_t)ys * nx + xs;
          if (o->solid[ns]) {
            double gout = o->g[n * q + OPP[i]];
            if (o->react_on) {
              double Ci, gin;
              orc_reaction_link(q, i, gout, o->kr, o->Cs, &Ci, &gin);
              gt[i] = gin;
              o->Cw[n] += Ci;
              o->nU[n] += 1;
              o->Ubits[n] |= 1 << i;
            } else {
              gt[i] = gout; /* bounce-back at the solid surface */
            }
          } else {
            gt[i] = o->g[ns * q + i];
          }
        }
        double Cs = 0.0;
        for (int i = 0; i < q; i++) Cs += gt[i];
        o->Cst[n] = Cs;
      }

    /* 9b. inlet_solute/outlet_solute rules (App. B) on the opening nodes,
     * then the node concentrations that enter the collision */
    const double Dsol = (o->taus - 0.5) / (q == 4 ? 2.0 : 3.0);
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        size_t n = (size_t)y * nx + x;
        double *gt = &o->gt[n * q];
        o->Cpre[n] = 0.0;
        if (o->solid[n]) continue;
        int id = o->open_id[n];
        const opening_t *p = (id >= 0) ? &o->op[id] : NULL;
        if (p) {
          /* dirichlet sets the crossing modes so that C = Cbar (split by
           * weight when several modes cross); adiabatic reflects the
           * opposite mode; flux balances v C0 against the advective and
           * diffusive flux to the nearest inner node and puts every mode
           * at equilibrium */
          if (p->sstyle == ORC_S_DIRICHLET) {
            double Cp = 0.0, wsum = 0.0;
            for (int i = 0; i < q; i++) {
              if (crosses(p->wall, EX[i], EY[i])) wsum += W[i];
              else Cp += gt[i];
            }
            for (int i = 0; i < q; i++)
              if (crosses(p->wall, EX[i], EY[i]))
                gt[i] = (p->Cbar - Cp) * W[i] / wsum;
          } else if (p->sstyle == ORC_S_ADIABATIC) {
            for (int i = 0; i < q; i++)
              if (crosses(p->wall, EX[i], EY[i])) gt[i] = gt[OPP[i]];
          } else if (p->sstyle == ORC_S_FLUX) {
            /* inward normal of the wall: xlo +x, xhi -x, ylo +y, yhi -y */
            static const int NXW[4] = {1, -1, 0, 0}, NYW[4] = {0, 0, 1, -1};
            size_t ni = (size_t)wrap(y + NYW[p->wall], ny) * nx +
                        wrap(x + NXW[p->wall], nx);
            double C1 = o->solid[ni] ? 0.0 : o->Cst[ni];
            double v = p->sv, C0 = p->Cbar, Cf;
            if (p->kind == ORC_INLET)
              Cf = (v * C0 + Dsol * C1) / (Dsol + v);
            else
              Cf = (v * C0 - Dsol * C1) / (v - Dsol);
            double u[2];
            solvent_velocity(o, n, u);
            double geq[9];
            solute_geq(q, Cf, u[0], u[1], geq);
            for (int i = 0; i < q; i++) gt[i] = geq[i];
          }
        }
        double C = 0.0;
        for (int i = 0; i < q; i++) C += gt[i];
        o->Cpre[n] = C;
      }

    /* 9c. collision with g^eq(C, u_s), u the solvent velocity of Eq. (4);
     * with intersolute u_s = u + taus F / C, F = -G psi(x) sum_{i=1..4}
     * psi(x + e_i) e_i over the D2Q4 neighbours, psi = psi0 exp(-C0/C)
     * from the concentrations of this step (0 on solid nodes and where
     * C <= 0) */
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        size_t n = (size_t)y * nx + x;
        double *gt = &o->gt[n * q];
        o->db[n] = 0.0;
        if (o->solid[n]) {
          for (int i = 0; i < q; i++) o->g[n * q + i] = 0.0;
          o->C[n] = 0.0;
          continue;
        }
        double C = o->Cpre[n];
        double u[2];
        solvent_velocity(o, n, u);
        double ux = u[0], uy = u[1];
        if (o->is_on && C > 0.0) {
          double Fx = 0.0, Fy = 0.0;
          for (int d = 0; d < 4; d++) {
            size_t nb = (size_t)wrap(y + EY4[d], ny) * nx + wrap(x + EX4[d], nx);
            double Cn = o->Cpre[nb];
            double psin = (o->solid[nb] || !(Cn > 0.0)) ? 0.0 : o->ispsi0 * exp(-o->isC0 / Cn);
            Fx += psin * EX4[d];
            Fy += psin * EY4[d];
          }
          double psi = o->ispsi0 * exp(-o->isC0 / C);
          Fx *= -o->isG * psi;
          Fy *= -o->isG * psi;
          ux += o->taus * Fx / C;
          uy += o->taus * Fy / C;
        }
        double geq[9];
        solute_geq(q, C, ux, uy, geq);
        for (int i = 0; i < q; i++)
          o->g[n * q + i] = gt[i] - (gt[i] - geq[i]) / o->taus;
        /* 10. precipitation after collision: dB = kr (C_w - Cs) if > 0,
         * removed in equal parts from the incoming modes (App. C rule 4) */
        int nU = o->nU[n];
        if (o->react_on && nU > 0) {
          double Cw = o->Cw[n] / nU;
          double dB = o->kr * (Cw - o->Cs);
          if (dB > 0.0) {
            for (int i = 0; i < q; i++)
              if (o->Ubits[n] & (1 << i)) o->g[n * q + i] -= dB / nU;
            o->db[n] = dB / nU;
          }
        }
        double Cn = 0.0;
        for (int i = 0; i < q; i++) Cn += o->g[n * q + i];
        o->C[n] = Cn;
      }

    /* ... and credited in equal parts to the solid nodes behind those
     * modes: each solid node gathers from its neighbours in index order */
    if (o->react_on) {
      for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
          size_t n = (size_t)y * nx + x;
          if (!o->solid[n]) continue;
          double acc = 0.0;
          for (int i = (q == 4 ? 0 : 1); i < q; i++) {
            int xf = x + EX[i], yf = y + EY[i];
            size_t nf = (size_t)wrap(yf, ny) * nx + wrap(xf, nx);
            if (o->solid[nf]) continue;
            int id = o->open_id[nf];
            if (id >= 0 && crosses(o->op[id].wall, EX[i], EY[i])) continue;
            acc += o->db[nf];
          }
          o->b[n] += acc;
        }

      /* 11. growth (surface_reaction command; App. C rules 3 and 5) */
      memset(o->flip, 0, nn);
      o->nmargin = 0;
      for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
          size_t n = (size_t)y * nx + x;
          if (o->solid[n] && o->margin_eps > 0.0 &&
              fabs(o->b[n] - o->bmax) <= o->margin_eps * fabs(o->bmax)) {
            if (o->nmargin < o->capmargin) {
              o->margin_node[o->nmargin] = (int64_t)n;
              o->margin_val[o->nmargin] = o->b[n] - o->bmax;
            }
            o->nmargin++;
          }
          if (!o->solid[n] || !(o->b[n] > o->bmax)) continue;
          size_t cand[4];
          int nc4 = 0;
          for (int d = 0; d < 4; d++) {
            size_t nb = (size_t)wrap(y + EY4[d], ny) * nx + wrap(x + EX4[d], nx);
            if (!o->solid[nb] && o->open_id[nb] < 0) cand[nc4++] = nb;
          }
          if (nc4 == 0) continue;
          uint64_t key = o->seed ^ ((uint64_t)o->t * (uint64_t)nn + n);
          int k = (int)(orc_splitmix64(key) % (uint64_t)nc4);
          o->flip[cand[k]] = 1;
          o->b[n] = 0.0;
        }
      o->nflips_last = 0;
      for (size_t n = 0; n < nn; n++) {
        if (!o->flip[n]) continue;
        o->nflips_last++;
        for (int s = 0; s < nc; s++) {
          double m = 0.0;
          for (int i = 0; i < 9; i++) {
            m += o->f[s][n * 9 + i];
            o->f[s][n * 9 + i] = 0.0;
          }
          o->removed[s] += m;
        }
        double ms = 0.0;
        for (int i = 0; i < q; i++) {
          ms += o->g[n * q + i];
          o->g[n * q + i] = 0.0;
        }
        o->removed_solute += ms;
        o->C[n] = 0.0;
        o->solid[n] = 1;
        o->b[n] = o->b0;
      }
    }
  }

  /* 12. thermo sums over the final state (thermo command) */
  double *T = o->thermo;
  for (int k = 0; k < ORC_T_COUNT; k++) T[k] = 0.0;
  for (size_t n = 0; n < nn; n++) {
    if (o->solid[n]) {
      T[ORC_T_NSOLID] += 1.0;
      T[ORC_T_BSUM] += o->b[n];
      continue;
    }
    T[ORC_T_NFLUID] += 1.0;
    for (int s = 0; s < nc; s++) {
      T[ORC_T_MASS1 + s] += o->rho[s][n];
      T[ORC_T_MASSEQ1 + s] += o->meq[s][n];
      T[ORC_T_MOMX] += o->px[s][n];
      T[ORC_T_MOMY] += o->py[s][n];
      T[ORC_T_MOMX1 + 2 * s] += o->px[s][n];
      T[ORC_T_MOMY1 + 2 * s] += o->py[s][n];
    }
    if (o->qs) T[ORC_T_SOLUTE] += o->C[n];
  }
  T[ORC_T_REMOVED1] = o->removed[0];
  T[ORC_T_REMOVED2] = o->removed[1];
  T[ORC_T_REMOVED_SOLUTE] = o->removed_solute;
  return 0;
}

int orc_get_fields(const orc_t *o, int comp, double *rho, double *px,
                   double *py, double *rho_eq) {
  if (comp < 0 || comp >= o->nc) return -1;
  size_t nn = (size_t)o->nx * o->ny;
  for (size_t n = 0; n < nn; n++) {
    int sol = o->solid[n];
    if (rho) rho[n] = sol ? 0.0 : o->rho[comp][n];
    if (px) px[n] = sol ? 0.0 : o->px[comp][n];
    if (py) py[n] = sol ? 0.0 : o->py[comp][n];
    if (rho_eq) rho_eq[n] = sol ? 0.0 : o->meq[comp][n];
  }
  return 0;
}

int orc_get_solute_C(const orc_t *o, double *C) {
  if (!o->qs) return -1;
  memcpy(C, o->C, (size_t)o->nx * o->ny * sizeof(double));
  return 0;
}

int orc_get_thermo(const orc_t *o, double *out) {
  memcpy(out, o->thermo, sizeof(o->thermo));
  return 0;
}

int orc_set_margin_eps(orc_t *o, double eps, int cap) {
  free(o->margin_node);
  free(o->margin_val);
  o->margin_eps = eps;
  o->capmargin = cap > 0 ? cap : 0;
  o->nmargin = 0;
  o->margin_node = o->capmargin ? (int64_t *)calloc((size_t)o->capmargin, sizeof(int64_t)) : NULL;
  o->margin_val = o->capmargin ? (double *)calloc((size_t)o->capmargin, sizeof(double)) : NULL;
  return 0;
}

int orc_get_margin_events(const orc_t *o, int64_t *node, double *val, int cap) {
  int n = o->nmargin < o->capmargin ? o->nmargin : o->capmargin;
  for (int k = 0; k < n && k < cap; k++) {
    node[k] = o->margin_node[k];
    val[k] = o->margin_val[k];
  }
  return o->nmargin;
}

int orc_get_flips(const orc_t *o, int64_t *idx, int cap) {
  size_t nn = (size_t)o->nx * o->ny;
  int k = 0;
  if (o->qs && o->react_on) {
    for (size_t n = 0; n < nn; n++)
      if (o->flip[n]) {
        if (k < cap) idx[k] = (int64_t)n;
        k++;
      }
  }
  return k;
}
