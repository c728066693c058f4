/*
 * lb2d_oracle.h -- interface of the FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow, single-threaded
 * restatement of the lattice Boltzmann update of arXiv:1202.0442
 * ("Introduction to Perl module lb2d.pm 0.1", D. Sergi).  Only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark call it; the
 * product library never links, loads or calls anything in this directory,
 * and the two share no code, header or constant table.
 *
 * Conventions
 *   - nodes (x, y), 0 <= x < nx, 0 <= y < ny; a paper script's
 *     lattice(N_x, N_y) has nx = N_x + 1 nodes (lattice command).
 *   - arrays handed in or out are SoA, fastest index x:
 *       populations  [q][ny][nx]   (q = 9 fluid, 4 or 9 solute)
 *       node fields  [ny][nx]
 *   - every function returning int gives 0 on success, < 0 on bad input.
 */
#ifndef LB2D_ORACLE_H
#define LB2D_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* walls of the domain (inlet/outlet commands) */
enum { ORC_XLO = 0, ORC_XHI = 1, ORC_YLO = 2, ORC_YHI = 3 };
/* opening kind */
enum { ORC_INLET = 0, ORC_OUTLET = 1 };
/* inlet_momentum/outlet_momentum styles */
enum { ORC_M_NONE = 0, ORC_M_POISEUILLE = 1, ORC_M_UNIFORM = 2,
       ORC_M_DIRICHLET = 3, ORC_M_GRADIENT = 4 };
/* inlet_solute/outlet_solute styles */
enum { ORC_S_NONE = 0, ORC_S_DIRICHLET = 1, ORC_S_ADIABATIC = 2, ORC_S_FLUX = 3 };

/* thermo record (thermo command), all sums in FP64 over the state at the
 * end of the last iteration */
enum {
  ORC_T_MASS1 = 0, ORC_T_MASS2, ORC_T_MOMX, ORC_T_MOMY,
  ORC_T_MASSEQ1, ORC_T_MASSEQ2, ORC_T_SOLUTE, ORC_T_BSUM,
  ORC_T_REMOVED1, ORC_T_REMOVED2, ORC_T_REMOVED_SOLUTE,
  ORC_T_NSOLID, ORC_T_NFLUID,
  ORC_T_MOMX1, ORC_T_MOMY1, ORC_T_MOMX2, ORC_T_MOMY2,
  ORC_T_COUNT
};

typedef struct orc orc_t;

orc_t *orc_create(int nx, int ny, int ncomp, int solute_q);
void   orc_destroy(orc_t *o);

int orc_set_tau(orc_t *o, int comp, double tau);
int orc_set_alpha(orc_t *o, int comp, double alpha);
int orc_set_taus(orc_t *o, double taus);
int orc_set_solid(orc_t *o, const uint8_t *mask);
int orc_get_solid(const orc_t *o, uint8_t *mask);
int orc_set_f(orc_t *o, int comp, const double *f);
int orc_get_f(const orc_t *o, int comp, double *f);
int orc_set_equilibrium(orc_t *o, int comp, const double *rho,
                        const double *ux, const double *uy);
int orc_set_g(orc_t *o, const double *g);
int orc_get_g(const orc_t *o, double *g);
int orc_set_solute_equilibrium(orc_t *o, const double *C,
                               const double *ux, const double *uy);
int orc_set_b(orc_t *o, const double *b);
int orc_get_b(const orc_t *o, double *b);

int orc_set_aveforce(orc_t *o, int comp, double fx, double fy);
int orc_set_aveacceleration(orc_t *o, int comp, double ax, double ay);
int orc_set_interforce(orc_t *o, double G, double psi0, double rho0);
int orc_set_adhesiveforce(orc_t *o, int comp, double G, double psi0,
                          double rho0);

/* boundary_style slip/mixed/hybrid: reflection coefficient R of the solid
 * nodes for component comp (0 = noslip, 1 = slip, else mixed).  R_all
 * applies to every solid node (also ones grown later) unless R_map is
 * given ([ny][nx], read on solid nodes; nodes that turn solid later get
 * R = 0). */
int orc_set_slip(orc_t *o, int comp, double R_all, const double *R_map);

int orc_add_opening(orc_t *o, int wall, int a0, int a1, int kind);
int orc_set_opening_momentum(orc_t *o, int opening, int comp, int style,
                             double v, double rho);
/* Cbar: dirichlet concentration, or C0 of the flux style; v: the flux
 * style's velocity (ignored by the others) */
int orc_set_opening_solute(orc_t *o, int opening, int style, double Cbar,
                           double v);
/* intersolute command: G, psi0, C0 */
int orc_set_intersolute(orc_t *o, double G, double psi0, double C0);

int orc_set_reaction(orc_t *o, double kr, double Cs, double b0,
                     double bmax, uint64_t seed);

int  orc_step(orc_t *o);
long orc_time(const orc_t *o);
int  orc_set_time(orc_t *o, long t);

/* fields of the last iteration: density, physical momentum density
 * (j + F/2) and the equilibrium density of each component */
int orc_get_fields(const orc_t *o, int comp, double *rho, double *px,
                   double *py, double *rho_eq);
int orc_get_solute_C(const orc_t *o, double *C);
int orc_get_thermo(const orc_t *o, double *out /* ORC_T_COUNT */);
/* last step's growth events: number of flips, and the flipped node
 * indices (y*nx + x) in increasing order, up to cap */
int orc_get_flips(const orc_t *o, int64_t *idx, int cap);
/* growth decisions near the threshold: from now on every iteration
 * records the solid nodes whose b lies within eps * |bmax| of bmax when the
 * growth rule reads it (up to cap of them); get returns their number and
 * copies (node index, b - bmax) */
int orc_set_margin_eps(orc_t *o, double eps, int cap);
int orc_get_margin_events(const orc_t *o, int64_t *node, double *val, int cap);

/* single-node pieces, exposed for the analytic pin tests */
void orc_feq(double rho, double ux, double uy, double alpha, double *feq);
int  orc_zouhe(int wall, int kind, int style, double v, double rho,
               double *f, double *out_rho, double *out_v);
void orc_reaction_link(int q, int i, double g_out, double kr, double Cs,
                       double *C_i, double *g_in);
uint64_t orc_splitmix64(uint64_t x);
double orc_poiseuille_v(double vmax, int a0, int a1, int coord);

#ifdef __cplusplus
}
#endif
#endif
