// k_fluid.cu -- one iteration of the D2Q9 fluid lattice(s).
//
// k_fluid_local: pull streaming with half-way bounce-back (Fig. 1 and the
//   noslip boundary_style of the paper), Zou-He inlet/outlet rules on
//   opening nodes (inlet_momentum/outlet_momentum, App. A), moments, forces
//   that need no neighbour density (aveforce, aveacceleration,
//   adhesiveforce), equilibrium velocity by velocity shift and BGK
//   collision with Eq. (2) -- all in one pass, one thread per node, nine
//   loads and nine stores per component.
// k_fluid_solute: k_fluid_local's node update followed, in the same
//   thread, by the solute node update of lbsolute.cuh (solute command,
//   Eq. (3); surface_reaction, App. C) with the solvent velocity of Eq. (4)
//   taken from registers: one pass for single-component runs with a solute
//   and no intersolute.
// k_fluid_sc: the same plus interforce, which needs the densities of the
//   eight neighbours after this step's streaming and opening rules (the sums
//   wrap periodically across every wall, openings or not).  Each CTA pulls
//   the populations of its tile and of a one-node ring around it, applies
//   the opening rules of the nodes that have one, stages
//   rho - rho_ref in shared memory, and reads the neighbours from there; the
//   ring's extra loads hit L1/L2, the HBM traffic stays nine loads and nine
//   stores per node.
// k_gradient: gradient openings, f(wall) = 2 f(wall+n) - f(wall+2n) after
//   the collision (inlet_momentum command).
// slip_fix: the slip, mixed and hybrid boundary styles, applied after the
//   bounce-back pull of either kernel.
//
// k_nbcode: every node slot's neighbour code from the mask.
//
// The kernels read each node's 3 x 3 solid neighbourhood as one 16-bit
// code (k_nbcode builds the codes from the mask once, k_apply_flips
// refreshes them around nodes that grow solid): two bytes per node in place
// of the mask-word arithmetic that otherwise dominated the streaming
// kernel's instruction count.
#include "lbcollide.cuh"
#include "lbpdl.cuh"
#include "lbsolute.cuh"

namespace lbk {

namespace {

// pull the nine populations of node (x, y) from `base` (one component),
// bouncing back from solid sources; `bits` is the node's neighbourhood.
// One load per direction: the streaming source x - e_i, or, where that
// node (neighbour opp(i)) is solid, the node's own outgoing population of
// the opposite direction (half-way bounce-back).
template <class S>
__device__ __forceinline__ void pull9(const S *base, const Geometry &g, int x, int y,
                                      uint32_t bits, float inv, float (&h)[9]) {
  const int xm = x ? x - 1 : g.nx - 1, xp = (x + 1 == g.nx) ? 0 : x + 1;
  const int ym = y ? y - 1 : g.ny - 1, yp = (y + 1 == g.ny) ? 0 : y + 1;
  const int P = (int)g.plane;
  const int r0 = y * g.pitch, rm = ym * g.pitch, rp = yp * g.pitch;
  const int self = r0 + x;
  const int src[9] = {self, r0 + xm, rm + x, r0 + xp, rp + x, rm + xm, rm + xp, rp + xp, rp + xm};
#pragma unroll
  for (int i = 0; i < 9; i++) {
    const int k = (i && nb(bits, OPP(i))) ? OPP(i) * P + self : i * P + src[i];
    h[i] = Store<S>::ld(base, k, inv);
  }
}

// solid test of node (x, y) given up to two nodes outside the lattice: 1
// solid, 0 fluid, -1 across an edge that carries an opening
__device__ __forceinline__ int solid_u(const FluidArgs &p, int x, int y) {
  const Geometry &g = p.g;
  if ((x < 0 || x >= g.nx) && p.edge_x) return -1;
  const int gy = grow(g, y);  // the lattice's edges, not a slab's
  if ((gy < 0 || gy >= g.gny) && p.edge_y) return -1;
  x = x < 0 ? x + g.nx : (x >= g.nx ? x - g.nx : x);
  y = y < 0 ? y + g.ny : (y >= g.ny ? y - g.ny : y);
  return solid_at(p.mask, g.mw, x, y);
}

// boundary_style slip (Fig. slip), mixed and hybrid, after pull9 has
// bounced back every mode with a solid source.  A diagonal mode i = (a, b)
// whose source x - (a, b) is solid with coefficient R > 0 takes
// R f_m(e) + (1 - R) (its bounce-back value), where e, m is the mirror
// reflection at a flat wall of that source: horizontal wall (x - (0, b)
// and x - (2a, b) solid, x - (a, 0) and x - (2a, 0) fluid): e = x - (2a, 0),
// m = (a, -b), as in f8(i+2, j) = f5(i, j); vertical wall (x - (a, 0) and
// x - (a, 2b) solid, x - (0, b) and x - (0, 2b) fluid): e = x - (0, 2b),
// m = (-a, b), as in f6(i, j+2) = f5(i, j).  Each reflection is paired with
// its reverse, so every population is used once and mass is kept; any
// other arrangement, or a path across an edge with an opening, stays
// bounce-back.  Axis modes always bounce back.
template <class S>
__device__ __forceinline__ void slip_fix(const FluidArgs &p, int c, const S *base, int x, int y,
                                      uint32_t bits, float inv, float (&h)[9]) {
  const Geometry &g = p.g;
#pragma unroll
  for (int i = 5; i < 9; i++) {
    if (!nb(bits, OPP(i))) continue;
    const int a = EX(i), b = EY(i);
    const int sx = wrapi(x - a, g.nx), sy = wrapi(y - b, g.ny);
    const float R = p.Rmap ? __ldg(p.Rmap + (size_t)c * g.plane + (size_t)sy * g.pitch + sx) : p.slipR[c];
    if (!(R > 0.f)) continue;
    int ex, ey, m;
    if (solid_u(p, x, y - b) == 1 && solid_u(p, x - 2 * a, y - b) == 1 && solid_u(p, x - a, y) == 0 &&
        solid_u(p, x - 2 * a, y) == 0) {
      ex = x - 2 * a;
      ey = y;
      m = (-b > 0) ? (a > 0 ? 5 : 6) : (a > 0 ? 8 : 7);
    } else if (solid_u(p, x - a, y) == 1 && solid_u(p, x - a, y - 2 * b) == 1 && solid_u(p, x, y - b) == 0 &&
               solid_u(p, x, y - 2 * b) == 0) {
      ex = x;
      ey = y - 2 * b;
      m = (b > 0) ? (-a > 0 ? 5 : 6) : (-a > 0 ? 8 : 7);
    } else {
      continue;
    }
    ex = wrapi(ex, g.nx);
    ey = wrapi(ey, g.ny);
    const float fs = Store<S>::ld(base, (size_t)m * g.plane + (size_t)ey * g.pitch + ex, inv);
    h[i] = R * fs + (1.0f - R) * h[i];
  }
}

// diagonal-neighbour bits of the 3 x 3 neighbourhood (sources of 5..8)
constexpr uint32_t DIAG_BITS = (1u << NBPOS(-1, -1)) | (1u << NBPOS(1, -1)) | (1u << NBPOS(-1, 1)) |
                               (1u << NBPOS(1, 1));

constexpr int LOC_BY = 8;

// SR: 0 rounding read from p.sr_seed, 1 nearest, 2 stochastic (16-bit,
// not ME).  Scaled 16-bit storage without ME runs folded (collide_store).
// The update of node (x, y) given its neighbour code (called by every lane
// of a warp: the warp votes on its solid lanes).  Returns false on solid
// nodes and row padding.  uo, if given, receives the node's solvent
// velocity of Eq. (4).  SLIP: the slip/mixed/hybrid boundary styles (a
// compile-time switch: the noslip kernels carry none of its registers).
template <class S, int NC, bool ME, bool PM, int SR, bool SLIP>
__device__ __forceinline__ bool fluid_node(const FluidArgs &p, int x, int y, uint32_t bits,
                                           float *uo = nullptr) {
  constexpr bool FOLD = Store<S>::kScaled && !ME;
  const float linv = FOLD ? 1.0f : p.inv_scale;
  const Geometry &g = p.g;
  // solid nodes (and the row padding past nx) hold no populations: their
  // slots are zero from the start and k_apply_flips clears grown nodes.  A
  // solid lane still stores zeros when its 32-byte sector holds a fluid
  // lane, so every sector the warp writes is written whole (a partial
  // sector costs the memory system a read-modify-write); sectors without a
  // fluid lane are left alone.
  const bool idle = (bits >> NBPOS(0, 0)) & 1u;
  const unsigned busy = __ballot_sync(0xffffffffu, !idle);
  if (idle) {
    constexpr int LPS = 32 / (int)sizeof(S);  // lanes per 32-byte sector
    if ((busy >> (threadIdx.x & ~(LPS - 1))) & ((1u << LPS) - 1u)) {
      const int self = y * g.pitch + x;
#pragma unroll
      for (int c = 0; c < NC; c++) {
        S *out = (S *)p.fout + (size_t)c * 9 * g.plane;
#pragma unroll
        for (int i = 0; i < 9; i++) Store<S>::st(out, i * (int)g.plane + self, 0.0f, 1.0f);
      }
    }
    return false;
  }
  float h[NC][9];
#pragma unroll
  for (int c = 0; c < NC; c++)
    pull9<S>((const S *)p.fin + (size_t)c * 9 * g.plane, g, x, y, bits, linv, h[c]);
  if (SLIP && (bits & DIAG_BITS)) {
#pragma unroll
    for (int c = 0; c < NC; c++)
      slip_fix<S>(p, c, (const S *)p.fin + (size_t)c * 9 * g.plane, x, y, bits, linv, h[c]);
  }
  if (p.nopen) apply_openings<NC>(p, x, y, h, FOLD ? p.scale : 1.0f);
  float F[NC][2];
#pragma unroll
  for (int c = 0; c < NC; c++) F[c][0] = F[c][1] = 0.f;
  collide_store<S, NC, ME, PM, FOLD, SR>(p, x, y, bits, h, F, uo);
  return true;
}

template <class S, int NC, bool ME, bool PM, int SR, bool SLIP>
__global__ void __launch_bounds__(32 * LOC_BY, ((NC == 1 && !ME && !PM) ? (SLIP ? 6 : 8) : 4) * 8 / LOC_BY)
    k_fluid_local(const FluidArgs p) {
  dep_wait();
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = p.g.clo + blockIdx.y * LOC_BY + threadIdx.y;
  if (y >= p.g.chi) return;
  // x < pitch: the grid covers whole 32-node words
  fluid_node<S, NC, ME, PM, SR, SLIP>(p, x, y, __ldg(p.nbc + (size_t)y * p.g.pitch + x));
}

// One fluid and one solute iteration of a single-component lattice in one
// pass (no intersolute): the solute update of a node needs only its own
// solvent velocity of this iteration, which stays in registers, and the
// previous iteration's solute populations around it.
template <class S, int SR, int Q, bool SLIP>
__global__ void __launch_bounds__(32 * LOC_BY, 4 * 8 / LOC_BY) k_fluid_solute(const FluidArgs p, const SoluteArgs sp) {
  dep_wait();
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = p.g.clo + blockIdx.y * LOC_BY + threadIdx.y;
  if (y >= p.g.chi) return;
  const uint32_t bits = __ldg(p.nbc + (size_t)y * p.g.pitch + x);
  float u[2];
  if (!fluid_node<S, 1, false, false, SR, SLIP>(p, x, y, bits, u)) return;
  solute_node<Q>(sp, x, y, bits, u[0], u[1]);
}

// 32 x 8 tiles, 4 CTAs/SM: measured fastest of 32 x {4, 8, 16, 32} (the
// barrier waits on fewer warps; the ring costs 33 % more pulls, from L1/L2)
constexpr int SC_TX = 32, SC_TY = 8;

template <class S, int NC, bool SLIP, bool OPEN>
__global__ void __launch_bounds__(SC_TX *SC_TY, 4) k_fluid_sc(const FluidArgs p) {
  // rho - rho_ref of every component for the tile and a one-node ring; slot
  // (ty + 1, tx + 1) holds node (x0 + tx, y0 + ty) wrapped periodically.
  // Solid nodes are told apart by the mask bits, not by the stored value.
  __shared__ float sd[NC][SC_TY + 2][SC_TX + 2];
  dep_wait();
  const Geometry &g = p.g;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = blockIdx.x * SC_TX, y0 = g.clo + blockIdx.y * SC_TY;
  const int xr = x0 + tx, yr = y0 + ty;
  const bool real = xr < g.nx && yr < g.chi;
  const int x = wrapi(xr, g.nx), y = wrapi(yr, g.ny);
  // the node's 3 x 3 solid neighbourhood (lanes past the lattice edge take
  // the wrapped node's)
  const uint32_t bits = __ldg(p.nbc + (size_t)y * g.pitch + x);
  const bool solid = (bits >> 4) & 1u;
  float h[NC][9];
#pragma unroll
  for (int c = 0; c < NC; c++) {
    float d = 0.f;
    if (!solid) {
      pull9<S>((const S *)p.fin + (size_t)c * 9 * g.plane, g, x, y, bits, p.inv_scale, h[c]);
      if (SLIP && (bits & DIAG_BITS))
        slip_fix<S>(p, c, (const S *)p.fin + (size_t)c * 9 * g.plane, x, y, bits, p.inv_scale, h[c]);
      if (OPEN) apply_opening_c(p, c, x, y, h[c]);
#pragma unroll
      for (int i = 0; i < 9; i++) d += h[c][i];
    }
    sd[c][ty + 1][tx + 1] = d;
  }
  // ring: 2 (TX + 2) + 2 TY slots, one thread each
  const int tid = ty * SC_TX + tx;
  constexpr int NRING = 2 * (SC_TX + 2) + 2 * SC_TY;
  if (tid < NRING) {
    int sx, sy;
    if (tid < SC_TX + 2) { sx = tid; sy = 0; }
    else if (tid < 2 * (SC_TX + 2)) { sx = tid - (SC_TX + 2); sy = SC_TY + 1; }
    else if (tid < 2 * (SC_TX + 2) + SC_TY) { sx = 0; sy = tid - 2 * (SC_TX + 2) + 1; }
    else { sx = SC_TX + 1; sy = tid - 2 * (SC_TX + 2) - SC_TY + 1; }
    const int hx = wrapi(x0 + sx - 1, g.nx), hy = wrapi(y0 + sy - 1, g.ny);
    const uint32_t hb = __ldg(p.nbc + (size_t)hy * g.pitch + hx);
    const bool hs = (hb >> 4) & 1u;
#pragma unroll
    for (int c = 0; c < NC; c++) {
      float d = 0.f;
      if (!hs) {
        float hh[9];
        pull9<S>((const S *)p.fin + (size_t)c * 9 * g.plane, g, hx, hy, hb, p.inv_scale, hh);
        if (SLIP && (hb & DIAG_BITS))
          slip_fix<S>(p, c, (const S *)p.fin + (size_t)c * 9 * g.plane, hx, hy, hb, p.inv_scale, hh);
        if (OPEN) apply_opening_c(p, c, hx, hy, hh);
#pragma unroll
        for (int i = 0; i < 9; i++) d += hh[i];
      }
      sd[c][sy][sx] = d;
    }
  }
  __syncthreads();
  if (!real || solid) return;
  // Since sum_i w_i e_i = 0, sum_i w_i psi(x + e_i) e_i equals
  // sum_i w_i (psi(x + e_i) - psi(x)) e_i; the differences are formed from
  // rho - rho_ref without cancellation:
  //   two components: rho_n - rho_c = drho_n - drho_c (psi = rho)
  //   one component:  psi_n - psi_c = psi_c expm1(rho0 (rho_n - rho_c)/(rho_n rho_c))
  // and a solid neighbour contributes psi = 0, i.e. a difference -psi_c.
  float F[NC][2];
  const int cx = tx + 1, cy = ty + 1;
#pragma unroll
  for (int c = 0; c < NC; c++) {
    const int o = (NC == 2) ? 1 - c : c;
    const float dc = sd[o][cy][cx];
    const float rc = p.rho_ref[o] + dc;
    const float psic = (NC == 1) ? p.psi0 * expf(-p.sc_rho0 / rc) : rc;
    float sx = 0.f, sy = 0.f;
#pragma unroll
    for (int i = 1; i < 9; i++) {
      float diff;
      if (nb(bits, i)) {
        diff = -psic;
      } else {
        const float dn = sd[o][cy + EY(i)][cx + EX(i)];
        if (NC == 1) {
          const float rn = p.rho_ref[o] + dn;
          diff = psic * expm1f(p.sc_rho0 * (dn - dc) / (rn * rc));
        } else {
          diff = dn - dc;
        }
      }
      sx += W9(i) * (float)EX(i) * diff;
      sy += W9(i) * (float)EY(i) * diff;
    }
    const float self = (NC == 1) ? psic : p.rho_ref[c] + sd[c][cy][cx];
    F[c][0] = -p.G * self * sx;
    F[c][1] = -p.G * self * sy;
  }
  collide_store<S, NC, true>(p, x, y, bits, h, F);
}

template <class S>
__global__ void k_gradient(const GradArgs a) {
  // one thread per opening node of every gradient opening
  dep_wait();
  const int k = blockIdx.y;
  const OpenDesc &o = a.op[k];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > o.a1 - o.a0) return;
  const Geometry &g = a.g;
  const int c = o.a0 + i;
  int x, y, dx = 0, dy = 0;
  switch (o.wall) {
    case 0: x = 0; y = c; dx = 1; break;
    case 1: x = g.nx - 1; y = c; dx = -1; break;
    case 2: x = c; y = 0; dy = 1; break;
    default: x = c; y = g.gny - 1; dy = -1; break;
  }
  y -= g.yoff;  // rows of the whole lattice -> rows held here
  if (y < g.clo || y >= g.chi || solid_at(a.mask, g.mw, x, y)) return;
  const size_t n0 = (size_t)y * g.pitch + x;
  const size_t n1 = (size_t)wrapi(y + dy, g.ny) * g.pitch + wrapi(x + dx, g.nx);
  const size_t n2 = (size_t)wrapi(y + 2 * dy, g.ny) * g.pitch + wrapi(x + 2 * dx, g.nx);
  for (int cc = 0; cc < a.nc; cc++) {
    if (o.style[cc] != OPEN_GRADIENT) continue;
    S *f = (S *)a.f + (size_t)cc * 9 * g.plane;
#pragma unroll
    for (int q = 0; q < 9; q++) {
      const size_t b = (size_t)q * g.plane;
      const float v1 = Store<S>::ld(f, b + n1, a.inv_scale);
      const float v2 = Store<S>::ld(f, b + n2, a.inv_scale);
      Store<S>::st(f, b + n0, 2.0f * v1 - v2, a.scale);
    }
    if (a.fields) {
      float *fl = a.fields + (size_t)cc * NFIELD * g.plane;
      for (int q = 0; q < NFIELD; q++) {
        const size_t b = (size_t)q * g.plane;
        fl[b + n0] = 2.0f * fl[b + n1] - fl[b + n2];
      }
    }
  }
}

// neighbour code of every node slot (periodic wrap, as the pull uses);
// slots past nx are coded solid
__global__ void k_nbcode(const uint32_t *mask, uint16_t *nbc, const Geometry g, int r0, int r1) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = r0 + blockIdx.y * 8 + threadIdx.y;
  if (y >= r1 || x >= g.pitch) return;
  uint32_t b = 1u << NBPOS(0, 0);
  if (x < g.nx) {
    const int xm = x ? x - 1 : g.nx - 1, xp = (x + 1 == g.nx) ? 0 : x + 1;
    const int ym = y ? y - 1 : g.ny - 1, yp = (y + 1 == g.ny) ? 0 : y + 1;
    b = nbr_bits(mask, g.mw, x, y, xm, xp, ym, yp);
  }
  nbc[(size_t)y * g.pitch + x] = (uint16_t)b;
}

template <class S, int NC, bool ME, bool PM, int SR>
void launch_local(const FluidArgs &a, cudaStream_t s) {
  dim3 blk(32, LOC_BY), grd((a.g.nx + 31) / 32, (a.g.chi - a.g.clo + LOC_BY - 1) / LOC_BY);
  if (a.slip) launch_pdl(k_fluid_local<S, NC, ME, PM, SR, true>, grd, blk, 0, s, a);
  else launch_pdl(k_fluid_local<S, NC, ME, PM, SR, false>, grd, blk, 0, s, a);
}

template <class S>
int launch_fluid_t(int nc, bool sc, bool me, const FluidArgs &a, cudaStream_t s) {
  if (sc) {
    dim3 blk(SC_TX, SC_TY), grd((a.g.nx + SC_TX - 1) / SC_TX, (a.g.chi - a.g.clo + SC_TY - 1) / SC_TY);
    // openings take their own instantiations: their rules would cost the
    // kernel without openings registers (spills in the two-component one)
    const bool op = a.nopen > 0;
    if (a.slip) {
      if (nc == 1) launch_pdl(op ? k_fluid_sc<S, 1, true, true> : k_fluid_sc<S, 1, true, false>, grd, blk, 0, s, a);
      else launch_pdl(op ? k_fluid_sc<S, 2, true, true> : k_fluid_sc<S, 2, true, false>, grd, blk, 0, s, a);
    } else {
      if (nc == 1) launch_pdl(op ? k_fluid_sc<S, 1, false, true> : k_fluid_sc<S, 1, false, false>, grd, blk, 0, s, a);
      else launch_pdl(op ? k_fluid_sc<S, 2, false, true> : k_fluid_sc<S, 2, false, false>, grd, blk, 0, s, a);
    }
  } else {
    if (nc == 1) {
      if (me) {
        if (a.pm) launch_local<S, 1, true, true, 0>(a, s);
        else launch_local<S, 1, true, false, 0>(a, s);
      } else if (a.sr_seed) {
        if (a.pm) launch_local<S, 1, false, true, 2>(a, s);
        else launch_local<S, 1, false, false, 2>(a, s);
      } else {
        if (a.pm) launch_local<S, 1, false, true, 1>(a, s);
        else launch_local<S, 1, false, false, 1>(a, s);
      }
    } else {
      launch_local<S, 2, true, false, 0>(a, s);
    }
  }
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace

int launch_fluid(int storage, int nc, bool sc, bool mass_exact, const FluidArgs &a, cudaStream_t s) {
  switch (storage) {
    case ST_FP16: return launch_fluid_t<__half>(nc, sc, mass_exact, a, s);
    case ST_BF16: return launch_fluid_t<__nv_bfloat16>(nc, sc, mass_exact, a, s);
    default: return launch_fluid_t<float>(nc, sc, mass_exact, a, s);
  }
}

template <class S, int SR>
int launch_fluid_solute_t(int q, const FluidArgs &a, const SoluteArgs &sa, cudaStream_t s) {
  dim3 blk(32, LOC_BY), grd((a.g.nx + 31) / 32, (a.g.chi - a.g.clo + LOC_BY - 1) / LOC_BY);
  if (a.slip) {
    if (q == 4) launch_pdl(k_fluid_solute<S, SR, 4, true>, grd, blk, 0, s, a, sa);
    else launch_pdl(k_fluid_solute<S, SR, 9, true>, grd, blk, 0, s, a, sa);
  } else {
    if (q == 4) launch_pdl(k_fluid_solute<S, SR, 4, false>, grd, blk, 0, s, a, sa);
    else launch_pdl(k_fluid_solute<S, SR, 9, false>, grd, blk, 0, s, a, sa);
  }
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_fluid_solute(int storage, int q, const FluidArgs &a, const SoluteArgs &sa, cudaStream_t s) {
  switch (storage) {
    case ST_FP16:
      return a.sr_seed ? launch_fluid_solute_t<__half, 2>(q, a, sa, s) : launch_fluid_solute_t<__half, 1>(q, a, sa, s);
    case ST_BF16:
      return a.sr_seed ? launch_fluid_solute_t<__nv_bfloat16, 2>(q, a, sa, s)
                       : launch_fluid_solute_t<__nv_bfloat16, 1>(q, a, sa, s);
    default: return launch_fluid_solute_t<float, 1>(q, a, sa, s);
  }
}

int launch_nbcode(const uint32_t *mask, uint16_t *nbc, const Geometry &g, cudaStream_t s, int r0, int r1) {
  if (r1 < 0) r1 = g.ny;
  if (r1 <= r0) return 0;
  dim3 blk(32, 8), grd(g.pitch / 32, (r1 - r0 + 7) / 8);
  k_nbcode<<<grd, blk, 0, s>>>(mask, nbc, g, r0, r1);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_gradient(int storage, const GradArgs &a, cudaStream_t s) {
  if (!a.nopen || a.maxlen <= 0) return 0;
  dim3 blk(128), grd((a.maxlen + 127) / 128, a.nopen);
  switch (storage) {
    case ST_FP16: launch_pdl(k_gradient<__half>, grd, blk, 0, s, a); break;
    case ST_BF16: launch_pdl(k_gradient<__nv_bfloat16>, grd, blk, 0, s, a); break;
    default: launch_pdl(k_gradient<float>, grd, blk, 0, s, a); break;
  }
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace lbk
