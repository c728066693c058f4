// lbsolute.cuh -- the per-node part of a solute iteration (solute command,
// Eq. (3); surface_reaction, App. C; inlet_solute/outlet_solute, App. B),
// shared by the solute kernels and the fused fluid-solute kernel.
#pragma once

#include "lbdev.cuh"

namespace lbk {

namespace {

template <int Q> __device__ __forceinline__ constexpr int sex(int i) { return Q == 4 ? EX4(i) : EX(i); }
template <int Q> __device__ __forceinline__ constexpr int sey(int i) { return Q == 4 ? EY4(i) : EY(i); }
template <int Q> __device__ __forceinline__ constexpr int sopp(int i) { return Q == 4 ? OPP4(i) : OPP(i); }
template <int Q> __device__ __forceinline__ constexpr float sw(int i) { return Q == 4 ? 0.25f : W9(i); }

// which opening (if any) holds node (x, y)
__device__ __forceinline__ int opening_of(const OpenSpan *sp, int nopen, int x, int y, int nx, int ny) {
  if (!(x == 0 || y == 0 || x == nx - 1 || y == ny - 1)) return -1;
  for (int k = 0; k < nopen; k++)
    if (opening_has(sp[k], x, y, nx, ny)) return k;
  return -1;
}

// Streamed populations of node (x, y): pull from x - e_i; at a solid source
// bounce-back, or the reaction rule on that link (then Ci is added to Cw,
// the link counted in nU and flagged in U).  Modes crossing the wall of an
// opening node (wall >= 0) are left 0 and flagged in `cross`.
// `bits`: the node's 3 x 3 solid neighbourhood (bit NBPOS(dx, dy)).
template <int Q>
__device__ __forceinline__ void solute_pull(const SoluteArgs &p, int x, int y, int wall, uint32_t bits,
                                            float (&gt)[Q], float &Cw, int &nU, uint32_t &U, uint32_t &cross) {
  const Geometry &g = p.g;
  const int self = y * g.pitch + x;
  const int xm = x ? x - 1 : g.nx - 1, xp = (x + 1 == g.nx) ? 0 : x + 1;
  const int rm = (y ? y - 1 : g.ny - 1) * g.pitch, r0 = y * g.pitch, rp = ((y + 1 == g.ny) ? 0 : y + 1) * g.pitch;
  const int P = (int)g.plane;
  Cw = 0.f;
  nU = 0;
  U = 0;
  cross = 0;
#pragma unroll
  for (int i = 0; i < Q; i++) {
    const int ex = sex<Q>(i), ey = sey<Q>(i);
    if (wall >= 0 && crosses_wall(wall, ex, ey)) {
      cross |= 1u << i;
      gt[i] = 0.f;
      continue;
    }
    if ((bits >> NBPOS(-ex, -ey)) & 1u) {
      const float gout = __ldg(p.gin + sopp<Q>(i) * P + self);
      if (p.react) {
        // (2 g_out + kr Cs) / (kr + 2 w_i), the denominator's reciprocal
        // precomputed per weight class
        const float Ci = (2.0f * gout + p.kr * p.Cs) * (Q == 4 ? p.rden[0] : (i < 5 ? p.rden[0] : p.rden[1]));
        gt[i] = -gout + 2.0f * sw<Q>(i) * Ci;
        Cw += Ci;
        nU++;
        U |= 1u << i;
      } else {
        gt[i] = gout;
      }
    } else {
      const int xs = ex > 0 ? xm : (ex < 0 ? xp : x);
      const int rs = ey > 0 ? rm : (ey < 0 ? rp : r0);
      gt[i] = __ldg(p.gin + i * P + rs + xs);
    }
  }
}

// 3 x 3 solid neighbourhood of node (x, y), x < pitch, y < ny: its
// neighbour code (slots past nx read as solid)
__device__ __forceinline__ uint32_t solute_bits(const SoluteArgs &p, int x, int y) {
  return __ldg(p.nbc + (size_t)y * p.g.pitch + x);
}

// concentration of node (x, y) right after streaming, before any opening
// rule (0 on solid nodes): the C1 of the flux rule
template <int Q>
__device__ float solute_streamed_C(const SoluteArgs &p, int x, int y) {
  const Geometry &g = p.g;
  if (solid_at(p.mask, g.mw, x, y)) return 0.f;
  const int k = p.nopen ? opening_of(p.span, p.nopen, x, grow(g, y), g.nx, g.gny) : -1;
  float gt[Q], Cw;
  int nU;
  uint32_t U, cross;
  solute_pull<Q>(p, x, y, k >= 0 ? span_wall(p.span[k]) : -1, solute_bits(p, x, y), gt, Cw, nU, U, cross);
  float C = 0.f;
#pragma unroll
  for (int i = 0; i < Q; i++) C += gt[i];
  return C;
}

// inlet_solute/outlet_solute rules (App. B) on an opening node.
// dirichlet: the crossing modes make C = Cbar (split by weight); adiabatic:
// crossing mode = opposite mode; flux: C from the flux balance with the
// nearest inner node, C = (v C0 + D C1)/(D + v) (inlet) or
// (v C0 - D C1)/(v - D) (outlet), every mode then at equilibrium (the
// caller sets them; returns true and the C to use).
template <int Q>
__device__ __forceinline__ bool solute_openings(const SoluteArgs &p, const OpenDesc &o, int x, int y,
                                                float (&gt)[Q], uint32_t cross, float &Cflux) {
  if (o.sstyle == SOL_DIRICHLET) {
    float Cp = 0.f, ws = 0.f;
#pragma unroll
    for (int i = 0; i < Q; i++) {
      if (cross & (1u << i)) ws += sw<Q>(i);
      else Cp += gt[i];
    }
    const float r = (o.Cbar - Cp) / ws;
#pragma unroll
    for (int i = 0; i < Q; i++)
      if (cross & (1u << i)) gt[i] = r * sw<Q>(i);
  } else if (o.sstyle == SOL_ADIABATIC) {
#pragma unroll
    for (int i = 0; i < Q; i++)
      if (cross & (1u << i)) gt[i] = gt[sopp<Q>(i)];
  } else if (o.sstyle == SOL_FLUX) {
    // inward normal: xlo +x, xhi -x, ylo +y, yhi -y
    const int xi = wrapi(x + (o.wall == 0 ? 1 : o.wall == 1 ? -1 : 0), p.g.nx);
    const int yi = wrapi(y + (o.wall == 2 ? 1 : o.wall == 3 ? -1 : 0), p.g.ny);
    const float C1 = solute_streamed_C<Q>(p, xi, yi);
    const float v = o.sv, C0 = o.Cbar, D = p.D;
    Cflux = (o.kind == 0) ? (v * C0 + D * C1) / (D + v) : (v * C0 - D * C1) / (v - D);
    return true;
  }
  return false;
}

// g_eq(C, u) of Eq. (3) (D2Q4) or w_i C (1 + 3 e.u) (D2Q9)
template <int Q>
__device__ __forceinline__ void solute_geq(float C, float ux, float uy, float (&geq)[Q]) {
#pragma unroll
  for (int i = 0; i < Q; i++) {
    const float eu = (float)sex<Q>(i) * ux + (float)sey<Q>(i) * uy;
    geq[i] = Q == 4 ? 0.25f * C * (1.0f + 2.0f * eu) : sw<Q>(i) * C * (1.0f + 3.0f * eu);
  }
  if (Q == 9) {
    // the rounded D2Q9 weights would bias sum g_eq and sum g_eq e (see
    // equilibrium_pairs); restore C and C u
    const float mx = geq[1] - geq[3] + geq[5] - geq[6] - geq[7] + geq[8];
    const float my = geq[2] - geq[4] + geq[5] + geq[6] - geq[7] - geq[8];
    const float cx = 0.5f * (C * ux - mx), cy = 0.5f * (C * uy - my);
    geq[1] += cx;
    geq[3] -= cx;
    geq[2] += cy;
    geq[4] -= cy;
    float m = 0.f;
#pragma unroll
    for (int i = 1; i < Q; i++) m += geq[i];
    geq[0] = C - m;
  }
}

// intersolute pseudopotential psi = psi0 exp(-C0/C); 0 on solid nodes and
// where C <= 0
__device__ __forceinline__ float solute_psi(const SoluteArgs &p, float C) {
  return C > 0.f ? p.ispsi0 * expf(-p.isC0 / C) : 0.f;
}

// One solute node update of fluid node (x, y): pull with bounce-back or the
// reaction rule, the opening rules, BGK with g_eq(C, u_s), precipitation;
// (ux, uy) is the node's solvent velocity of this iteration (Eq. (4)).
template <int Q>
__device__ __forceinline__ void solute_node(const SoluteArgs &p, int x, int y, uint32_t bits, float ux,
                                            float uy) {
  const Geometry &g = p.g;
  const size_t self = (size_t)y * g.pitch + x;
  const int k = p.nopen ? opening_of(p.span, p.nopen, x, grow(g, y), g.nx, g.gny) : -1;
  float gt[Q], Cw, Cflux = 0.f;
  int nU;
  uint32_t U, cross;
  solute_pull<Q>(p, x, y, k >= 0 ? span_wall(p.span[k]) : -1, bits, gt, Cw, nU, U, cross);
  bool flux = false;
  if (k >= 0) flux = solute_openings<Q>(p, p.op[k], x, y, gt, cross, Cflux);
  float C = 0.f;
#pragma unroll
  for (int i = 0; i < Q; i++) C += gt[i];
  if (flux) C = Cflux;
  if (p.inter && C > 0.f) {
    // intersolute: u_s = u + tau_s F / C, F = -G psi(x) sum_{i=1..4}
    // psi(x + e_i) e_i over the D2Q4 neighbours (their concentrations of
    // this step, from the first pass)
    float Fx = 0.f, Fy = 0.f;
#pragma unroll
    for (int d = 0; d < 4; d++) {
      const int xn = wrapi(x + EX4(d), g.nx), yn = wrapi(y + EY4(d), g.ny);
      const float psin = solid_at(p.mask, g.mw, xn, yn)
                             ? 0.f
                             : solute_psi(p, __ldg(p.Cpre + (size_t)yn * g.pitch + xn));
      Fx += psin * (float)EX4(d);
      Fy += psin * (float)EY4(d);
    }
    const float f = -p.isG * solute_psi(p, C);
    ux += p.taus * f * Fx / C;
    uy += p.taus * f * Fy / C;
  }
  const float om = p.omega;
  float geq[Q];
  solute_geq<Q>(C, ux, uy, geq);
  if (flux) {
#pragma unroll
    for (int i = 0; i < Q; i++) gt[i] = geq[i];
  }
  float gs[Q];
#pragma unroll
  for (int i = 0; i < Q; i++) gs[i] = gt[i] + om * (geq[i] - gt[i]);
  if (p.react && nU) {
    const float share_n = nU == 1 ? 1.0f : nU == 2 ? 0.5f : nU == 3 ? (1.0f / 3.0f) : nU == 4 ? 0.25f : 1.0f / (float)nU;
    const float dB = p.kr * (Cw * share_n - p.Cs);
    float share = 0.f;
    if (dB > 0.f) {
      share = dB * share_n;
#pragma unroll
      for (int i = 0; i < Q; i++)
        if (U & (1u << i)) gs[i] -= share;
    }
    p.db[self] = share;
  }
  float Cn = 0.f;
#pragma unroll
  for (int i = 0; i < Q; i++) {
    p.gout[(size_t)i * g.plane + self] = gs[i];
    Cn += gs[i];
  }
  if (p.Cfield) p.Cfield[self] = Cn;
}

}  // namespace

}  // namespace lbk
