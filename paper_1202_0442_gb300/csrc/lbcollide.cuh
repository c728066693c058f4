// lbcollide.cuh -- the per-node part of a fluid iteration shared by the
// fluid kernels: moments, forces, equilibrium velocity, BGK collision and
// the stores (collide_store), and the inlet/outlet rules on opening nodes
// (apply_openings).  The kernels differ only in where the pulled
// populations come from.
#pragma once

#include "lbdev.cuh"

namespace lbk {

namespace {

// random word for (node, component, direction, step)
__device__ __forceinline__ uint32_t rnd(uint32_t seed, int self, int c, int i) {
  return mix32(((uint32_t)self * 0x9e3779b1u) ^ (seed + 0x632be5abu * (uint32_t)c) ^
               (0x85ebca6bu * (uint32_t)(i + 1)));
}

// momentum sum_i e_i f_i of one component as an unevaluated sum hi + lo,
// every addition error-free (two_sum): a moment rounded to FP32 feeds its
// rounding error back into the state as a spurious force (the collision
// relaxes toward the computed momentum), which in slow force-driven flows
// is comparable with the force itself
__device__ __forceinline__ void momentum_exact(const float (&f)[9], float &jx, float &jxl, float &jy,
                                               float &jyl) {
  float a, ea, b, eb, d, ed, s, es, t, et;
  two_sum(f[1], -f[3], a, ea);
  two_sum(f[5], -f[7], b, eb);
  two_sum(f[8], -f[6], d, ed);
  two_sum(a, b, s, es);
  two_sum(s, d, t, et);
  jx = t;
  jxl = ((ea + eb) + (ed + es)) + et;
  two_sum(f[2], -f[4], a, ea);
  two_sum(f[5], -f[7], b, eb);
  two_sum(f[6], -f[8], d, ed);
  two_sum(a, b, s, es);
  two_sum(s, d, t, et);
  jy = t;
  jyl = ((ea + eb) + (ed + es)) + et;
}

// moments, forces, equilibrium velocity, BGK and the stores of one node.
// Fsc: interforce already evaluated (zero when off).  ME: mass-exact
// collision (see below).  PM: the momentum as an exact hi + lo sum (single
// component; the storage flag LB_PRECISE_MOMENTUM).  FOLD (scaled 16-bit
// storage, not ME): h arrives and leaves in the stored units 2^s h, so the
// loads and stores skip their scale factors; the moments are unscaled once
// and the equilibrium is formed directly in stored units.  SR: 0 read
// p.sr_seed, 1 round to nearest, 2 stochastic rounding.
template <class S, int NC, bool ME, bool PM = false, bool FOLD = false, int SR = 0>
__device__ __forceinline__ void collide_store(const FluidArgs &p, int x, int y, uint32_t bits,
                                              float (&h)[NC][9], const float (&Fsc)[NC][2],
                                              float *uo = nullptr) {
  const Geometry &g = p.g;
  const int self = y * g.pitch + x;
  // the node's slot in the whole lattice: the random words are the same
  // whether the lattice is held whole or in slabs
  const int hself = self + g.yoff * g.pitch;
  const int P = (int)g.plane;
  float drho[NC], rho[NC], jx[NC], jy[NC], jxl[NC], jyl[NC], Fx[NC], Fy[NC];
  // stored units -> physical units (a power of two: exact)
  const float un = FOLD ? p.inv_scale : 1.0f;
#pragma unroll
  for (int c = 0; c < NC; c++) {
    const float(&f)[9] = h[c];
    drho[c] = (((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8]) * un;
    rho[c] = p.rho_ref[c] + drho[c];
    if (PM && NC == 1) {
      momentum_exact(f, jx[c], jxl[c], jy[c], jyl[c]);
    } else {
      jx[c] = (f[1] - f[3]) + (f[5] - f[7]) + (f[8] - f[6]);
      jy[c] = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
      jxl[c] = jyl[c] = 0.f;
    }
    jx[c] *= un;
    jy[c] *= un;
    jxl[c] *= un;
    jyl[c] *= un;
    Fx[c] = p.fx[c] + rho[c] * p.ax[c] + Fsc[c][0];
    Fy[c] = p.fy[c] + rho[c] * p.ay[c] + Fsc[c][1];
    if (p.ads[c]) {
      float sx, sy;
      wall_sum(bits, sx, sy);
      const float psi = (NC == 1) ? p.ads_psi0[c] * expf(-p.ads_rho0[c] / rho[c]) : rho[c];
      Fx[c] -= p.Gads[c] * psi * sx;
      Fy[c] -= p.Gads[c] * psi * sy;
    }
  }
  // equilibrium velocity (velocity shift) and the momentum rho u_eq it
  // carries, the latter formed without a division
  float uex[NC], uey[NC], mxt[NC], myt[NC];
  if (NC == 1) {
    mxt[0] = PM ? jx[0] + (jxl[0] + p.tau[0] * Fx[0]) : jx[0] + p.tau[0] * Fx[0];
    myt[0] = PM ? jy[0] + (jyl[0] + p.tau[0] * Fy[0]) : jy[0] + p.tau[0] * Fy[0];
    const float ir = 1.0f / rho[0];
    uex[0] = mxt[0] * ir;
    uey[0] = myt[0] * ir;
  } else {
    // common velocity sum(j/tau) / sum(rho/tau), shifted per component
    float nxs = 0.f, nys = 0.f, den = 0.f;
#pragma unroll
    for (int c = 0; c < NC; c++) {
      nxs += jx[c] * p.omega[c];
      nys += jy[c] * p.omega[c];
      den += rho[c] * p.omega[c];
    }
    const float upx = nxs / den, upy = nys / den;
#pragma unroll
    for (int c = 0; c < NC; c++) {
      mxt[c] = rho[c] * upx + p.tau[c] * Fx[c];
      myt[c] = rho[c] * upy + p.tau[c] * Fy[c];
      uex[c] = upx + p.tau[c] * Fx[c] / rho[c];
      uey[c] = upy + p.tau[c] * Fy[c] / rho[c];
    }
  }
#pragma unroll
  for (int c = 0; c < NC; c++) {
    S *out = (S *)p.fout + (size_t)c * 9 * P;
    float heq[9];
    if (FOLD) {
      // the equilibrium is linear in (drho, rho, rho u): in stored units
      // it takes 2^s drho, 2^s rho and 2^s rho u at the same velocity
      const float sc = p.scale;
      equilibrium_pairs(drho[c] * sc, rho[c] * sc, uex[c], uey[c], mxt[c] * sc, myt[c] * sc, p.wa[c],
                        p.wd[c], heq);
    } else {
      equilibrium_pairs(drho[c], rho[c], uex[c], uey[c], mxt[c], myt[c], p.wa[c], p.wd[c], heq);
    }
    const float om = p.omega[c];
    if (!ME && SR == 2) {
      // stochastic rounding: one hash per node and component, then a
      // linear congruential sequence, one step per pair of stores (each
      // state is uniform for a uniformly random start, so both dithers of
      // the paired conversion are uniform: unbiased rounding); the ninth
      // store takes the single conversion's high bits
      uint32_t r = rnd(p.sr_seed, hself, c, 0);
      const float sc = FOLD ? 1.0f : p.scale;
#pragma unroll
      for (int i = 0; i < 8; i += 2) {
        const float v0 = (h[c][i] + om * (heq[i] - h[c][i])) * sc;
        const float v1 = (h[c][i + 1] + om * (heq[i + 1] - h[c][i + 1])) * sc;
        r = r * 1664525u + 1013904223u;
        Store<S>::st2_dither(out, i * P + self, (i + 1) * P + self, v0, v1, r);
      }
      r = r * 1664525u + 1013904223u;
      Store<S>::st_dither(out, 8 * P + self, (h[c][8] + om * (heq[8] - h[c][8])) * sc, r);
    } else if (!ME && SR == 1) {
#pragma unroll
      for (int i = 0; i < 9; i++)
        Store<S>::st(out, i * P + self, h[c][i] + om * (heq[i] - h[c][i]), FOLD ? 1.0f : p.scale);
    } else if (!ME) {
      uint32_t r = p.sr_seed ? rnd(p.sr_seed, hself, c, 0) : 0u;
#pragma unroll
      for (int i = 0; i < 9; i++) {
        // dither of the 16-bit stores: one hash per node and component,
        // then a linear congruential sequence (its high bits) per direction
        r = r * 1664525u + 1013904223u;
        Store<S>::st(out, i * P + self, h[c][i] + om * (heq[i] - h[c][i]), p.scale,
                     p.sr_seed ? (r >> 13) | 1u : 0u);
      }
    } else {
      // Mass-exact collision: when |h| is large (two components, or one far
      // from rho_ref) the rounding of nine stored values of a slowly
      // changing state repeats every step and drifts the mass.  Here the
      // exact sum D of the pulled values and the exact sum S of the eight
      // stored moving populations are formed with error-free sums, and the
      // rest population is set to D - S -- the BGK value in exact
      // arithmetic -- rounded stochastically, so the node's mass is kept
      // up to an unbiased last-bit step.
      float Dh = h[c][0], Dl = 0.f;
#pragma unroll
      for (int i = 1; i < 9; i++) {
        float s, e;
        two_sum(Dh, h[c][i], s, e);
        Dh = s;
        Dl += e;
      }
      float Sh = 0.f, Sl = 0.f;
#pragma unroll
      for (int i = 1; i < 9; i++) {
        // 16-bit dither: an independent hash per store (a linear
        // congruential sequence per node, as in the plain collision, was
        // measurably worse for the two-component runs)
        const uint32_t r = p.sr_seed ? (rnd(p.sr_seed, hself, c, i) | 1u) : 0u;
        const float v = Store<S>::st_ret(out, i * P + self, h[c][i] + om * (heq[i] - h[c][i]),
                                         p.scale, p.inv_scale, r);
        float s, e;
        two_sum(Sh, v, s, e);
        Sh = s;
        Sl += e;
      }
      float rh, rl;
      two_sum(Dh, -Sh, rh, rl);
      rl += Dl - Sl;
      float h0, rem;
      two_sum(rh, rl, h0, rem);
      if (rem != 0.f && h0 != 0.f) {
        const int step = ((rem > 0.f) == (h0 > 0.f)) ? 1 : -1;
        const float nxt = __int_as_float(__float_as_int(h0) + step);
        // |nxt - h0| is a power of two, so the quotient is exact up to the
        // fast division's last bit: a probability, compared with a uniform
        // variate
        const float pr = __fdividef(fabsf(rem), fabsf(nxt - h0));
        const float u01 = (float)(rnd(p.step_seed, hself, c, 9) >> 8) * (1.0f / 16777216.0f);
        if (u01 < pr) h0 = nxt;
      }
      const uint32_t r0 = p.sr_seed ? (rnd(p.sr_seed, hself, c, 0) | 1u) : 0u;
      Store<S>::st(out, self, h0, p.scale, r0);
    }
    if (p.fields) {
      float *fl = p.fields + (size_t)c * NFIELD * P;
      fl[self] = drho[c];
      fl[P + self] = jx[c] + (jxl[c] + 0.5f * Fx[c]);
      fl[2 * P + self] = jy[c] + (jyl[c] + 0.5f * Fy[c]);
      // sum of the equilibrium populations (Mass_eq of the thermo command)
      fl[3 * P + self] = (heq[0] + ((heq[1] + heq[3]) + (heq[2] + heq[4])) +
                          ((heq[5] + heq[7]) + (heq[6] + heq[8]))) * un;
    }
  }
  if (p.uout || uo) {
    // the solvent velocity of Eq. (4)
    float pxs = 0.f, pys = 0.f, rs = 0.f;
#pragma unroll
    for (int c = 0; c < NC; c++) {
      pxs += jx[c] + (jxl[c] + 0.5f * Fx[c]);
      pys += jy[c] + (jyl[c] + 0.5f * Fy[c]);
      rs += rho[c];
    }
    const float vx = pxs / rs, vy = pys / rs;
    if (uo) {
      uo[0] = vx;
      uo[1] = vy;
    }
    if (p.uout) {
      p.uout[self] = vx;
      p.uout[P + self] = vy;
    }
  }
}

// component c's opening rule at node (x, y) if an opening holds it (the
// rule of a component reads only that component's populations, so the
// interforce kernel applies it per component, to its own node and to the
// ring nodes whose densities it stages); h in unscaled units
__device__ __forceinline__ void apply_opening_c(const FluidArgs &p, int c, int x, int y, float (&h)[9]) {
  const Geometry &g = p.g;
  const int gy = grow(g, y);
  if (!(x == 0 || gy == 0 || x == g.nx - 1 || gy == g.gny - 1)) return;
#pragma unroll 1
  for (int k = 0; k < p.nopen; k++) {
    if (!opening_has(p.span[k], x, gy, g.nx, g.gny)) continue;
    apply_opening(p.span[k], p.rule[k], c, h, x, gy, p.rho_ref[c]);
    return;
  }
}

template <int NC>
__device__ __forceinline__ void apply_openings(const FluidArgs &p, int x, int y,
                                               float (&h)[NC][9], float sc = 1.0f) {
  const Geometry &g = p.g;
  const int gy = grow(g, y);  // openings are placed on the whole lattice
  if (!(x == 0 || gy == 0 || x == g.nx - 1 || gy == g.gny - 1)) return;
#pragma unroll 1
  for (int k = 0; k < p.nopen; k++) {
    if (!opening_has(p.span[k], x, gy, g.nx, g.gny)) continue;
#pragma unroll
    for (int c = 0; c < NC; c++) apply_opening(p.span[k], p.rule[k], c, h[c], x, gy, p.rho_ref[c], sc);
    break;
  }
}

}  // namespace

}  // namespace lbk
