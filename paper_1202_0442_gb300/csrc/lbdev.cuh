// lbdev.cuh -- device-side building blocks shared by the library's kernels.
//
// Lattice: D2Q9 with e0=(0,0) e1=(1,0) e2=(0,1) e3=(-1,0) e4=(0,-1)
// e5=(1,1) e6=(-1,1) e7=(-1,-1) e8=(1,-1) -- the numbering the unknown-mode
// sets of the paper's inlet/outlet rules require (xlo: 1,5,8; xhi: 3,6,7;
// ylo: 2,5,6; yhi: 4,7,8; inlet_momentum command and App. A).  Solute D2Q4
// g1..g4 = +x,+y,-x,-y at index 0..3 (solute command, App. B/C).
//
// HBM layout (all planes share one pitch, a multiple of 32 nodes):
//   populations  [buffer 2][component][q][ny][pitch]  storage type S
//   mask         [ny][pitch/32] uint32, bit x%32 of word x/32, 1 = solid
//   node fields  float planes [ny][pitch]
// Populations are stored as deviations h_i = f_i - w_i rho_ref (times 2^s
// for FP16) and all arithmetic is FP32.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbint.h"

namespace lbk {

__host__ __device__ constexpr int EX(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0;
}
__host__ __device__ constexpr int EY(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0;
}
__host__ __device__ constexpr int OPP(int i) {
  return i == 0 ? 0 : i == 1 ? 3 : i == 2 ? 4 : i == 3 ? 1 : i == 4 ? 2
       : i == 5 ? 7 : i == 6 ? 8 : i == 7 ? 5 : 6;
}
__host__ __device__ constexpr float W9(int i) {
  return i == 0 ? 4.0f / 9.0f : (i < 5 ? 1.0f / 9.0f : 1.0f / 36.0f);
}
// D2Q4 solute directions at index 0..3
__host__ __device__ constexpr int EX4(int i) { return i == 0 ? 1 : i == 2 ? -1 : 0; }
__host__ __device__ constexpr int EY4(int i) { return i == 1 ? 1 : i == 3 ? -1 : 0; }
__host__ __device__ constexpr int OPP4(int i) { return (i + 2) & 3; }

// ---------------------------------------------------------------------
// population storage
// ---------------------------------------------------------------------
template <class S> struct Store;
template <> struct Store<float> {
  static constexpr bool kScaled = false;  // stored values carry no 2^s factor
  static __device__ __forceinline__ void st_dither(float *p, size_t k, float v, uint32_t) { p[k] = v; }
  static __device__ __forceinline__ float ld(const float *p, size_t k, float) {
    return __ldg(p + k);
  }
  static __device__ __forceinline__ float ld_smem(const float *p, int k, float) { return p[k]; }
  static __device__ __forceinline__ void st(float *p, size_t k, float v, float) {
    p[k] = v;
  }
  static __device__ __forceinline__ void st(float *p, size_t k, float v, float, uint32_t) {
    p[k] = v;
  }
  // store and return the value as it now reads back
  static __device__ __forceinline__ float st_ret(float *p, size_t k, float v, float, float,
                                                 uint32_t) {
    p[k] = v;
    return v;
  }
  static __device__ __forceinline__ void st2_dither(float *p, size_t k0, size_t k1, float v0, float v1,
                                                    uint32_t) {
    p[k0] = v0;
    p[k1] = v1;
  }
};
// 16-bit stores take an optional 32-bit random word r: with r = 0 they
// round to nearest even; otherwise r's low bits are added below the
// format's last kept bit before truncation (stochastic rounding).  A value
// that stays nearly the same from step to step then no longer rounds the
// same way every step, which would otherwise act as a steady bias.
template <> struct Store<__half> {
  static constexpr bool kScaled = true;
  // v already scaled; d: a random word, its top 13 bits dither the 13
  // fraction bits binary16 drops (stochastic rounding)
  static __device__ __forceinline__ void st_dither(__half *p, size_t k, float v, uint32_t d) {
    p[k] = __float2half_rz(__uint_as_float(__float_as_uint(v) + (d >> 19)));
  }
  static __device__ __forceinline__ float ld(const __half *p, size_t k, float inv) {
    return __half2float(__ldg(p + k)) * inv;
  }
  static __device__ __forceinline__ float ld_smem(const __half *p, int k, float inv) {
    return __half2float(p[k]) * inv;
  }
  static __device__ __forceinline__ void st(__half *p, size_t k, float v, float sc) {
    p[k] = __float2half_rn(v * sc);
  }
  static __device__ __forceinline__ void st(__half *p, size_t k, float v, float sc, uint32_t r) {
    if (!r) {
      p[k] = __float2half_rn(v * sc);
      return;
    }
    // binary16 keeps 10 of FP32's 23 fraction bits: dither the low 13
    const uint32_t b = __float_as_uint(v * sc) + (r & 0x1fffu);
    p[k] = __float2half_rz(__uint_as_float(b));
  }
  static __device__ __forceinline__ float st_ret(__half *p, size_t k, float v, float sc, float inv,
                                                 uint32_t r) {
    const __half q = r ? __float2half_rz(__uint_as_float(__float_as_uint(v * sc) + (r & 0x1fffu)))
                       : __float2half_rn(v * sc);
    p[k] = q;
    return __half2float(q) * inv;
  }
  // two values (already scaled) rounded stochastically by one paired
  // conversion (cvt.rs.f16x2.f32, sm_100 and later): bits 0-12 of r dither
  // v0, bits 16-28 dither v1; v0 goes to slot k0, v1 to slot k1
  static __device__ __forceinline__ void st2_dither(__half *p, size_t k0, size_t k1, float v0, float v1,
                                                    uint32_t r) {
    uint32_t d;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(v1), "f"(v0), "r"(r));
    p[k0] = __ushort_as_half((unsigned short)(d & 0xffffu));
    p[k1] = __ushort_as_half((unsigned short)(d >> 16));
  }
};
template <> struct Store<__nv_bfloat16> {
  static constexpr bool kScaled = false;
  // d: a random word, its top 16 bits dither the 16 fraction bits bfloat16
  // drops (stochastic rounding)
  static __device__ __forceinline__ void st_dither(__nv_bfloat16 *p, size_t k, float v, uint32_t d) {
    p[k] = __float2bfloat16_rz(__uint_as_float(__float_as_uint(v) + (d >> 16)));
  }
  static __device__ __forceinline__ float ld(const __nv_bfloat16 *p, size_t k, float) {
    return __bfloat162float(__ldg(p + k));
  }
  static __device__ __forceinline__ float ld_smem(const __nv_bfloat16 *p, int k, float) {
    return __bfloat162float(p[k]);
  }
  static __device__ __forceinline__ void st(__nv_bfloat16 *p, size_t k, float v, float) {
    p[k] = __float2bfloat16_rn(v);
  }
  static __device__ __forceinline__ void st(__nv_bfloat16 *p, size_t k, float v, float, uint32_t r) {
    if (!r) {
      p[k] = __float2bfloat16_rn(v);
      return;
    }
    // bfloat16 keeps 7 fraction bits: dither the low 16
    const uint32_t b = __float_as_uint(v) + (r & 0xffffu);
    p[k] = __float2bfloat16_rz(__uint_as_float(b));
  }
  static __device__ __forceinline__ float st_ret(__nv_bfloat16 *p, size_t k, float v, float, float,
                                                 uint32_t r) {
    const __nv_bfloat16 q = r ? __float2bfloat16_rz(__uint_as_float(__float_as_uint(v) + (r & 0xffffu)))
                              : __float2bfloat16_rn(v);
    p[k] = q;
    return __bfloat162float(q);
  }
  // paired stochastic rounding (cvt.rs.bf16x2.f32): bits 0-15 of r dither
  // v0, bits 16-31 dither v1
  static __device__ __forceinline__ void st2_dither(__nv_bfloat16 *p, size_t k0, size_t k1, float v0, float v1,
                                                    uint32_t r) {
    uint32_t d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(v1), "f"(v0), "r"(r));
    p[k0] = __ushort_as_bfloat16((unsigned short)(d & 0xffffu));
    p[k1] = __ushort_as_bfloat16((unsigned short)(d >> 16));
  }
};

// integer hash (C. Wellons' "lowbias32"), used to draw the rounding dither
// from (node, direction, step)
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// ---------------------------------------------------------------------
// solid mask
// ---------------------------------------------------------------------
__device__ __forceinline__ int solid_at(const uint32_t *m, int mw, int x, int y) {
  return (int)((__ldg(m + (size_t)y * mw + (x >> 5)) >> (x & 31)) & 1u);
}

// row of the whole lattice of an updated local row y
__device__ __forceinline__ int grow(const Geometry &g, int y) { return y + g.yoff; }

// a mod n in [0, n)
__device__ __forceinline__ int wrapi(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

// Solid bits of the 3 x 3 neighbourhood of a node: bit (dy+1)*3 + (dx+1)
// is node (x+dx, y+dy); bit 4 is the node itself.
__host__ __device__ constexpr int NBPOS(int dx, int dy) { return (dy + 1) * 3 + (dx + 1); }

// neighbourhood bits read straight from the mask (any node, periodic wrap)
__device__ __forceinline__ uint32_t nbr_bits(const uint32_t *m, int mw, int x, int y,
                                             int xm, int xp, int ym, int yp) {
  const int xs[3] = {xm, x, xp}, ys[3] = {ym, y, yp};
  uint32_t b = 0;
#pragma unroll
  for (int j = 0; j < 3; j++)
#pragma unroll
    for (int i = 0; i < 3; i++) b |= (uint32_t)solid_at(m, mw, xs[i], ys[j]) << (j * 3 + i);
  return b;
}

// is node x + e_i solid (i = 1..8)
__device__ __forceinline__ int nb(uint32_t bits, int i) {
  return (bits >> NBPOS(EX(i), EY(i))) & 1;
}

// the three bits x-1, x, x+1 (as bits 0, 1, 2) of a mask row whose words
// around x are l (left), c (holding x) and r (right); lane = x % 32
__device__ __forceinline__ uint32_t row3(uint32_t l, uint32_t c, uint32_t r, int lane) {
  const uint64_t win = ((uint64_t)(r & 1u) << 33) | ((uint64_t)c << 1) | (uint64_t)(l >> 31);
  return (uint32_t)(win >> lane) & 7u;
}

// sum_i w_i s(x + e_i) e_i over the eight neighbours (adhesiveforce)
__device__ __forceinline__ void wall_sum(uint32_t bits, float &sx, float &sy) {
  const float a = 1.0f / 9.0f, d = 1.0f / 36.0f;
  sx = a * (float)(nb(bits, 1) - nb(bits, 3)) +
       d * (float)(nb(bits, 5) - nb(bits, 6) - nb(bits, 7) + nb(bits, 8));
  sy = a * (float)(nb(bits, 2) - nb(bits, 4)) +
       d * (float)(nb(bits, 5) + nb(bits, 6) - nb(bits, 7) - nb(bits, 8));
}

// ---------------------------------------------------------------------
// Equilibrium of Eq. (2), generalised by the fluids command to
// f_eq,i = w_i rho [A_i + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u] with A_0 = 9/4 alpha,
// A_{1..8} = 9/5 (1 - alpha), as deviations h_eq,i = f_eq,i - s_i rho_ref
// from the rest state s_i = w_i A_i (s_0 = alpha, wa = s_{1..4} =
// (1 - alpha)/5, wd = s_{5..8} = (1 - alpha)/20; 4/9, 1/9, 1/36 at
// alpha = 4/9), drho = rho - rho_ref, in symmetric/antisymmetric pairs
// (i, opp(i)):
//   A_i = s_i drho + w_i rho (9/2 (e_i.u)^2 - 3/2 u.u),  B_i = 3 w_i rho e_i.u
//   h_eq,i = A_i + B_i,  h_eq,opp(i) = A_i - B_i
// (sum_i s_i = 1, so h_eq,0 = drho - the other eight holds for any alpha)
// The rounded FP32 weights would make sum h_eq and sum h_eq e miss drho and
// rho u by a fixed relative 1e-8..1e-7, repeated by every collision (a
// spurious force proportional to the momentum).  So the two moments are
// imposed instead: the axis B's come from the target momentum (mx, my)
// minus the diagonal B's, and h_eq,0 from drho minus the other eight;
// in exact arithmetic both are the formula above.
// Output slots: heq[0..8] in direction order.
// ---------------------------------------------------------------------
__device__ __forceinline__ void equilibrium_pairs(float drho, float rho, float ux, float uy,
                                                  float mx, float my, float wa, float wd,
                                                  float (&heq)[9]) {
  const float q = rho * (ux * ux + uy * uy);
  const float sp = ux + uy, sm = uy - ux;  // e5.u and e6.u
  const float d9 = drho * wa, d36 = drho * wd;
  const float A1 = d9 + 0.5f * rho * ux * ux - q * (1.0f / 6.0f);
  const float A2 = d9 + 0.5f * rho * uy * uy - q * (1.0f / 6.0f);
  const float A5 = d36 + 0.125f * rho * sp * sp - q * (1.0f / 24.0f);
  const float A6 = d36 + 0.125f * rho * sm * sm - q * (1.0f / 24.0f);
  const float B5 = rho * sp * (1.0f / 12.0f);
  const float B6 = rho * sm * (1.0f / 12.0f);
  const float B1 = 0.5f * mx - B5 + B6;
  const float B2 = 0.5f * my - B5 - B6;
  heq[1] = A1 + B1;
  heq[3] = A1 - B1;
  heq[2] = A2 + B2;
  heq[4] = A2 - B2;
  heq[5] = A5 + B5;
  heq[7] = A5 - B5;
  heq[6] = A6 + B6;
  heq[8] = A6 - B6;
  heq[0] = drho - 2.0f * ((A1 + A2) + (A5 + A6));
}

// error-free sum: s + e == a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// ---------------------------------------------------------------------
// inlet/outlet rules in one rotated form.
//
// Every wall is mapped onto a canonical one whose inward normal n is e1 and
// tangent t is e2; canonical slot k then holds direction PERM[wall][k]:
//   k: 0  1=n  2=t  3=-n  4=-t  5=n+t  6=-n+t  7=-n-t  8=n-t
// With u_n the velocity along n, S = h0 + h2 + h4 + 2 (h3 + h6 + h7):
//   velocity styles:  rho = (rho_ref + S)/(1 - u_n)
//   dirichlet:        u_n = (rho - rho_ref - S)/rho
//   h1 = h3 + 2/3 rho u_n
//   h5 = h7 - (h2 - h4)/2 + rho u_n / 6
//   h8 = h6 + (h2 - h4)/2 + rho u_n / 6
// which is the set of printed rules for each wall and style (inlet: u_n =
// +v, outlet: u_n = -v), written for deviations h = f - w rho_ref.
// ---------------------------------------------------------------------
template <int WALL> __device__ __forceinline__ constexpr int PERM(int k) {
  // xlo: n=+x t=+y; xhi: n=-x t=+y; ylo: n=+y t=+x; yhi: n=-y t=-x
  return WALL == 0 ? k
       : WALL == 1 ? (k == 1 ? 3 : k == 3 ? 1 : k == 5 ? 6 : k == 6 ? 5 : k == 7 ? 8 : k == 8 ? 7 : k)
       : WALL == 2 ? (k == 1 ? 2 : k == 2 ? 1 : k == 3 ? 4 : k == 4 ? 3 : k == 6 ? 8 : k == 8 ? 6 : k)
                   : (k == 1 ? 4 : k == 2 ? 3 : k == 3 ? 2 : k == 4 ? 1 : k == 5 ? 7 : k == 7 ? 5 : k);
}

template <int WALL>
__device__ __forceinline__ void zou_he(float (&h)[9], bool dirichlet, float un_in,
                                       float drho_in, float rho_ref) {
  constexpr int c0 = PERM<WALL>(0), c1 = PERM<WALL>(1), c2 = PERM<WALL>(2),
                c3 = PERM<WALL>(3), c4 = PERM<WALL>(4), c5 = PERM<WALL>(5),
                c6 = PERM<WALL>(6), c7 = PERM<WALL>(7), c8 = PERM<WALL>(8);
  const float S = h[c0] + h[c2] + h[c4] + 2.0f * (h[c3] + h[c6] + h[c7]);
  float rho, un;
  if (dirichlet) {
    rho = rho_ref + drho_in;
    un = (drho_in - S) / rho;
  } else {
    un = un_in;
    rho = rho_ref + (S + rho_ref * un) / (1.0f - un);
  }
  const float a = rho * un;
  const float tdiff = 0.5f * (h[c2] - h[c4]);
  h[c1] = h[c3] + (2.0f / 3.0f) * a;
  h[c5] = h[c7] - tdiff + a * (1.0f / 6.0f);
  h[c8] = h[c6] + tdiff + a * (1.0f / 6.0f);
}

__device__ __forceinline__ int span_wall(const OpenSpan &s) { return s.wa0 & 3; }

__device__ __forceinline__ bool opening_has(const OpenSpan &s, int x, int y, int nx, int ny) {
  const int a0 = s.wa0 >> 2;
  switch (s.wa0 & 3) {
    case 0: return x == 0 && y >= a0 && y <= s.a1;
    case 1: return x == nx - 1 && y >= a0 && y <= s.a1;
    case 2: return y == 0 && x >= a0 && x <= s.a1;
    default: return y == ny - 1 && x >= a0 && x <= s.a1;
  }
}

// Poiseuille inlet profile: 4 vmax/L^2 [(L/2)^2 - ((2c - a1 - a0)/2)^2]
__device__ __forceinline__ float poiseuille(float vmax, int a0, int a1, int c) {
  const float L = (float)(a1 - a0 + 1);
  const float d = 0.5f * (float)(2 * c - a1 - a0);
  return 4.0f * vmax / (L * L) * (0.25f * L * L - d * d);
}

// apply the velocity/dirichlet rule r of the opening at s to component c's
// h; sc: the units h is in (the rule is homogeneous of degree one in h, drho
// and rho_ref, so scaled storage units take sc = 2^s)
__device__ __forceinline__ void apply_opening(const OpenSpan &s, const OpenRule &r, int c, float (&h)[9],
                                              int x, int y, float rho_ref, float sc = 1.0f) {
  const int st = (r.bits >> (3 * c)) & 7;
  if (st != OPEN_POISEUILLE && st != OPEN_UNIFORM && st != OPEN_DIRICHLET) return;
  const bool dir = (st == OPEN_DIRICHLET);
  const int wall = span_wall(s);
  float un = 0.0f, dr = 0.0f;
  if (!dir) {
    const int coord = (wall <= 1) ? y : x;
    const float v = (st == OPEN_UNIFORM) ? r.val[c] : poiseuille(r.val[c], s.wa0 >> 2, s.a1, coord);
    un = ((r.bits >> 6) & 1) == 0 ? v : -v;
  } else {
    dr = r.val[c];
  }
  switch (wall) {
    case 0: zou_he<0>(h, dir, un, dr * sc, rho_ref * sc); break;
    case 1: zou_he<1>(h, dir, un, dr * sc, rho_ref * sc); break;
    case 2: zou_he<2>(h, dir, un, dr * sc, rho_ref * sc); break;
    default: zou_he<3>(h, dir, un, dr * sc, rho_ref * sc); break;
  }
}

// does direction (ex, ey) arriving at a node of `wall` come from outside?
__device__ __forceinline__ bool crosses_wall(int wall, int ex, int ey) {
  return wall == 0 ? ex > 0 : wall == 1 ? ex < 0 : wall == 2 ? ey > 0 : ey < 0;
}

// SplitMix64 (Steele, Lea and Flood 2014): one step from state x
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

}  // namespace lbk
