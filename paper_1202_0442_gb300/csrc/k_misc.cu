// k_misc.cu -- thermo reduction and state conversion kernels.
//
// k_thermo_partial: the thermo command's sums (mass,
//   momentum j + F/2, equilibrium mass, solute, deposit, removed mass,
//   node counts) over the state at the end of an iteration.  The first
//   kernel gives every thread a fixed, strided set of nodes; a thread sums
//   the FP32 fields of its nodes as an unevaluated pair hi + lo of FP32
//   values with error-free additions (GB300's FP64 rate is a small fraction
//   of its FP32 rate, and a plain FP64 add per node and quantity made the
//   pass ALU-bound), counts nodes in integers and adds the FP64 arrays in
//   FP64; the block then reduces in FP64 with warp shuffles and one
//   shared-memory pass into a per-block slot of a scratch array, and the
//   last block to finish (a counter) reduces the slots in a fixed tree and
//   appends the flip count and the error word, so the host reads one
//   record.  The order of every addition is fixed by the launch shape, so
//   the result is the same bits on every run.
// Conversions between FP64 arrays in the caller's layout ([q][ny][nx],
// dense) and the library's storage (deviations from w_i rho_ref, pitched,
// FP32/FP16/BF16), equilibrium initialisation from rho and u, and field
// export.
#include "lbdev.cuh"
#include "lbpdl.cuh"

namespace lbk {

namespace {

constexpr int TB = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// hi + lo += v without rounding error in hi + lo's leading part (Knuth's
// two-sum; the rounding of lo's own additions is second order)
__device__ __forceinline__ void pair_add(float &hi, float &lo, float v) {
  const float s = hi + v;
  const float bb = s - hi;
  lo += (hi - (s - bb)) + (v - bb);
  hi = s;
}

// The final sums of the per-block slots: one warp per quantity, lanes
// striding over the blocks in a fixed order (four independent chains, so
// the loads overlap), then a shuffle tree.  L2 reads: other blocks wrote
// the slots during this launch.
__device__ __forceinline__ void thermo_final(const double *partials, int nblocks, double *out) {
  const int lane = threadIdx.x & 31;
  for (int q = threadIdx.x >> 5; q < NTHERMO; q += TB / 32) {
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
    int k = lane;
    for (; k + 96 < nblocks; k += 128) {
      v0 += __ldcg(partials + (size_t)k * NTHERMO + q);
      v1 += __ldcg(partials + (size_t)(k + 32) * NTHERMO + q);
      v2 += __ldcg(partials + (size_t)(k + 64) * NTHERMO + q);
      v3 += __ldcg(partials + (size_t)(k + 96) * NTHERMO + q);
    }
    for (; k < nblocks; k += 32) v0 += __ldcg(partials + (size_t)k * NTHERMO + q);
    double v = (v0 + v1) + (v2 + v3);
    v = warp_sum(v);
    if (lane == 0) out[q] = v;
  }
}

// Block b handles rows b, b + gridDim.x, ...; its threads stride over x.
// 64 registers keep THERMO_BLOCKS_PER_SM blocks per SM, so a grid of that
// many blocks per SM is resident at once.
// Quantities 0..8 come from FP32 planes and are summed per thread as FP32
// pairs; 9..12 are FP64 arrays (reaction runs only); 13, 14 are counts.
__global__ void __launch_bounds__(TB, THERMO_BLOCKS_PER_SM) k_thermo_partial(const ThermoArgs a) {
  dep_wait();
  const Geometry &g = a.g;
  float hi[9], lo[9];
#pragma unroll
  for (int q = 0; q < 9; q++) hi[q] = lo[q] = 0.f;
  double dacc[4] = {0.0, 0.0, 0.0, 0.0};
  unsigned nsolid = 0, nfluid = 0;
  const size_t P = g.plane;
  const float *f0 = a.fields;
  const float *f1 = a.nc > 1 ? a.fields + (size_t)NFIELD * P : nullptr;
  for (int y = g.ylo + blockIdx.x; y < g.yhi; y += gridDim.x) {
#pragma unroll 2
    for (int x = threadIdx.x; x < g.nx; x += TB) {
      const size_t self = (size_t)y * g.pitch + x;
      if (solid_at(a.mask, g.mw, x, y)) {
        nsolid++;
        if (a.b) dacc[0] += a.b[self];
      } else {
        nfluid++;
        pair_add(hi[0], lo[0], f0[self]);
        pair_add(hi[2], lo[2], f0[3 * P + self]);
        pair_add(hi[4], lo[4], f0[P + self]);
        pair_add(hi[5], lo[5], f0[2 * P + self]);
        if (f1) {
          pair_add(hi[1], lo[1], f1[self]);
          pair_add(hi[3], lo[3], f1[3 * P + self]);
          pair_add(hi[6], lo[6], f1[P + self]);
          pair_add(hi[7], lo[7], f1[2 * P + self]);
        }
        if (a.Cfield) pair_add(hi[8], lo[8], a.Cfield[self]);
      }
      if (a.removed) {
        dacc[1] += a.removed[self];
        if (a.nc > 1) dacc[2] += a.removed[P + self];
        dacc[3] += a.removed[(size_t)a.nc * P + self];
      }
    }
  }
  // warp: the FP32 pairs with error-free additions, the counts in
  // integers; FP64 shuffles only for the FP64 arrays of reaction runs
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < 9; q++) {
      const float oh = __shfl_down_sync(0xffffffffu, hi[q], o);
      const float ol = __shfl_down_sync(0xffffffffu, lo[q], o);
      const float l = lo[q] + ol;
      lo[q] = l;
      pair_add(hi[q], lo[q], oh);
    }
  }
  nsolid = __reduce_add_sync(0xffffffffu, nsolid);
  nfluid = __reduce_add_sync(0xffffffffu, nfluid);
  if (a.b || a.removed) {
#pragma unroll
    for (int q = 0; q < 4; q++) dacc[q] = warp_sum(dacc[q]);
  }
  __shared__ double sm[TB / 32][NTHERMO];
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < 9; q++) sm[w][q] = (double)hi[q] + (double)lo[q];
#pragma unroll
    for (int q = 0; q < 4; q++) sm[w][9 + q] = dacc[q];
    sm[w][13] = (double)nsolid;
    sm[w][14] = (double)nfluid;
#pragma unroll
    for (int q = 15; q < NTHERMO; q++) sm[w][q] = 0.0;
  }
  __syncthreads();
  if (threadIdx.x < NTHERMO) {
    double s = 0.0;
    for (int k = 0; k < TB / 32; k++) s += sm[k][threadIdx.x];
    a.partials[(size_t)blockIdx.x * NTHERMO + threadIdx.x] = s;
  }
  // the last block to finish reduces every block's slot
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(a.done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  thermo_final(a.partials, gridDim.x, a.out);
  if (threadIdx.x == 0) {
    *a.done = 0u;
    reinterpret_cast<unsigned long long *>(a.out)[NTHERMO] = a.nflips ? *a.nflips : 0ull;
    a.out[NTHERMO + 1] = a.errw ? (double)*a.errw : 0.0;
  }
}

// node of dense index idx over the rows [ylo, yhi): the host-side arrays
// of the conversion kernels are [yhi - ylo][nx], index (y - ylo) nx + x
__device__ __forceinline__ bool node_of(int idx, const Geometry &g, int &x, int &y) {
  if (idx >= g.nx * (g.yhi - g.ylo)) return false;
  const int r = idx / g.nx;
  x = idx - r * g.nx;
  y = g.ylo + r;
  return true;
}

template <class S>
__global__ void k_import_pops(const double *src, S *dst, const uint32_t *mask, Geometry g,
                              int q, float rho_ref, float scale, bool shift, double alpha) {
  int x, y;
  if (!node_of(blockIdx.x * blockDim.x + threadIdx.x, g, x, y)) return;
  const bool sol = solid_at(mask, g.mw, x, y);
  const size_t dense = (size_t)(y - g.ylo) * g.nx + x, self = (size_t)y * g.pitch + x;
  const size_t nn = (size_t)g.nx * (g.yhi - g.ylo);
  for (int i = 0; i < q; i++) {
    double v = sol ? 0.0 : src[(size_t)i * nn + dense];
    if (shift && !sol) v -= wshare(i, alpha) * (double)rho_ref;
    Store<S>::st(dst, (size_t)i * g.plane + self, (float)v, scale);
  }
}

template <class S>
__global__ void k_export_pops(const S *src, double *dst, const uint32_t *mask, Geometry g,
                              int q, float rho_ref, float inv_scale, bool shift, double alpha) {
  int x, y;
  if (!node_of(blockIdx.x * blockDim.x + threadIdx.x, g, x, y)) return;
  const bool sol = solid_at(mask, g.mw, x, y);
  const size_t dense = (size_t)(y - g.ylo) * g.nx + x, self = (size_t)y * g.pitch + x;
  const size_t nn = (size_t)g.nx * (g.yhi - g.ylo);
  for (int i = 0; i < q; i++) {
    double v = 0.0;
    if (!sol) {
      v = (double)Store<S>::ld(src, (size_t)i * g.plane + self, inv_scale);
      if (shift) v += wshare(i, alpha) * (double)rho_ref;
    }
    dst[(size_t)i * nn + dense] = v;
  }
}

// f_eq(rho, u) of Eq. (2) (with the fluids command's alpha), evaluated in
// FP64, stored as deviations from s_i rho_ref
template <class S>
__global__ void k_equilibrium(const double *rho, const double *ux, const double *uy, S *dst,
                              const uint32_t *mask, Geometry g, float rho_ref, float scale,
                              double alpha) {
  int x, y;
  if (!node_of(blockIdx.x * blockDim.x + threadIdx.x, g, x, y)) return;
  const bool sol = solid_at(mask, g.mw, x, y);
  const size_t dense = (size_t)(y - g.ylo) * g.nx + x, self = (size_t)y * g.pitch + x;
  const double r = rho[dense], u = ux ? ux[dense] : 0.0, v = uy ? uy[dense] : 0.0;
  const double dr = r - (double)rho_ref, usq = u * u + v * v;
#pragma unroll
  for (int i = 0; i < 9; i++) {
    const double eu = EX(i) * u + EY(i) * v;
    const double w = (i == 0) ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    const double h = (alpha == 4.0 / 9.0) ? w * (dr + r * (3.0 * eu + 4.5 * eu * eu - 1.5 * usq))
                                          : wshare(i, alpha) * dr + w * r * (3.0 * eu + 4.5 * eu * eu - 1.5 * usq);
    Store<S>::st(dst, (size_t)i * g.plane + self, sol ? 0.0f : (float)h, scale);
  }
}

// g_eq(C, u) of Eq. (3) (D2Q4) or w_i C (1 + 3 e.u) (D2Q9), FP32 storage
__global__ void k_solute_equilibrium(const double *C, const double *ux, const double *uy,
                                     float *dst, const uint32_t *mask, Geometry g, int q) {
  int x, y;
  if (!node_of(blockIdx.x * blockDim.x + threadIdx.x, g, x, y)) return;
  const bool sol = solid_at(mask, g.mw, x, y);
  const size_t dense = (size_t)(y - g.ylo) * g.nx + x, self = (size_t)y * g.pitch + x;
  const double c = C[dense], u = ux ? ux[dense] : 0.0, v = uy ? uy[dense] : 0.0;
  for (int i = 0; i < q; i++) {
    double val;
    if (q == 4) val = 0.25 * c * (1.0 + 2.0 * (EX4(i) * u + EY4(i) * v));
    else {
      const double w = (i == 0) ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
      val = w * c * (1.0 + 3.0 * (EX(i) * u + EY(i) * v));
    }
    dst[(size_t)i * g.plane + self] = sol ? 0.0f : (float)val;
  }
}

__global__ void k_export_fields(const float *fields, const uint32_t *mask, Geometry g,
                                float rho_ref, double *rho, double *px, double *py,
                                double *req) {
  int x, y;
  if (!node_of(blockIdx.x * blockDim.x + threadIdx.x, g, x, y)) return;
  const bool sol = solid_at(mask, g.mw, x, y);
  const size_t dense = (size_t)(y - g.ylo) * g.nx + x, self = (size_t)y * g.pitch + x;
  const double R = (double)rho_ref;
  if (rho) rho[dense] = sol ? 0.0 : R + (double)fields[self];
  if (px) px[dense] = sol ? 0.0 : (double)fields[g.plane + self];
  if (py) py[dense] = sol ? 0.0 : (double)fields[2 * g.plane + self];
  if (req) req[dense] = sol ? 0.0 : R + (double)fields[3 * g.plane + self];
}

__global__ void k_export_velocity(const float *fields, int nc, const uint32_t *mask, Geometry g,
                                  float r0, float r1, float *rho, float *ux, float *uy) {
  int x, y;
  if (!node_of(blockIdx.x * blockDim.x + threadIdx.x, g, x, y)) return;
  const bool sol = solid_at(mask, g.mw, x, y);
  const size_t dense = (size_t)(y - g.ylo) * g.nx + x, self = (size_t)y * g.pitch + x;
  float rs = 0.f, pxs = 0.f, pys = 0.f;
  for (int c = 0; c < nc; c++) {
    const float *fl = fields + (size_t)c * NFIELD * g.plane;
    rs += (c ? r1 : r0) + fl[self];
    pxs += fl[g.plane + self];
    pys += fl[2 * g.plane + self];
  }
  rho[dense] = sol ? 0.f : rs;
  ux[dense] = sol ? 0.f : pxs / rs;
  uy[dense] = sol ? 0.f : pys / rs;
}

__global__ void k_export_plane_f32(const float *src, const uint32_t *mask, Geometry g, double *dst) {
  int x, y;
  if (!node_of(blockIdx.x * blockDim.x + threadIdx.x, g, x, y)) return;
  const bool sol = solid_at(mask, g.mw, x, y);
  dst[(size_t)(y - g.ylo) * g.nx + x] = sol ? 0.0 : (double)src[(size_t)y * g.pitch + x];
}

__global__ void k_export_plane_f64(const double *src, Geometry g, double *dst) {
  int x, y;
  if (!node_of(blockIdx.x * blockDim.x + threadIdx.x, g, x, y)) return;
  dst[(size_t)(y - g.ylo) * g.nx + x] = src[(size_t)y * g.pitch + x];
}

__global__ void k_import_plane_f64(const double *src, Geometry g, double *dst) {
  int x, y;
  if (!node_of(blockIdx.x * blockDim.x + threadIdx.x, g, x, y)) return;
  dst[(size_t)y * g.pitch + x] = src[(size_t)(y - g.ylo) * g.nx + x];
}

inline unsigned grid1(const Geometry &g) {
  return (unsigned)(((long long)g.nx * (g.yhi - g.ylo) + 255) / 256);
}

inline int ok() { return cudaGetLastError() == cudaSuccess ? 1 : -1; }

}  // namespace

int thermo_blocks(const Geometry &g, int sms) {
  // one block per updated row, at most THERMO_BLOCKS_PER_SM per SM (all resident)
  int b = g.yhi - g.ylo;
  const int cap = THERMO_BLOCKS_PER_SM * (sms > 0 ? sms : 1);
  if (b > cap) b = cap;
  return b < 1 ? 1 : b;
}

namespace {

// contiguous runs copied between device buffers (the halo rows of slabs):
// run k goes from src[k] to dst[k], bytes[k] of them (a multiple of 4; in
// 16-byte words where both ends and the size allow); blockIdx.y picks the
// run
__global__ void k_copy_runs(const CopyRuns r) {
  const int k = blockIdx.y;
  const unsigned step = gridDim.x * blockDim.x, i0 = blockIdx.x * blockDim.x + threadIdx.x;
  if ((((uintptr_t)r.src[k] | (uintptr_t)r.dst[k] | r.bytes[k]) & 15u) == 0) {
    const uint4 *s = (const uint4 *)r.src[k];
    uint4 *d = (uint4 *)r.dst[k];
    for (unsigned i = i0; i < (r.bytes[k] >> 4); i += step) d[i] = s[i];
  } else {
    const uint32_t *s = (const uint32_t *)r.src[k];
    uint32_t *d = (uint32_t *)r.dst[k];
    for (unsigned i = i0; i < (r.bytes[k] >> 2); i += step) d[i] = s[i];
  }
}

}  // namespace

int launch_copy_runs(const CopyRuns &r, cudaStream_t s) {
  if (r.n <= 0) return 0;
  unsigned most = 0;
  for (int k = 0; k < r.n; k++) most = max(most, r.bytes[k] >> 4);
  const unsigned bx = (most + 255) / 256;
  k_copy_runs<<<dim3(bx < 1 ? 1 : (bx > 16 ? 16 : bx), r.n), 256, 0, s>>>(r);
  return ok();
}

int launch_thermo(const ThermoArgs &a, int nblocks, cudaStream_t s) {
  return launch_pdl(k_thermo_partial, dim3(nblocks), dim3(TB), 0, s, a) == cudaSuccess ? 1 : -1;
}

int launch_import_pops(int storage, const double *src, void *dst, const uint32_t *mask,
                       Geometry g, int q, float rho_ref, float scale, bool shift,
                       double alpha, cudaStream_t s) {
  switch (storage) {
    case ST_FP16:
      k_import_pops<__half><<<grid1(g), 256, 0, s>>>(src, (__half *)dst, mask, g, q, rho_ref, scale, shift, alpha);
      break;
    case ST_BF16:
      k_import_pops<__nv_bfloat16><<<grid1(g), 256, 0, s>>>(src, (__nv_bfloat16 *)dst, mask, g, q, rho_ref, scale, shift, alpha);
      break;
    default:
      k_import_pops<float><<<grid1(g), 256, 0, s>>>(src, (float *)dst, mask, g, q, rho_ref, scale, shift, alpha);
  }
  return ok();
}

int launch_export_pops(int storage, const void *src, double *dst, const uint32_t *mask,
                       Geometry g, int q, float rho_ref, float inv_scale, bool shift,
                       double alpha, cudaStream_t s) {
  switch (storage) {
    case ST_FP16:
      k_export_pops<__half><<<grid1(g), 256, 0, s>>>((const __half *)src, dst, mask, g, q, rho_ref, inv_scale, shift, alpha);
      break;
    case ST_BF16:
      k_export_pops<__nv_bfloat16><<<grid1(g), 256, 0, s>>>((const __nv_bfloat16 *)src, dst, mask, g, q, rho_ref, inv_scale, shift, alpha);
      break;
    default:
      k_export_pops<float><<<grid1(g), 256, 0, s>>>((const float *)src, dst, mask, g, q, rho_ref, inv_scale, shift, alpha);
  }
  return ok();
}

int launch_equilibrium(int storage, const double *rho, const double *ux, const double *uy,
                       void *dst, const uint32_t *mask, Geometry g, float rho_ref,
                       float scale, double alpha, cudaStream_t s) {
  switch (storage) {
    case ST_FP16:
      k_equilibrium<__half><<<grid1(g), 256, 0, s>>>(rho, ux, uy, (__half *)dst, mask, g, rho_ref, scale, alpha);
      break;
    case ST_BF16:
      k_equilibrium<__nv_bfloat16><<<grid1(g), 256, 0, s>>>(rho, ux, uy, (__nv_bfloat16 *)dst, mask, g, rho_ref, scale, alpha);
      break;
    default:
      k_equilibrium<float><<<grid1(g), 256, 0, s>>>(rho, ux, uy, (float *)dst, mask, g, rho_ref, scale, alpha);
  }
  return ok();
}

int launch_solute_equilibrium(int q, const double *C, const double *ux, const double *uy,
                              float *dst, const uint32_t *mask, Geometry g, cudaStream_t s) {
  k_solute_equilibrium<<<grid1(g), 256, 0, s>>>(C, ux, uy, dst, mask, g, q);
  return ok();
}

int launch_export_fields(const float *fields, int comp, const uint32_t *mask, Geometry g,
                         float rho_ref, double *rho, double *px, double *py, double *req,
                         cudaStream_t s) {
  k_export_fields<<<grid1(g), 256, 0, s>>>(fields + (size_t)comp * NFIELD * g.plane, mask, g,
                                           rho_ref, rho, px, py, req);
  return ok();
}

int launch_export_velocity(const float *fields, int nc, const uint32_t *mask, Geometry g,
                           const float *rho_ref, float *rho, float *ux, float *uy,
                           cudaStream_t s) {
  k_export_velocity<<<grid1(g), 256, 0, s>>>(fields, nc, mask, g, rho_ref[0],
                                             nc > 1 ? rho_ref[1] : 0.f, rho, ux, uy);
  return ok();
}

int launch_export_plane_f32(const float *src, const uint32_t *mask, Geometry g, double *dst,
                            cudaStream_t s) {
  k_export_plane_f32<<<grid1(g), 256, 0, s>>>(src, mask, g, dst);
  return ok();
}

int launch_export_plane_f64(const double *src, Geometry g, double *dst, cudaStream_t s) {
  k_export_plane_f64<<<grid1(g), 256, 0, s>>>(src, g, dst);
  return ok();
}

int launch_import_plane_f64(const double *src, Geometry g, double *dst, cudaStream_t s) {
  k_import_plane_f64<<<grid1(g), 256, 0, s>>>(src, g, dst);
  return ok();
}

}  // namespace lbk
