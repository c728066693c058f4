// k_batch.cu -- many independent lattices advanced by one persistent launch.
//
// Each lattice is a periodic single-component D2Q9 lattice with body
// forces (pull streaming, half-way bounce-back at its solid nodes, velocity
// shift, BGK; the same update as k_fluid_local, with the same per-node
// neighbour codes and one load per direction).  The lattices are cut into
// TX x TY tiles listed in one array; a grid of (SM count x resident CTAs)
// blocks walks that list either statically (tile k, k + grid, ...) or
// dynamically (an atomic counter hands out the next tile), so a launch
// costs the same whatever the number and sizes of the lattices.  The tile
// shape and the schedule are chosen by timing (lb_batch_autotune).
#include "lbcollide.cuh"
#include "lbbatch.h"

namespace lbk {

namespace {

// One warp updates 32 consecutive nodes x0 .. x0+31 of row y (x0 a
// multiple of 32): each lane's 3 x 3 solid neighbourhood from its
// neighbour code, pull with half-way bounce-back by one load per
// direction, BGK with the velocity shift.  Solid and padding lanes store
// zeros where their 32-byte sector holds a fluid lane, so the warp writes
// whole sectors and leaves sectors without fluid alone.
template <class S>
__device__ __forceinline__ void batch_warp(const BatchLat &L, const S *fin, S *fout, int x, int y,
                                           uint32_t seed) {
  const int ym = y ? y - 1 : L.ny - 1, yp = (y + 1 == L.ny) ? 0 : y + 1;
  const int P = (int)L.plane;
  const int self = y * L.pitch + x;
  // x < pitch; slots past nx are coded solid
  const uint32_t bits = __ldg(L.nbc + self);
  const bool idle = (bits >> NBPOS(0, 0)) & 1u;
  const unsigned busy = __ballot_sync(0xffffffffu, !idle);
  if (idle) {
    constexpr int LPS = 32 / (int)sizeof(S);  // lanes per 32-byte sector
    if ((busy >> (threadIdx.x & ~(LPS - 1))) & ((1u << LPS) - 1u)) {
#pragma unroll
      for (int i = 0; i < 9; i++) Store<S>::st(fout, i * P + self, 0.0f, 1.0f);
    }
    return;
  }
  const int xm = x ? x - 1 : L.nx - 1, xp = (x + 1 == L.nx) ? 0 : x + 1;
  const int r0 = y * L.pitch, rm = ym * L.pitch, rp = yp * L.pitch;
  const int src[9] = {self, r0 + xm, rm + x, r0 + xp, rp + x, rm + xm, rm + xp, rp + xp, rp + xm};
  float h[9];
#pragma unroll
  for (int i = 0; i < 9; i++) {
    const int k = (i && nb(bits, OPP(i))) ? OPP(i) * P + self : i * P + src[i];
    h[i] = Store<S>::ld(fin, k, L.inv_scale);
  }
  const float d = ((h[0] + h[1]) + (h[2] + h[3])) + ((h[4] + h[5]) + (h[6] + h[7])) + h[8];
  float jx, jy, jxl = 0.f, jyl = 0.f;
  if (L.pm) {
    momentum_exact(h, jx, jxl, jy, jyl);
  } else {
    jx = (h[1] - h[3]) + (h[5] - h[7]) + (h[8] - h[6]);
    jy = (h[2] - h[4]) + (h[5] - h[7]) + (h[6] - h[8]);
  }
  const float rho = L.rho_ref + d;
  const float Fx = L.fx + rho * L.ax, Fy = L.fy + rho * L.ay;
  const float ir = 1.0f / rho;
  const float mx = jx + (jxl + L.tau * Fx), my = jy + (jyl + L.tau * Fy);
  const float ux = mx * ir, uy = my * ir;
  float heq[9];
  equilibrium_pairs(d, rho, ux, uy, mx, my, 1.0f / 9.0f, 1.0f / 36.0f, heq);
  if (L.sr) {
    // stochastic rounding as in the single-lattice kernels: one hash per
    // node and launch, a linear congruential step per pair of stores
    uint32_t r = rnd(seed, self, 0, 0);
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
      r = r * 1664525u + 1013904223u;
      Store<S>::st2_dither(fout, i * P + self, (i + 1) * P + self, (h[i] + L.omega * (heq[i] - h[i])) * L.scale,
                           (h[i + 1] + L.omega * (heq[i + 1] - h[i + 1])) * L.scale, r);
    }
    r = r * 1664525u + 1013904223u;
    Store<S>::st_dither(fout, 8 * P + self, (h[8] + L.omega * (heq[8] - h[8])) * L.scale, r);
  } else {
#pragma unroll
    for (int i = 0; i < 9; i++)
      Store<S>::st(fout, i * P + self, h[i] + L.omega * (heq[i] - h[i]), L.scale);
  }
}

template <class S, int TX, int TY>
__global__ void __launch_bounds__(256, 5) k_batch(const BatchLat *__restrict__ lat,
                                               const int4 *__restrict__ tiles, int ntiles,
                                               int parity, int dynamic,
                                               unsigned int *counters, unsigned int *tick) {
  __shared__ int s_next;
  // this launch's number (read by every block); block 0 numbers the next
  const unsigned int launch_no = tick[parity];
  if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) tick[1 - parity] = launch_no + 1u;
  if (dynamic && blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0)
    counters[1 - parity] = 0;  // the other parity's counter is idle now
  int k = blockIdx.x;
  if (dynamic) {
    if (threadIdx.x == 0 && threadIdx.y == 0) s_next = (int)atomicAdd(&counters[parity], 1u);
    __syncthreads();
    k = s_next;
  }
  while (k < ntiles) {
    const int4 t = tiles[k];
    const BatchLat &L = lat[t.x];
    const int in = (L.cur + parity) & 1;
    const S *fin = (const S *)L.buf[in];
    S *fout = (S *)L.buf[1 - in];
#pragma unroll
    for (int dy = 0; dy < TY; dy += 8) {
      const int y = t.z + dy + threadIdx.y;
      if (y >= L.ny) break;
#pragma unroll
      for (int dx = 0; dx < TX; dx += 32) {
        if (t.y + dx >= L.pitch) break;  // warp-uniform: the tile runs past the row
        batch_warp<S>(L, fin, fout, t.y + dx + threadIdx.x, y, mix32(launch_no * 0x9e3779b9u + (uint32_t)t.x));
      }
    }
    if (dynamic) {
      __syncthreads();
      if (threadIdx.x == 0 && threadIdx.y == 0) s_next = (int)atomicAdd(&counters[parity], 1u);
      __syncthreads();
      k = s_next;
    } else {
      k += gridDim.x;
    }
  }
}

template <class S, int TX, int TY>
int launch_t(const BatchLaunch &b, int parity, cudaStream_t s) {
  dim3 blk(32, 8);
  k_batch<S, TX, TY><<<b.grid, blk, 0, s>>>(b.lat, b.tiles, b.ntiles, parity, b.dynamic, b.counters, b.tick);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

template <class S>
int launch_s(const BatchLaunch &b, int parity, cudaStream_t s) {
  switch (b.shape) {
    case 0: return launch_t<S, 32, 8>(b, parity, s);
    case 1: return launch_t<S, 32, 16>(b, parity, s);
    case 2: return launch_t<S, 64, 8>(b, parity, s);
    case 3: return launch_t<S, 64, 16>(b, parity, s);
    case 4: return launch_t<S, 32, 32>(b, parity, s);
    default: return launch_t<S, 128, 8>(b, parity, s);
  }
}

template <class S, int TX, int TY>
int occ_t() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<S, TX, TY>, 256, 0);
  return n;
}

}  // namespace

int batch_shape_tx(int shape) { return shape == 2 || shape == 3 ? 64 : shape == 5 ? 128 : 32; }
int batch_shape_ty(int shape) { return shape == 1 || shape == 3 ? 16 : shape == 4 ? 32 : 8; }

int batch_occupancy(int storage, int shape) {
  // occupancy is a property of the kernel's resources; the shapes share them
  (void)shape;
  switch (storage) {
    case ST_FP16: return occ_t<__half, 32, 8>();
    case ST_BF16: return occ_t<__nv_bfloat16, 32, 8>();
    default: return occ_t<float, 32, 8>();
  }
}

int launch_batch(int storage, const BatchLaunch &b, int parity, cudaStream_t s) {
  switch (storage) {
    case ST_FP16: return launch_s<__half>(b, parity, s);
    case ST_BF16: return launch_s<__nv_bfloat16>(b, parity, s);
    default: return launch_s<float>(b, parity, s);
  }
}

}  // namespace lbk
