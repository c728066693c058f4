// k_tma.cu -- the single-component fluid iteration as a persistent,
// TMA-pipelined kernel.
//
// A persistent grid (a multiple of the SM count, as many CTAs per SM as the
// shared memory allows) walks the lattice's 128 x 4 tiles.  For each tile
// it needs, per population plane, the 6 rows y0-1 .. y0+4 and the columns
// x0-HX .. x0+128+HX (HX = one 16 byte granule of halo on each side),
// periodic wrap included.  One warp
// issues those rows as bulk asynchronous copies (cp.async.bulk, tracked by
// the stage's mbarrier transaction count) into one of two shared-memory
// stages while the CTA computes the previous tile from the other stage, so
// HBM streams whole 0.5 KB rows and the loads of the next tile overlap the
// arithmetic of this one.  The arithmetic and the stores are those of
// k_fluid_local (lbcollide.cuh), and the results are bit-identical.
//
// Measured on GB300 it is slower than the streaming kernel (about 44-45
// against 75-85 GMLUPS on a 4096^2 lattice): the shared-memory stages cap
// the resident warps well below the streaming kernel's 64 per SM, and the
// per-node arithmetic then lacks the warps to hide its latency.  It is kept
// as a selectable kernel (lb_set_kernel "tma"); "auto" picks streaming.
//
// Every mbarrier wait is bounded by a clock-cycle limit the host sets
// (lb_set_wait_limit; by default about two seconds): a wait that runs out
// records the failure in the error word, then waits for the copies already
// issued with the long default limit, so no copy into shared memory is in
// flight when the CTA returns.
#include "lbcollide.cuh"

namespace lbk {

namespace {

constexpr int TT_W = 128, TT_H = 4, TT_THREADS = 512;

template <class S>
struct TmaLayout {
  static constexpr int HX = 16 / (int)sizeof(S);   // halo columns (16 bytes)
  static constexpr int COLS = TT_W + 2 * HX;       // shared-memory columns per row
  static constexpr int ROWS = TT_H + 2;            // rows y0-1 .. y0+TT_H
  static constexpr int PLANE = ROWS * COLS;        // elements per plane and stage
  static constexpr int STAGE = 9 * PLANE;          // elements per stage
  static constexpr int MW = 12;                    // mask words per row: c0-4 .. c0+7
  static constexpr size_t SMEM =
      2 * (size_t)STAGE * sizeof(S) + 2 * (size_t)ROWS * MW * 4 + 2 * 8;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// wait for the stage's phase with a clock limit; false on timeout
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// column pieces of one shared-memory row for the tile starting at x0: the
// columns j hold nodes x0 - HX + j (mod nx); returns the bytes per row
template <class S>
__device__ __forceinline__ int row_pieces(int x0, int nx, int (&gx)[3], int (&sj)[3], int (&len)[3]) {
  constexpr int HX = TmaLayout<S>::HX;
  const int lo = x0 - HX, hi = min(x0 + TT_W + HX, nx);
  const int a = max(lo, 0);
  gx[0] = a;
  sj[0] = a - lo;
  len[0] = hi - a;
  // left halo of the first tile column: the last HX nodes of the row
  gx[1] = nx - HX;
  sj[1] = 0;
  len[1] = lo < 0 ? HX : 0;
  // right halo past the row end: the first HX nodes of the row
  gx[2] = 0;
  sj[2] = nx - lo;
  len[2] = (x0 + TT_W + HX > nx) ? HX : 0;
  return (len[0] + len[1] + len[2]) * (int)sizeof(S);
}

// issue the bulk copies of tile (x0, y0) into stage `st` (all lanes of the
// calling warp take part); lane 0 first registers the byte count
template <class S>
__device__ __forceinline__ void issue_tile(const FluidArgs &p, const S *fin, S *st, uint64_t *bar,
                                           int x0, int y0) {
  constexpr int ROWS = TmaLayout<S>::ROWS, COLS = TmaLayout<S>::COLS, PLANE = TmaLayout<S>::PLANE;
  const Geometry &g = p.g;
  const int lane = threadIdx.x & 31;
  int gx[3], sj[3], len[3];
  const int row_bytes = row_pieces<S>(x0, g.nx, gx, sj, len);
  if (lane == 0) {
    fence_proxy_async();
    mbar_expect_tx(bar, (uint32_t)(9 * ROWS * row_bytes));
  }
  __syncwarp();
  for (int t = lane; t < 9 * ROWS; t += 32) {
    const int i = t / ROWS, r = t - i * ROWS;
    int gy = y0 - 1 + r;
    gy %= g.ny;
    if (gy < 0) gy += g.ny;
    const S *src = fin + (size_t)i * g.plane + (size_t)gy * g.pitch;
    S *dst = st + i * PLANE + r * COLS;
#pragma unroll
    for (int q = 0; q < 3; q++)
      if (len[q]) bulk_g2s(dst + sj[q], src + gx[q], (uint32_t)(len[q] * (int)sizeof(S)), bar);
  }
}

// mask words of tile (x0, y0): rows y0-1 .. y0+TT_H, word columns c0-4 ..
// c0+7 (zero outside the row); thread t < ROWS*MW loads word t
__device__ __forceinline__ uint32_t mask_word(const uint32_t *m, const Geometry &g, int x0, int y0, int t,
                                              int rows, int mw_tile) {
  const int r = t / mw_tile, k = t - r * mw_tile;
  int gy = (y0 - 1 + r) % g.ny;
  if (gy < 0) gy += g.ny;
  const int w = (x0 >> 5) - 4 + k;
  (void)rows;
  return (w >= 0 && w < g.mw) ? __ldg(m + (size_t)gy * g.mw + w) : 0u;
}

// the limit of the waits that let issued copies land before a CTA gives up
constexpr long long DRAIN_LIMIT = 4000000000LL;  // clock cycles (~2 s at 2 GHz)

template <class S, int SR>
__global__ void __launch_bounds__(TT_THREADS, 3) k_fluid_tma(const FluidArgs p, int *err, long long limit) {
  using L = TmaLayout<S>;
  // the same arithmetic as the streaming kernel (scaled 16-bit storage
  // folded, rounding mode SR), so the two agree bit for bit
  constexpr bool FOLD = Store<S>::kScaled;
  const float linv = FOLD ? 1.0f : p.inv_scale;
  extern __shared__ __align__(128) unsigned char sm_raw[];
  // stage q: populations at stage0 + q * STAGE, mask words at msk0 + q *
  // ROWS * MW, barrier bar[q]
  S *const stage0 = (S *)sm_raw;
  uint32_t *const msk0 = (uint32_t *)(stage0 + 2 * L::STAGE);
  uint64_t *const bar = (uint64_t *)(msk0 + 2 * L::ROWS * L::MW);
  const Geometry &g = p.g;
  const int tiles_x = (g.nx + TT_W - 1) / TT_W, tiles_y = (g.ny + TT_H - 1) / TT_H;
  const int ntiles = tiles_x * tiles_y;
  const int tid = threadIdx.x;
  const S *fin = (const S *)p.fin;

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  int k = blockIdx.x;
  if (k >= ntiles) return;
  // prologue: tile k into stage 0
  if (tid < 32) issue_tile<S>(p, fin, stage0, &bar[0], (k % tiles_x) * TT_W, (k / tiles_x) * TT_H);
  if (tid < L::ROWS * L::MW)
    msk0[tid] = mask_word(p.mask, g, (k % tiles_x) * TT_W, (k / tiles_x) * TT_H, tid, L::ROWS, L::MW);
  __syncthreads();
  uint32_t phase = 0u;    // bit q: parity to wait for on bar[q]
  uint32_t pending = 1u;  // bit q: copies issued into stage q not yet waited for
  int s = 0;
  for (; k < ntiles; k += gridDim.x) {
    const int kn = k + gridDim.x;
    uint32_t mnext = 0;
    if (kn < ntiles) {
      if (tid < 32)
        issue_tile<S>(p, fin, stage0 + (s ^ 1) * L::STAGE, &bar[s ^ 1], (kn % tiles_x) * TT_W,
                      (kn / tiles_x) * TT_H);
      pending |= 1u << (s ^ 1);
      if (tid < L::ROWS * L::MW)
        mnext = mask_word(p.mask, g, (kn % tiles_x) * TT_W, (kn / tiles_x) * TT_H, tid, L::ROWS, L::MW);
    }
    // limit 0: give up at the first wait (the give-up path on demand; a
    // blocking try_wait can otherwise see the copies land within its own
    // suspend time)
    const bool ok = limit > 0 && mbar_wait_bounded(&bar[s], (phase >> s) & 1u, limit);
    if (__syncthreads_or(!ok)) {
      // record the failure, let the copies already issued land, leave
      if (tid == 0) atomicOr(err, 1);
      if (pending & 1u) mbar_wait_bounded(&bar[0], phase & 1u, DRAIN_LIMIT);
      if (pending & 2u) mbar_wait_bounded(&bar[1], (phase >> 1) & 1u, DRAIN_LIMIT);
      return;
    }
    phase ^= 1u << s;
    pending &= ~(1u << s);

    // compute tile k from stage s
    const int x0 = (k % tiles_x) * TT_W, y0 = (k / tiles_x) * TT_H;
    const S *sb = stage0 + s * L::STAGE;
    const uint32_t(*win)[L::MW] = (const uint32_t(*)[L::MW])(msk0 + s * L::ROWS * L::MW);
    for (int n = tid; n < TT_W * TT_H; n += TT_THREADS) {
      const int ly = n / TT_W, lx = n - ly * TT_W;
      const int x = x0 + lx, y = y0 + ly;
      if (x >= g.nx || y >= g.ny) continue;
      const int wc = (lx >> 5) + 4, lane = lx & 31;
      if ((win[ly + 1][wc] >> lane) & 1u) continue;  // solid nodes hold no populations
      uint32_t bits;
      if (x == 0 || x == g.nx - 1) {
        const int xm = x ? x - 1 : g.nx - 1, xp = (x + 1 == g.nx) ? 0 : x + 1;
        const int ym = y ? y - 1 : g.ny - 1, yp = (y + 1 == g.ny) ? 0 : y + 1;
        bits = nbr_bits(p.mask, g.mw, x, y, xm, xp, ym, yp);
      } else {
        bits = row3(win[ly][wc - 1], win[ly][wc], win[ly][wc + 1], lane) |
               (row3(win[ly + 1][wc - 1], win[ly + 1][wc], win[ly + 1][wc + 1], lane) << 3) |
               (row3(win[ly + 2][wc - 1], win[ly + 2][wc], win[ly + 2][wc + 1], lane) << 6);
      }
      float h[1][9];
      const int cself = (ly + 1) * L::COLS + lx + L::HX;
#pragma unroll
      for (int i = 0; i < 9; i++) {
        const int off = (i && nb(bits, OPP(i))) ? OPP(i) * L::PLANE + cself
                                                : i * L::PLANE + cself - EY(i) * L::COLS - EX(i);
        h[0][i] = Store<S>::ld_smem(sb, off, linv);
      }
      if (p.nopen) apply_openings<1>(p, x, y, h, FOLD ? p.scale : 1.0f);
      const float F[1][2] = {{0.f, 0.f}};
      collide_store<S, 1, false, false, FOLD, SR>(p, x, y, bits, h, F);
    }
    if (kn < ntiles && tid < L::ROWS * L::MW) msk0[(s ^ 1) * L::ROWS * L::MW + tid] = mnext;
    __syncthreads();
    s ^= 1;
  }
}

template <class S>
int launch_tma_t(const FluidArgs &a, int *err, long long limit, cudaStream_t s, int sms) {
  using L = TmaLayout<S>;
  static bool configured[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return -1;
  if (!configured[dev]) {
    if (cudaFuncSetAttribute(k_fluid_tma<S, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::SMEM) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_fluid_tma<S, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::SMEM) !=
            cudaSuccess)
      return -1;
    configured[dev] = true;
  }
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fluid_tma<S, 1>, TT_THREADS, L::SMEM);
  if (per < 1) per = 1;
  const int ntiles = ((a.g.nx + TT_W - 1) / TT_W) * ((a.g.ny + TT_H - 1) / TT_H);
  int grid = sms * per;
  if (grid > ntiles) grid = ntiles;
  if (a.sr_seed) k_fluid_tma<S, 2><<<grid, TT_THREADS, L::SMEM, s>>>(a, err, limit);
  else k_fluid_tma<S, 1><<<grid, TT_THREADS, L::SMEM, s>>>(a, err, limit);
  return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace

bool tma_supported(int storage, const Geometry &g) {
  const int hx = storage == ST_FP32 ? 4 : 8;
  // whole 16-byte granules on every row piece, and a halo inside the row
  return g.nx % hx == 0 && g.nx >= 2 * hx && (long long)g.plane * 9 < (1LL << 31);
}

int launch_fluid_tma(int storage, const FluidArgs &a, int *err, long long limit, cudaStream_t s, int sms) {
  if (limit < 0) limit = DRAIN_LIMIT;
  switch (storage) {
    case ST_FP16: return launch_tma_t<__half>(a, err, limit, s, sms);
    case ST_BF16: return launch_tma_t<__nv_bfloat16>(a, err, limit, s, sms);
    default: return launch_tma_t<float>(a, err, limit, s, sms);
  }
}

}  // namespace lbk
