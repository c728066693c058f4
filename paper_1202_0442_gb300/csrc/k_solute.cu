// k_solute.cu -- solute lattice, precipitation and surface growth.
//
// The per-node solute update lives in lbsolute.cuh, shared with the fused
// fluid-solute kernel of k_fluid.cu (the default for single-component runs
// without intersolute); the kernels here run it on their own:
// k_solute<Q>: one iteration of the solute populations g (solute command,
//   Eq. (3); Q = 4 is the paper's D2Q4, Q = 9 the D2Q9 variant): pull
//   streaming; at a solid source either bounce-back or the reactive rule of
//   the surface_reaction command (App. C) on that link,
//     C_i = (2 g_out + kr Cs)/(kr + 2 w_i),  g_in = -g_out + 2 w_i C_i
//   (w_i = 1/4 on D2Q4 is the printed rule); the inlet_solute/outlet_solute
//   rules (dirichlet: the crossing modes make C = Cbar, split by weight;
//   adiabatic: crossing mode = opposite mode; flux: C from the flux balance
//   with the nearest inner node, all modes at equilibrium; App. B); BGK
//   with g_eq(C, u_s), u the solvent velocity of Eq. (4) written by the
//   fluid kernel in the same iteration, u_s = u + tau_s F / C with the
//   intersolute force F (else u_s = u); then precipitation
//   dB = kr (C_w - Cs) if positive, taken in equal parts from the incoming
//   modes, the share dB/|U| recorded for the solid neighbours.
// k_solute_pre<Q>: with intersolute, a first pass that writes every node's
//   concentration after streaming and the opening rules, so the update can
//   read its neighbours' psi of the same step.
// k_gather_grow: every solid node adds its fluid neighbours' shares to its
//   FP64 deposit b in a fixed order, and, if b > bmax, picks one fluid
//   4-neighbour (SplitMix64 of seed ^ (t nx ny + node) mod the number of
//   candidates, in the order +x, +y, -x, -y), flags and lists it; b := 0.
//   On a whole lattice it runs over a list of the solid nodes with a fluid
//   neighbour (k_surface_list builds it once from the neighbour codes,
//   k_apply_flips appends the nodes it turns solid) instead of scanning
//   every node: some 3 % of the nodes, one short wave in place of two
//   latency-bound waves over the lattice.
// k_apply_flips: one CTA walks the list: the nodes become solid (mask bit),
//   start with b0, and their fluid and solute mass is booked as removed.
// The two growth kernels run back to back, so every decision sees the
// state before any flip.
#include "lbpdl.cuh"
#include "lbsolute.cuh"

namespace lbk {

namespace {

// first pass of an intersolute iteration: every node's concentration after
// streaming and the opening rules (the C its collision will use)
template <int Q>
__global__ void __launch_bounds__(256) k_solute_pre(const SoluteArgs p) {
  dep_wait();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const Geometry &g = p.g;
  const int y = g.clo + blockIdx.y * blockDim.y + threadIdx.y;
  if (y >= g.chi) return;
  const uint32_t bits = solute_bits(p, x, y);
  if (x >= g.nx) return;
  const size_t self = (size_t)y * g.pitch + x;
  if ((bits >> 4) & 1u) {
    p.Cpre_out[self] = 0.f;
    return;
  }
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
  p.Cpre_out[self] = flux ? Cflux : C;
}

template <int Q>
__global__ void __launch_bounds__(256) k_solute(const SoluteArgs p) {
  dep_wait();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const Geometry &g = p.g;
  const int y = g.clo + blockIdx.y * blockDim.y + threadIdx.y;
  if (y >= g.chi) return;
  const uint32_t bits = solute_bits(p, x, y);
  if (x >= g.nx || ((bits >> 4) & 1u)) return;
  const size_t self = (size_t)y * g.pitch + x;
  solute_node<Q>(p, x, y, bits, __ldg(p.u + self), __ldg(p.u + g.plane + self));
}

// 3 x 3 solid neighbourhood of node (x, y) from its neighbour code
__device__ __forceinline__ uint32_t growth_bits(const GrowthArgs &a, int x, int y) {
  return __ldg(a.nbc + (size_t)y * a.g.pitch + x);
}

// Every solid node with a fluid neighbour adds the shares its fluid
// neighbours set aside for it (in index order, FP64), and if b > bmax picks
// one fluid 4-neighbour that is not an opening node (SplitMix64 of
// seed ^ (t nx ny + node) mod the number of candidates, candidates in the
// order +x, +y, -x, -y); the pick is flagged once and listed.  Solid nodes
// without a fluid neighbour are untouched (their b cannot change).
// The loads come first and all at once: the node's neighbour code, its
// deposit and the share slot of every neighbour, whether or not that
// neighbour is fluid (the slots of solid neighbours are read and dropped),
// so that one memory latency, not two, precedes the arithmetic.
template <int Q>
__device__ __forceinline__ void gather_grow_node(const GrowthArgs &a, int x, int y) {
  const Geometry &g = a.g;
  const int xm = x ? x - 1 : g.nx - 1, xp = (x + 1 == g.nx) ? 0 : x + 1;
  const int ym = y ? y - 1 : g.ny - 1, yp = (y + 1 == g.ny) ? 0 : y + 1;
  const size_t self = (size_t)y * g.pitch + x;
  const uint32_t bits = growth_bits(a, x, y);
  constexpr int I0 = Q == 4 ? 0 : 1;
  float slot[Q];
#pragma unroll
  for (int i = I0; i < Q; i++) {
    const int ex = Q == 4 ? EX4(i) : EX(i), ey = Q == 4 ? EY4(i) : EY(i);
    const int xf = ex > 0 ? xp : (ex < 0 ? xm : x), yf = ey > 0 ? yp : (ey < 0 ? ym : y);
    slot[i] = __ldg(a.db + (size_t)yf * g.pitch + xf);
  }
  double b = a.b[self];
  if (!((bits >> 4) & 1u) || (bits | (1u << 4)) == 0x1ffu) return;
  // the fluid neighbours' shares, added in index order (FP64)
  double acc = 0.0;
#pragma unroll
  for (int i = I0; i < Q; i++) {
    const int ex = Q == 4 ? EX4(i) : EX(i), ey = Q == 4 ? EY4(i) : EY(i);
    if ((bits >> NBPOS(ex, ey)) & 1u) continue;
    const int xf = ex > 0 ? xp : (ex < 0 ? xm : x), yf = ey > 0 ? yp : (ey < 0 ? ym : y);
    const int k = a.nopen ? opening_of(a.span, a.nopen, xf, grow(g, yf), g.nx, g.gny) : -1;
    if (k >= 0 && crosses_wall(span_wall(a.span[k]), ex, ey)) continue;
    acc += (double)slot[i];
  }
  b += acc;
  if (b > a.bmax) {
    unsigned int c0 = 0, c1 = 0, c2 = 0, c3 = 0;
    int n = 0;
#pragma unroll
    for (int d = 0; d < 4; d++) {
      const int ex = EX4(d), ey = EY4(d);
      if ((bits >> NBPOS(ex, ey)) & 1u) continue;
      const int xf = ex > 0 ? xp : (ex < 0 ? xm : x), yf = ey > 0 ? yp : (ey < 0 ? ym : y);
      if (a.nopen && opening_of(a.span, a.nopen, xf, grow(g, yf), g.nx, g.gny) >= 0) continue;
      // a candidate outside the own rows counts (the slab that owns it
      // takes the same decision) but is marked unowned
      const unsigned int off = (yf >= g.ylo && yf < g.yhi) ? (unsigned int)(yf * g.pitch + xf) : 0xffffffffu;
      if (n == 0) c0 = off;
      else if (n == 1) c1 = off;
      else if (n == 2) c2 = off;
      else c3 = off;
      n++;
    }
    if (n) {
      // node and lattice size of the whole lattice (a slab decides as it does)
      const uint64_t node = (uint64_t)grow(g, y) * (uint64_t)g.nx + (uint64_t)x;
      const uint64_t key = a.seed ^ ((uint64_t)a.t * (uint64_t)g.nx * (uint64_t)g.gny + node);
      const int pick = (int)(splitmix64(key) % (uint64_t)n);
      const unsigned int off = pick == 0 ? c0 : pick == 1 ? c1 : pick == 2 ? c2 : c3;
      if (off != 0xffffffffu && atomicExch(a.flip + off, 1u) == 0u) a.flist[atomicAdd(a.fcount, 1u)] = off;
      b = 0.0;
    }
  }
  a.b[self] = b;
}

// every solid node with a fluid neighbour in the rows [rlo, rhi)
__global__ void __launch_bounds__(256) k_gather_grow(const GrowthArgs a) {
  dep_wait();
  const Geometry &g = a.g;
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = a.rlo + blockIdx.y * 8 + threadIdx.y;
  if (y >= a.rhi) return;
  const uint32_t bits = growth_bits(a, x, y);
  if (x >= g.nx || !((bits >> 4) & 1u) || (bits | (1u << 4)) == 0x1ffu) return;
  if (a.q == 4) gather_grow_node<4>(a, x, y);
  else gather_grow_node<9>(a, x, y);
}

// the solid nodes of rows [rlo, rhi) with a fluid neighbour, appended to
// the surface list (in no particular order: each node's gather and decision
// touch only its own deposit and its own flag, so the order of the list
// does not change any result)
__global__ void __launch_bounds__(256) k_surface_list(const GrowthArgs a) {
  dep_wait();
  const Geometry &g = a.g;
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = a.rlo + blockIdx.y * 8 + threadIdx.y;
  if (y >= a.rhi || x >= g.nx) return;
  const uint32_t bits = growth_bits(a, x, y);
  if (((bits >> 4) & 1u) && (bits | (1u << 4)) != 0x1ffu)
    a.slist[atomicAdd(a.scount, 1u)] = (unsigned int)((size_t)y * g.pitch + x);
}

// One CTA's part of a growth step: it turns the listed nodes solid (mask
// bit, b = b0, their fluid and solute mass booked as removed, their
// populations cleared), appends them to the surface list if there is one,
// refreshes the neighbour codes around them, then empties the list (the
// entries stay, their number moves to fcount[1] for the host to read).
// Flips of one step are independent of each other, so their order does not
// matter.  The list and its count are read from L2: other CTAs of the same
// kernel may have written them.
template <class S>
__device__ __forceinline__ void apply_flips_cta(const GrowthArgs &a) {
  const Geometry &g = a.g;
  const unsigned int n = __ldcg(a.fcount);
  for (unsigned int k = threadIdx.x; k < n; k += blockDim.x) {
    const size_t self = __ldcg(a.flist + k);
    const int y = (int)(self / (size_t)g.pitch), x = (int)(self - (size_t)y * g.pitch);
    a.flip[self] = 0u;
    atomicOr(a.mask + (size_t)y * g.mw + (x >> 5), 1u << (x & 31));
    if (a.slist) a.slist[atomicAdd(a.scount, 1u)] = (unsigned int)self;
    a.b[self] = a.b0;
    for (int c = 0; c < a.nc; c++) {
      S *f = (S *)a.f + (size_t)c * 9 * g.plane;
      S *fp = (S *)a.f_prev + (size_t)c * 9 * g.plane;
      float d = 0.f;
      for (int i = 0; i < 9; i++) d += Store<S>::ld(f, (size_t)i * g.plane + self, a.inv_scale);
      a.removed[(size_t)c * g.plane + self] += (double)a.rho_ref[c] + (double)d;
      // a solid node holds no populations: its slots read zero in both
      // buffers, as the fluid kernels leave solid sectors untouched
      for (int i = 0; i < 9; i++) {
        Store<S>::st(f, (size_t)i * g.plane + self, 0.0f, 1.0f);
        Store<S>::st(fp, (size_t)i * g.plane + self, 0.0f, 1.0f);
      }
    }
    if (a.gpop) {
      float m = 0.f;
      for (int i = 0; i < a.q; i++) m += a.gpop[(size_t)i * g.plane + self];
      a.removed[(size_t)a.nc * g.plane + self] += (double)m;
    }
  }
  __syncthreads();
  // neighbour codes of the 3 x 3 neighbourhood of every flipped node, from
  // the mask as it now stands (L2 reads: its words changed in this kernel).
  // Overlapping neighbourhoods write the same value.
  for (unsigned int k = threadIdx.x; k < 9u * n; k += blockDim.x) {
    const size_t self = __ldcg(a.flist + k / 9);
    const int y0 = (int)(self / (size_t)g.pitch), x0 = (int)(self - (size_t)y0 * g.pitch);
    const int d = (int)(k % 9);
    int x = x0 + d % 3 - 1, y = y0 + d / 3 - 1;
    x = x < 0 ? g.nx - 1 : (x == g.nx ? 0 : x);
    y = y < 0 ? g.ny - 1 : (y == g.ny ? 0 : y);
    const int xs[3] = {x ? x - 1 : g.nx - 1, x, (x + 1 == g.nx) ? 0 : x + 1};
    const int ys[3] = {y ? y - 1 : g.ny - 1, y, (y + 1 == g.ny) ? 0 : y + 1};
    uint32_t b = 0;
#pragma unroll
    for (int j = 0; j < 3; j++)
#pragma unroll
      for (int i = 0; i < 3; i++)
        b |= ((__ldcg(a.mask + (size_t)ys[j] * g.mw + (xs[i] >> 5)) >> (xs[i] & 31)) & 1u) << (j * 3 + i);
    a.nbc[(size_t)y * g.pitch + x] = (uint16_t)b;
  }
  if (threadIdx.x == 0) {
    if (n) atomicAdd(a.nflips, (unsigned long long)n);
    a.fcount[0] = 0u;
    a.fcount[1] = n;  // kept for reading back the step's flip list
  }
}

// A whole growth step over the surface list.  Nodes only turn solid, so a
// solid node never gains a fluid neighbour: the list holds every solid node
// with a fluid neighbour (listed ones whose neighbours have all turned solid
// since are skipped by the gather).  Each CTA gathers and decides its
// entries; the last CTA to finish (a ticket taken after a fence, so it sees
// every other CTA's flags, list entries and deposits) then applies the
// step's flips: one launch where the scan needs two.
template <class S>
__global__ void __launch_bounds__(256) k_grow_list(const GrowthArgs a) {
  dep_wait();
  const Geometry &g = a.g;
  const unsigned int stride = gridDim.x * blockDim.x;
  unsigned int k = blockIdx.x * blockDim.x + threadIdx.x;
  // the thread's first entry is loaded beside the count, not after it (the
  // list has room for every node slot, so the slot exists)
  unsigned int self = k < (unsigned int)g.plane ? a.slist[k] : 0u;
  const unsigned int n = *a.scount;
  const bool wrote = k < n;
  while (k < n) {
    const int y = (int)(self / (unsigned int)g.pitch), x = (int)(self - (unsigned int)y * (unsigned int)g.pitch);
    if (a.q == 4) gather_grow_node<4>(a, x, y);
    else gather_grow_node<9>(a, x, y);
    k += stride;
    if (k < n) self = a.slist[k];
  }
  __shared__ unsigned int ticket;
  if (wrote) __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(a.done, 1u);
  __syncthreads();
  if (ticket != gridDim.x - 1) return;
  __threadfence();
  if (threadIdx.x == 0) *a.done = 0u;  // ready for the next step
  apply_flips_cta<S>(a);
}

// the flips of a scanned growth step, by one CTA
template <class S>
__global__ void __launch_bounds__(256) k_apply_flips(const GrowthArgs a) {
  dep_wait();
  apply_flips_cta<S>(a);
}

}  // namespace

int launch_solute(int q, const SoluteArgs &a, cudaStream_t s) {
  dim3 blk(32, 8), grd((a.g.nx + 31) / 32, (a.g.chi - a.g.clo + 7) / 8);
  int n = 0;
  if (a.inter) {
    if ((q == 4 ? launch_pdl(k_solute_pre<4>, grd, blk, 0, s, a) : launch_pdl(k_solute_pre<9>, grd, blk, 0, s, a)) !=
        cudaSuccess)
      return -1;
    n++;
  }
  const cudaError_t e = q == 4 ? launch_pdl(k_solute<4>, grd, blk, 0, s, a) : launch_pdl(k_solute<9>, grd, blk, 0, s, a);
  return e == cudaSuccess ? n + 1 : -1;
}

int launch_surface_list(const GrowthArgs &a, cudaStream_t s) {
  dim3 blk(32, 8), grd((a.g.nx + 31) / 32, (a.rhi - a.rlo + 7) / 8);
  return launch_pdl(k_surface_list, grd, blk, 0, s, a) == cudaSuccess ? 1 : -1;
}

int launch_growth(int storage, const GrowthArgs &a, cudaStream_t s) {
  if (a.slist) {
    const dim3 grd(a.sblocks), blk(256);
    cudaError_t e;
    switch (storage) {
      case ST_FP16: e = launch_pdl(k_grow_list<__half>, grd, blk, 0, s, a); break;
      case ST_BF16: e = launch_pdl(k_grow_list<__nv_bfloat16>, grd, blk, 0, s, a); break;
      default: e = launch_pdl(k_grow_list<float>, grd, blk, 0, s, a); break;
    }
    return e == cudaSuccess ? 1 : -1;
  }
  dim3 blk(32, 8), grd((a.g.nx + 31) / 32, (a.rhi - a.rlo + 7) / 8);
  if (launch_pdl(k_gather_grow, grd, blk, 0, s, a) != cudaSuccess) return -1;
  switch (storage) {
    case ST_FP16: return launch_pdl(k_apply_flips<__half>, dim3(1), dim3(256), 0, s, a) == cudaSuccess ? 2 : -1;
    case ST_BF16: return launch_pdl(k_apply_flips<__nv_bfloat16>, dim3(1), dim3(256), 0, s, a) == cudaSuccess ? 2 : -1;
    default: return launch_pdl(k_apply_flips<float>, dim3(1), dim3(256), 0, s, a) == cudaSuccess ? 2 : -1;
  }
}

}  // namespace lbk
