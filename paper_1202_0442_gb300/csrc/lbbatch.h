// lbbatch.h -- descriptors of the batched multi-lattice launch.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace lbk {

// one lattice of a batch (periodic, one component, body forces only)
struct BatchLat {
  int nx, ny, pitch, mw;
  size_t plane;
  void *buf[2];        // the lattice's two population buffers
  int cur;             // buf[cur] is the input of the batch's parity-0 launch
  const uint32_t *mask;
  const uint16_t *nbc; // per node slot: solid bits of the 3 x 3 neighbourhood
  float rho_ref, scale, inv_scale, tau, omega, fx, fy, ax, ay;
  int pm;              // momentum as an exact hi + lo sum
  int sr;              // 16-bit stores rounded stochastically
};

struct BatchLaunch {
  const BatchLat *lat;   // device array
  const int4 *tiles;     // device array of (lattice, x0, y0, 0)
  int ntiles;
  int grid;              // persistent grid size
  int shape;             // tile shape id (batch_shape_tx/ty)
  int dynamic;           // 0: static round robin, 1: atomic work counter
  unsigned int *counters; // two work counters (one per parity)
  unsigned int *tick;     // two launch counters (one per parity): the
                          // stochastic-rounding dither changes every launch
};

constexpr int BATCH_SHAPES = 6;
int batch_shape_tx(int shape);
int batch_shape_ty(int shape);
int batch_occupancy(int storage, int shape);
int launch_batch(int storage, const BatchLaunch &b, int parity, cudaStream_t s);

}  // namespace lbk
