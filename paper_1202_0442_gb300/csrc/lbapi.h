// lbapi.h -- what the files of the library's host side share: the host
// direction tables and five functions (lb2d_api.cu defines four of them,
// lb2d_slab.cu exchange_slabs, which lb_iteration calls for a lattice held
// as one slab).
#pragma once

#include <cstddef>

#include "lbctx.h"

// the lattice directions on the host: D2Q9 weights and vectors, D2Q4 vectors
constexpr double W9D[9] = {4.0 / 9,  1.0 / 9,  1.0 / 9,  1.0 / 9, 1.0 / 9,
                           1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
constexpr int EXD[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
constexpr int EYD[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
constexpr int EX4D[4] = {1, 0, -1, 0};
constexpr int EY4D[4] = {0, 1, 0, -1};

// bytes of one stored population (FP32: 4, FP16/BF16: 2)
size_t storage_bytes(int st);
// make ctx's device current; LB_E_CUDA if that fails
int set_device(lb_ctx *ctx);
// move the painted setup to the GPU (first call that needs device state);
// LB_OK at once if that has happened
int commit(lb_ctx *ctx);
// read every deferred thermo record still waiting, oldest first; the first
// record's LB_E_NAN or LB_E_TIMEOUT
int read_all_deferred(lb_ctx *ctx);
// the halo rows of n slabs of one lattice held in this process, device to
// device (lb2d_slab.cu)
int exchange_slabs(lb_ctx *const *ctxs, int n);
