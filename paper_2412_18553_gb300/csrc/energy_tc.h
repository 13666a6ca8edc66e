// Launch interface of the TMA-fed energy epilogue (energy_tc.cu).
#pragma once
#include <cuda.h>

#include <algorithm>

#include "te_internal.h"

namespace te {

struct EnergyLaunch {
  int o, v, nslots, cw, num_sms;
  int64_t nbt, t0;
  const float* gbuf;           // cube-major G: [slot][g][X][Y][Z][cw planes][512 swizzled], X,Y,Z < ceil(v/8)
  const CUtensorMap* map_ovs;  // ovs32 [o][v][o][vq], 4D (b, j, a, i), box (8, 1, 8, 1)
  const CUtensorMap* map_t1;   // t1 [o][vq], 2D (a, i), box (8, 1)
  const Triple* triples;
  const double* eps_o;
  const double* eps_v;
  double* partials;  // [nslots][energy_tc_grid(num_sms, nslots*nbt)][ENERGY_TC_WARPS], zeroed by the launch
  unsigned int* err;
  unsigned long long wait_ns;
};

// Layout of one 8x8x8 G cube (shared by the contraction epilogue that writes it
// and the energy kernel that reads it): element (u, w, z) of a plane sits at
//   u*64 + (w ^ (u & 3))*8 + (z ^ h),  h = (u & 3) | (((w ^ u) >> 2 & 1) << 2),
// an XOR swizzle under which every access pattern of the energy kernel (one
// of the three local indices fixed per warp, the other two spread over 4 x 8
// threads) touches 32 distinct shared-memory banks.  A cube holds one plane
// (FP32) or two (hi plane, then lo plane) of 512 floats.
__host__ __device__ __forceinline__ int cube_row(int u, int w) { return u * 64 + (w ^ (u & 3)) * 8; }
__host__ __device__ __forceinline__ int cube_zx(int u, int w) { return (u & 3) | ((((w ^ u) >> 2) & 1) << 2); }
__host__ __device__ __forceinline__ int cube_off(int u, int w, int z) { return cube_row(u, w) + (z ^ cube_zx(u, w)); }

constexpr int ENERGY_TC_WARPS = 16;
int64_t energy_tc_grid(int num_sms, int64_t items);
size_t energy_tc_smem(int cw);
cudaError_t launch_energy_tc(const EnergyLaunch& e, cudaStream_t s);

}  // namespace te
