// Launch interface of the TMA-fed energy epilogue (energy_tc.cu).
#pragma once
#include <cuda.h>

#include <algorithm>

#include "te_internal.h"

namespace te {

// A launch of the contraction and energy kernels covers up to TC_MAX_CL
// clusters and TC_MAX_PIECES pieces: a piece is one cluster's run of
// consecutive canonical triples, each with its own G slot.  The per-cluster
// constants, tensor maps and pieces travel as kernel parameters.
constexpr int TC_MAX_CL = 8;
constexpr int TC_MAX_PIECES = 48;

struct TcPiece {
  int cl;          // cluster (index into the launch's cluster table)
  int ns;          // triples (G slots) of the piece
  int slot0;       // first G slot, counted over the launch's pieces
  int64_t t0;      // first canonical triple
  int64_t tile0;   // first contraction tile of the piece
  int64_t item0;   // first energy item of the piece
  int64_t nbt;     // energy items per triple (the cluster's block triples)
  float* gbuf;     // G of the piece's first slot
  double* shares;  // per-triple shares of the piece (ns doubles)
};

// Per-cluster constants of the energy kernel.
struct EnergyCl {
  int o, v, nb;
  int64_t nbt;          // block triples X >= Y >= Z of 8-wide virtual blocks
  const double* eps_o;  // caller's arrays
  const double* eps_v;
};

struct EnergyLaunch {
  int ncl, npieces, cw, num_sms, nslots;  // nslots: G slots over all pieces
  int64_t items;                          // sum over pieces of ns * nbt
  EnergyCl cl[TC_MAX_CL];
  TcPiece pc[TC_MAX_PIECES];
  const CUtensorMap* map_ovs[TC_MAX_CL];  // ovs32 [o][v][o][vq], 4D (b, j, a, i), box (8, 1, 8, 1)
  const CUtensorMap* map_t1[TC_MAX_CL];   // t1 [o][vq], 2D (a, i), box (8, 1)
  const Triple* triples;
  double* partials;  // [nslots][energy_tc_grid(num_sms, items)][ENERGY_TC_WARPS], zeroed by the launch
  unsigned int* err;
  unsigned long long wait_ns;
};

// Per-triple shares of every slot of a launch: shares[t] = (m_t / 3) times the
// fixed-order sum of the slot's nper = grid x ENERGY_TC_WARPS partials.  A
// block takes the same items of a triple in the same order in any launch (the
// grid is one block per SM), so a triple's share has the same bits in a
// single-cluster call and in a batch.
cudaError_t launch_reduce_pieces(const double* partials, int nper, const Triple* triples,
                                 const TcPiece* pieces, int npieces, int nslots, cudaStream_t s);

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

// Orbit-major placement of the G cubes.  The energy kernel's work item is a
// block triple S0 >= S1 >= S2 of 8-wide virtual blocks; it needs, for each of
// the 3 G blocks g, the cubes at the 6 block orders
//   pid: (S0,S1,S2) (S0,S2,S1) (S1,S0,S2) (S1,S2,S0) (S2,S0,S1) (S2,S1,S0).
// They are stored contiguously as [slot][bt][g][pid][CW planes][512], so one
// bulk copy brings an item's 18 cubes.  A cube (X,Y,Z) whose indices repeat
// serves several orders and is stored once per order.
__host__ __device__ __forceinline__ int64_t block_triple_index(int s0, int s1, int s2) {
  return (int64_t)s0 * (s0 + 1) * (s0 + 2) / 6 + (int64_t)s1 * (s1 + 1) / 2 + s2;
}

// bt of the sorted block triple of cube (X,Y,Z) and the set of orders pid
// (bit pid) at which that cube appears
__host__ __device__ __forceinline__ void orbit_slots(int X, int Y, int Z, int64_t* bt, unsigned* mask) {
  int s0 = X, s1 = Y, s2 = Z, t;
  if (s0 < s1) { t = s0; s0 = s1; s1 = t; }
  if (s1 < s2) { t = s1; s1 = s2; s2 = t; }
  if (s0 < s1) { t = s0; s0 = s1; s1 = t; }
  *bt = block_triple_index(s0, s1, s2);
  *mask = (unsigned)(s0 == X && s1 == Y && s2 == Z) | ((unsigned)(s0 == X && s2 == Y && s1 == Z) << 1) |
          ((unsigned)(s1 == X && s0 == Y && s2 == Z) << 2) | ((unsigned)(s1 == X && s2 == Y && s0 == Z) << 3) |
          ((unsigned)(s2 == X && s0 == Y && s1 == Z) << 4) | ((unsigned)(s2 == X && s1 == Y && s0 == Z) << 5);
}

// floats of the G buffer per triple slot
__host__ __device__ __forceinline__ int64_t g_slot_floats(int v, int cw) {
  const int64_t nb = (v + 7) / 8;
  return nb * (nb + 1) * (nb + 2) / 6 * 18 * 512 * cw;
}

constexpr int ENERGY_TC_WARPS = 16;
int64_t energy_tc_grid(int num_sms, int64_t items);
size_t energy_tc_smem(int cw);
cudaError_t launch_energy_tc(const EnergyLaunch& e, cudaStream_t s);

}  // namespace te
