// Launch interface of the TMA-fed energy epilogue (energy_tc.cu).
#pragma once
#include <cuda.h>

#include <algorithm>

#include "te_internal.h"

namespace te {

struct EnergyLaunch {
  int o, v, nslots, cw, num_sms;
  int64_t nbt, t0;
  const CUtensorMap* map_g;    // G buffer, 5D (z*cw, y, x, g, slot), FP32, box (8cw, 8, 8, 1, 1)
  const CUtensorMap* map_ovs;  // ovs32 [o][v][o][vq], 4D (b, j, a, i), box (8, 1, 8, 1)
  const CUtensorMap* map_t1;   // t1 [o][vq], 2D (a, i), box (8, 1)
  const CUtensorMap* map_eps;  // eps_v copy [v], 1D FP64, box 8
  const Triple* triples;
  const double* eps_o;
  double* partials;
  unsigned int* err;
  unsigned long long wait_ns;
};

size_t energy_tc_smem(int cw);
cudaError_t launch_energy_tc(const EnergyLaunch& e, cudaStream_t s);

}  // namespace te
