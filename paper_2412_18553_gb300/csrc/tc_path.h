// Tensor-core (tcgen05) path for the mixed precision modes.
#pragma once
#include "te_internal.h"

namespace te {
te_status run_tc(Handle* h, const te_cluster* c, te_precision p, int64_t t_begin, int64_t t_end,
                 double* e_tri_out, double* e_total_out, cudaStream_t s);
te_status tc_workspace_bytes(Handle* h, const te_cluster* c, te_precision p, size_t* bytes);
void destroy_tc_state(Handle* h);
// Time the candidate tile shapes of the contraction for this cluster's (nocc,
// nvir, mode) on its first triples and remember the fastest in the handle.
// Synchronous; must not run inside a stream capture.
te_status tc_autotune(Handle* h, const te_cluster* c, te_precision p, cudaStream_t s);
}  // namespace te
