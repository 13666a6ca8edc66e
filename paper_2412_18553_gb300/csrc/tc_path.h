// Tensor-core (tcgen05) path for the mixed precision modes.
#pragma once
#include "te_internal.h"

namespace te {
// df (nullable): ovvv formed from density-fitting factors (c->ovvv unread)
te_status run_tc(Handle* h, const te_cluster* c, te_precision p, int64_t t_begin, int64_t t_end,
                 double* e_tri_out, double* e_total_out, cudaStream_t s, const te_df* df = nullptr);
te_status tc_workspace_bytes(Handle* h, const te_cluster* c, te_precision p, size_t* bytes,
                             const te_df* df = nullptr);
// n clusters in rounds of multi-cluster launches (every member's operands
// prepared first); e_out[x] = E(T) of cluster x.  tc_batched_bytes: the
// workspace it needs (the tuned tile shapes must be known already).
te_status tc_batched_bytes(Handle* h, const te_cluster* cs, int64_t n, te_precision p, size_t* bytes);
te_status run_tc_batched(Handle* h, const te_cluster* cs, int64_t n, te_precision p, double* e_out,
                         cudaStream_t s);
void destroy_tc_state(Handle* h);
// Time the candidate tile shapes of the contraction for this cluster's (nocc,
// nvir, mode) on its first triples and remember the fastest in the handle.
// Synchronous; must not run inside a stream capture.
te_status tc_autotune(Handle* h, const te_cluster* c, te_precision p, cudaStream_t s);

// Exact-slice planes (ns = 4 or 5 7-bit BF16 slices) of the contraction
// operands, for the strided exact-slice GEMMs to read.
// Element e of slice s of an array sits at base + s * plane + e, e being
//   ovvv[p,x,y,d]:  p * ovvv_p + (x v + y) vp + d
//   t2[r,q,z,d]:    (r o + q) * t2_rq + z vp + d
//   t2L[q,x,y,l] = t2[l,q,x,y]:    q * t2L_q + (x v + y) op + l
//   nooT[p,r,z,l] = -ooov[p,l,r,z]: (p o + r) * nooT_pr + z op + l
// and the value of an element is 2^e times the sum of its slices, e the scale
// exponent of its row group (device arrays): e_ovvv[p], e_t2[r o + q],
// e_t2L[q], e_nooT[p o + r].  Each strided GEMM reads one group of each
// operand, so a group far below its array's largest entry keeps every bit.
struct SliceSet {
  const void *ovvv, *t2, *t2L, *nooT;  // __nv_bfloat16 planes
  int64_t ovvv_plane, t2_plane, t2L_plane, nooT_plane;
  int64_t ovvv_p, t2_rq, t2L_q, nooT_pr;
  int vp, op;
  int ns;  // slices per element
  const int *e_ovvv, *e_t2, *e_t2L, *e_nooT;
};
// Bytes the slice planes need; tc_prepare_slices lays them out from base
// (256-byte aligned) and launches the slicing on s.
size_t tc_slices_bytes(int o, int v, int ns = 4);
te_status tc_prepare_slices(const te_cluster* c, void* base, SliceSet* out, int num_sms, cudaStream_t s,
                            int ns = 4);
}  // namespace te
