// Tensor-core (tcgen05) path for the mixed precision modes.
#pragma once
#include "te_internal.h"

namespace te {
te_status run_tc(Handle* h, const te_cluster* c, te_precision p, int64_t t_begin, int64_t t_end,
                 double* e_tri_out, double* e_total_out, cudaStream_t s);
te_status tc_workspace_bytes(Handle* h, const te_cluster* c, te_precision p, size_t* bytes);
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

// Exact-slice planes (four 7-bit BF16 slices) of the contraction operands,
// as the 7-bit mode prepares them, for other kernels to read by strides.
// Element e of slice s of an array sits at base + s * plane + e, e being
//   ovvv[p,x,y,d]:  p * ovvv_p + (x v + y) vp + d
//   t2[r,q,z,d]:    (r o + q) * t2_rq + z vp + d
//   t2L[q,x,y,l] = t2[l,q,x,y]:    q * t2L_q + (x v + y) op + l
//   nooT[p,r,z,l] = -ooov[p,l,r,z]: (p o + r) * nooT_pr + z op + l
// and the value of an array element is 2^exps[w] times the sum of its slices
// (w = 0 ovvv, 1 t2, 2 t2L, 3 nooT; exps lives on the device).
struct SliceSet {
  const void *ovvv, *t2, *t2L, *nooT;  // __nv_bfloat16 planes
  int64_t ovvv_plane, t2_plane, t2L_plane, nooT_plane;
  int64_t ovvv_p, t2_rq, t2L_q, nooT_pr;
  int vp, op;
  const int* exps;
};
// Bytes the slice planes need; tc_prepare_slices lays them out from base
// (256-byte aligned) and launches the slicing on s.
size_t tc_slices_bytes(int o, int v);
te_status tc_prepare_slices(const te_cluster* c, void* base, SliceSet* out, cudaStream_t s);
}  // namespace te
