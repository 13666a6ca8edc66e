// Device-side checks of the input values, launched at the head of every call
// on the caller's stream (no host synchronisation):
//  * every entry of the seven arrays is finite;
//  * max(eps_o) < min(eps_v), so that every denominator D of Eq. D is
//    negative (the orbital energies need not be sorted).
// A violation sets ERR_BAD_INPUT in the handle's error word with the site
// (1..7: the array, in the order eps_o, eps_v, ovvv, ooov, ovov, t1, t2;
// 8: the ordering of the orbital energies; 9, 10: the density-fitting
// factors Bov, Bvv) and the cluster index; te_sync
// reports it as TE_EINVAL.  The kernels that follow still run (they never
// fault on such values); their results are then unspecified.
#include <algorithm>

#include "te_internal.h"

namespace te {

namespace {

constexpr unsigned long long EXP_MASK = 0x7FF0000000000000ull;

constexpr int kCheckArrays = 9;

struct CheckArgs {
  const unsigned long long* p[kCheckArrays];
  int64_t n[kCheckArrays];
  unsigned int site[kCheckArrays];  // reported for a non-finite entry of array w (n = 0: unused)
  const double* eps_o;
  const double* eps_v;
  int o, v;
  unsigned int cluster;
};

__device__ __forceinline__ bool nonfinite(unsigned long long x) { return (x & EXP_MASK) == EXP_MASK; }

__device__ __forceinline__ void report(unsigned int* err, unsigned int site, unsigned int cluster) {
  if (atomicOr(err, ERR_BAD_INPUT) == 0) {
    err[1] = site;
    err[2] = cluster;
  }
}

__global__ void __launch_bounds__(256) k_check_inputs(const CheckArgs a, unsigned int* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  unsigned int bad = 0;
  for (int w = 0; w < kCheckArrays; ++w) {
    const unsigned long long* q = a.p[w];
    const int64_t n = a.n[w];
    bool any = false;
    int64_t i = tid;
    for (; i + 3 * stride < n; i += 4 * stride) {  // four loads in flight
      const unsigned long long x0 = __ldg(q + i), x1 = __ldg(q + i + stride);
      const unsigned long long x2 = __ldg(q + i + 2 * stride), x3 = __ldg(q + i + 3 * stride);
      any |= nonfinite(x0) | nonfinite(x1) | nonfinite(x2) | nonfinite(x3);
    }
    for (; i < n; i += stride) any |= nonfinite(__ldg(q + i));
    if (any && bad == 0) bad = a.site[w];
  }
  if (bad) report(err, bad, a.cluster);

  if (blockIdx.x == 0) {  // max(eps_o) < min(eps_v)
    __shared__ double smax[8], smin[8];
    double mo = -1.0e308, mv = 1.0e308;
    for (int i = threadIdx.x; i < a.o; i += blockDim.x) mo = fmax(mo, a.eps_o[i]);
    for (int i = threadIdx.x; i < a.v; i += blockDim.x) mv = fmin(mv, a.eps_v[i]);
    for (int off = 16; off > 0; off >>= 1) {
      mo = fmax(mo, __shfl_down_sync(0xffffffffu, mo, off));
      mv = fmin(mv, __shfl_down_sync(0xffffffffu, mv, off));
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
      smax[warp] = mo;
      smin[warp] = mv;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        mo = fmax(mo, smax[w]);
        mv = fmin(mv, smin[w]);
      }
      if (!(mo < mv)) report(err, 8u, a.cluster);
    }
  }
}

}  // namespace

cudaError_t launch_check_inputs(const te_cluster* c, int64_t cluster, unsigned int* err, int num_sms,
                                cudaStream_t s, const te_df* df) {
  const int64_t o = c->nocc, v = c->nvir, P = df ? df->naux : 0;
  CheckArgs a{};
  // with density-fitting factors, ovvv is not read: Bov and Bvv instead
  const double* ptr[kCheckArrays] = {c->eps_o, c->eps_v, df ? nullptr : c->ovvv, c->ooov, c->ovov, c->t1, c->t2,
                                     df ? df->Bov : nullptr, df ? df->Bvv : nullptr};
  const int64_t n[kCheckArrays] = {o, v, df ? 0 : o * v * v * v, o * o * o * v, o * v * o * v, o * v, o * o * v * v,
                                   P * o * v, P * v * v};
  int64_t nmax = 0;
  for (int w = 0; w < kCheckArrays; ++w) {
    a.p[w] = reinterpret_cast<const unsigned long long*>(ptr[w]);
    a.n[w] = n[w];
    a.site[w] = (unsigned int)w + 1u + (w >= 7 ? 1u : 0u);  // 1..7, then 9, 10
    nmax = std::max(nmax, n[w]);
  }
  a.eps_o = c->eps_o;
  a.eps_v = c->eps_v;
  a.o = (int)o;
  a.v = (int)v;
  a.cluster = (unsigned int)cluster;
  const int64_t want = (nmax + 4 * 256 - 1) / (4 * 256);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, 4LL * std::max(1, num_sms)));
  k_check_inputs<<<grid, 256, 0, s>>>(a, err);
  return cudaGetLastError();
}

// The MP2 step's inputs: eps_o (site 1), eps_v (site 2), the DF factor's ov
// block (site 9), and the eps ordering (site 8).
cudaError_t launch_check_mp2(const double* eps_o, int64_t o, const double* eps_v, int64_t v, const double* Bov,
                             int64_t nB, int64_t cluster, unsigned int* err, int num_sms, cudaStream_t s) {
  CheckArgs a{};
  const double* ptr[3] = {eps_o, eps_v, Bov};
  const int64_t n[3] = {o, v, nB};
  const unsigned int site[3] = {1u, 2u, 9u};
  for (int w = 0; w < kCheckArrays; ++w) {
    const int q = w < 3 ? w : 2;  // the unused entries repeat Bov with no elements
    a.p[w] = reinterpret_cast<const unsigned long long*>(ptr[q]);
    a.n[w] = w < 3 ? n[q] : 0;
    a.site[w] = site[q];
  }
  a.eps_o = eps_o;
  a.eps_v = eps_v;
  a.o = (int)o;
  a.v = (int)v;
  a.cluster = (unsigned int)cluster;
  const int64_t want = (nB + 4 * 256 - 1) / (4 * 256);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, 4LL * std::max(1, num_sms)));
  k_check_inputs<<<grid, 256, 0, s>>>(a, err);
  return cudaGetLastError();
}

}  // namespace te
