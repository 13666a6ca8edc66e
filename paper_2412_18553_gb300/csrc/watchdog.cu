// Self-test of the device watchdog: a bounded wait that is bound to expire.
#include "ptx_sm100.cuh"
#include "te_internal.h"

namespace te {

// Site code reported in the error word by the self-test.
constexpr unsigned int SITE_SELFTEST = 99;

__global__ void k_watchdog_selftest(uint64_t limit_ns, unsigned int* err) {
  __shared__ __align__(8) uint64_t bar;
  ptx::mbar_init(&bar, 1);
  ptx::fence_barrier_init();
  // nothing arrives on bar: phase 0 never completes
  if (!ptx::mbar_wait(&bar, 0, limit_ns)) {
    if (atomicOr(err, ERR_WAIT_TIMEOUT) == 0) {
      err[1] = SITE_SELFTEST;
      err[2] = blockIdx.x;
    }
  }
}

}  // namespace te

using namespace te;

extern "C" te_status te_watchdog_selftest(te_handle hh, uint64_t limit_ns, te_stream_t ss) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return fail(TE_EINVAL, "null handle");
  if (limit_ns < 1000000ull || limit_ns > 10000000000ull)
    return fail(TE_EINVAL, "limit_ns must lie in [1 ms, 10 s] (got %llu)", (unsigned long long)limit_ns);
  if (h->cc_major < 9) return fail(TE_EUNSUPPORTED, "mbarrier waits need compute capability 9.0 or newer");
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != h->device && cudaSetDevice(h->device) != cudaSuccess)
    return fail(TE_ECUDA, "cudaSetDevice(%d) failed", h->device);
  k_watchdog_selftest<<<1, 1, 0, reinterpret_cast<cudaStream_t>(ss)>>>(limit_ns, h->d_err);
  cudaError_t e = cudaGetLastError();
  ++h->n_launches;
  if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
  if (e != cudaSuccess) return fail(TE_ECUDA, "self-test launch: %s", cudaGetErrorString(e));
  return TE_OK;
}
