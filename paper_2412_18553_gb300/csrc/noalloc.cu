// Float64 E(T) without any device allocation: every scratch byte of the
// float64 path (prepared operand copies, G blocks, partial sums, triple table)
// is carved from one fixed-size array that the library image carries.
#include "te_internal.h"

namespace te {

// The scratch array.  It is part of the loaded library image, so every GPU
// that loads libtenergy holds these bytes until the process exits.
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(64) << 20;  // 64 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// In host code the array's name is only a host-side stand-in, never a usable
// device pointer: each call asks the runtime for its address on the current
// device (no caching, so a device reset that reloads the image is harmless).

// Canonical unique triples (lexicographic i >= j >= k, i = j = k left out):
// thread i writes the C(i+2,2) - 1 triples whose first index is i, starting
// at C(i+2,3) - i.
__global__ void k_noalloc_fill_triples(Triple* out, int nocc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nocc) return;
  int64_t t = (int64_t)i * (i + 1) * (i + 2) / 6 - i;
  for (int j = 0; j <= i; ++j)
    for (int k = 0; k <= j; ++k) {
      if (i == j && j == k) continue;
      out[t++] = Triple{i, j, k, (i == j || j == k) ? 3 : 6};
    }
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Bytes of scratch for a cluster processed `slots` triples at a time.
static size_t noalloc_bytes(int64_t o, int64_t v, int64_t slots) {
  const int64_t nt = num_unique_triples(o);
  const int64_t nbt = energy_num_block_triples(v);
  size_t b = 0;
  b += align256(sizeof(Triple) * (size_t)std::max<int64_t>(1, nt));
  b += align256(sizeof(double) * (size_t)(o * v * v * o));         // t2L
  b += align256(sizeof(double) * (size_t)(o * o * v * o));         // nooT
  b += align256(sizeof(double) * (size_t)(o * v * o * v));         // ovs
  b += align256(sizeof(double) * (size_t)(slots * 3 * v * v * v));  // G blocks
  b += align256(sizeof(double) * (size_t)(slots * nbt));           // partials
  b += align256(sizeof(double) * (size_t)std::max<int64_t>(1, nt));  // shares
  return b;
}

}  // namespace te

using namespace te;

extern "C" te_status t_energy_fp64_noalloc(const te_cluster* c, double* e_out, te_stream_t ss) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(ss);
  if (!c || !e_out) return fail(TE_EINVAL, "null cluster descriptor or e_out");
  if (c->nocc < 1 || c->nvir < 1) return fail(TE_EINVAL, "nocc and nvir must be >= 1");
  if (c->nocc > 1024 || c->nvir > 4096) return fail(TE_EINVAL, "cluster too large for the no-allocation entry point");
  const int64_t o = c->nocc, v = c->nvir;
  // size check before any device memory is touched
  if (noalloc_bytes(o, v, 1) > NOALLOC_SCRATCH_BYTES)
    return fail(TE_EINVAL,
                "cluster nocc=%lld nvir=%lld needs %zu bytes of scratch; the no-allocation entry point "
                "has a fixed %zu-byte scratch array",
                (long long)o, (long long)v, noalloc_bytes(o, v, 1), NOALLOC_SCRATCH_BYTES);
  if (!c->eps_o || !c->eps_v || !c->ovvv || !c->ooov || !c->ovov || !c->t1 || !c->t2)
    return fail(TE_EINVAL, "null array pointer in cluster descriptor");

  void* base = nullptr;
  {
    const cudaError_t e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
    if (e != cudaSuccess || !base) {
      cudaGetLastError();
      return fail(TE_ECUDA, "cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
    }
  }

  // every denominator must be negative: max eps_o < min eps_v
  double eo[1024], ev[4096];
  if (cudaMemcpyAsync(eo, c->eps_o, o * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(ev, c->eps_v, v * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(TE_ECUDA, "reading orbital energies failed: %s", cudaGetErrorString(cudaGetLastError()));
  double mo = -1e300, mv = 1e300;
  for (int64_t i = 0; i < o; ++i) {
    if (!(eo[i] == eo[i]) || eo[i] > 1e300 || eo[i] < -1e300) return fail(TE_EINVAL, "non-finite eps_o");
    mo = eo[i] > mo ? eo[i] : mo;
  }
  for (int64_t a = 0; a < v; ++a) {
    if (!(ev[a] == ev[a]) || ev[a] > 1e300 || ev[a] < -1e300) return fail(TE_EINVAL, "non-finite eps_v");
    mv = ev[a] < mv ? ev[a] : mv;
  }
  if (!(mo < mv)) return fail(TE_EINVAL, "max(eps_o) = %g must be below min(eps_v) = %g", mo, mv);

  // as many triples per launch as the scratch holds (at most 64)
  int64_t slots = 1;
  const int64_t nt = num_unique_triples(o);
  while (slots < 64 && slots < nt && noalloc_bytes(o, v, slots * 2) <= NOALLOC_SCRATCH_BYTES) slots *= 2;

  char* p = static_cast<char*>(base);
  size_t off = 0;
  auto take = [&](size_t bytes) -> void* {
    void* r = p + off;
    off += align256(bytes);
    return r;
  };
  const int64_t nbt = energy_num_block_triples(v);
  Triple* triples = static_cast<Triple*>(take(sizeof(Triple) * (size_t)std::max<int64_t>(1, nt)));
  Prepared P{};
  P.o = (int)o;
  P.v = (int)v;
  P.eps_o = c->eps_o;
  P.eps_v = c->eps_v;
  P.ovvv = c->ovvv;
  P.t2 = c->t2;
  P.t1 = c->t1;
  P.t2L = static_cast<double*>(take(sizeof(double) * (size_t)(o * v * v * o)));
  P.nooT = static_cast<double*>(take(sizeof(double) * (size_t)(o * o * v * o)));
  P.ovs = static_cast<double*>(take(sizeof(double) * (size_t)(o * v * o * v)));
  P.ovs32 = nullptr;
  P.t1_32 = nullptr;
  double* gbuf = static_cast<double*>(take(sizeof(double) * (size_t)(slots * 3 * v * v * v)));
  double* partials = static_cast<double*>(take(sizeof(double) * (size_t)(slots * nbt)));
  double* shares = static_cast<double*>(take(sizeof(double) * (size_t)std::max<int64_t>(1, nt)));

  if (nt == 0) {
    if (cudaMemsetAsync(e_out, 0, sizeof(double), s) != cudaSuccess) return fail(TE_ECUDA, "memset failed");
    return TE_OK;
  }
  // Every scratch byte read below is first written by this call: the triple
  // table, the prepared copies, each G block (all x,y,z < v), each partial
  // and each share; nothing has to start at zero.
  k_noalloc_fill_triples<<<(unsigned)((o + 127) / 128), 128, 0, s>>>(triples, (int)o);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_prep_fp64(c, &P, s);
  for (int64_t t0 = 0; e == cudaSuccess && t0 < nt; t0 += slots) {
    const int ns = (int)std::min<int64_t>(slots, nt - t0);
    e = launch_gemm_fp64(&P, triples, t0, ns, gbuf, s);
    if (e == cudaSuccess) e = launch_energy_f64(&P, triples, t0, ns, gbuf, partials, nbt, s);
    if (e == cudaSuccess) e = launch_reduce_triples(partials, nbt, triples, t0, ns, shares + t0, s);
  }
  if (e == cudaSuccess) e = launch_reduce_total(shares, nt, e_out, s);
  if (e != cudaSuccess) return fail(TE_ECUDA, "launch failed: %s", cudaGetErrorString(e));
  return TE_OK;
}
