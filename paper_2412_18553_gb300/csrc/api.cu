// C-ABI entry points of libtenergy (declared in include/tenergy.h): argument
// validation, handle workspace, and the launch sequence of each call.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <vector>

#include "te_internal.h"
#include "tc_path.h"

namespace te {

static thread_local char g_last_error[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
}

te_status fail(te_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return st;
}

std::vector<Triple> unique_triples(int nocc) {
  std::vector<Triple> out;
  for (int i = 0; i < nocc; ++i)
    for (int j = 0; j <= i; ++j)
      for (int k = 0; k <= j; ++k) {
        if (i == j && j == k) continue;
        const int m = (i == j || j == k) ? 3 : 6;
        out.push_back(Triple{i, j, k, m});
      }
  return out;
}

int64_t num_unique_triples(int64_t nocc) { return nocc * (nocc + 1) * (nocc + 2) / 6 - nocc; }

void drop_graphs(Handle* h) {
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Bump allocator over the handle workspace.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <typename T>
  T* take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += n * sizeof(T);
    return p;
  }
};

static te_status ensure_workspace(Handle* h, size_t bytes) {
  if (h->ws_bytes >= bytes) return TE_OK;
  if (h->ws_limit && bytes > h->ws_limit)
    return fail(TE_ENOMEM, "workspace of %zu bytes needed, above the handle's limit of %zu bytes", bytes,
                h->ws_limit);
  if (h->capturing) return fail(TE_EUNSUPPORTED, "workspace growth inside a graph capture");
  drop_graphs(h);  // captured graphs hold the old workspace's addresses
  if (h->ws) {
    cudaDeviceSynchronize();  // no launch may still read the old workspace
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  // room to grow a little without reallocating; at most 1 GiB of it, so a
  // workspace of a hundred gigabytes does not crowd out the caller's arrays
  size_t want = bytes + std::min(bytes / 8, (size_t)1 << 30);
  if (h->ws_limit) want = std::min(want, h->ws_limit);
  if (h->log) std::fprintf(stderr, "[tenergy] workspace: %zu bytes (needed %zu)\n", want, bytes);
  if (cudaMalloc(&h->ws, want) != cudaSuccess) {
    cudaGetLastError();
    h->ws = nullptr;
    if (cudaMalloc(&h->ws, bytes) != cudaSuccess) {
      cudaGetLastError();
      h->ws = nullptr;
      return fail(TE_ENOMEM, "workspace allocation of %zu bytes failed", bytes);
    }
    h->ws_bytes = bytes;
    return TE_OK;
  }
  h->ws_bytes = want;
  return TE_OK;
}

// The canonical order is prefix-closed (the triples of nocc = n are the first
// ones of any larger nocc), so one table for the largest nocc serves all.
static te_status ensure_triples(Handle* h, int nocc) {
  if (h->triples_nocc >= nocc) return TE_OK;
  if (h->capturing) return fail(TE_EUNSUPPORTED, "triple table growth inside a graph capture");
  drop_graphs(h);
  std::vector<Triple> t = unique_triples(nocc);
  const size_t need = std::max<size_t>(1, t.size());
  if (h->triples_cap < need) {
    if (h->d_triples) {
      cudaDeviceSynchronize();
      cudaFree(h->d_triples);
      h->d_triples = nullptr;
    }
    if (cudaMalloc(&h->d_triples, need * sizeof(Triple)) != cudaSuccess) {
      cudaGetLastError();
      h->d_triples = nullptr;
      h->triples_cap = 0;
      h->triples_nocc = -1;
      return fail(TE_ENOMEM, "triple table allocation failed");
    }
    h->triples_cap = need;
  } else {
    cudaDeviceSynchronize();  // earlier launches may still read the table
  }
  if (!t.empty() && cudaMemcpy(h->d_triples, t.data(), t.size() * sizeof(Triple),
                               cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(TE_ECUDA, "triple table upload failed: %s", cudaGetErrorString(cudaGetLastError()));
  h->triples_nocc = nocc;
  return TE_OK;
}

static te_status host_check(const Handle* h, const te_cluster* c, te_precision p, bool need_ovvv = true) {
  if (!h) return fail(TE_EINVAL, "null handle");
  if (!c) return fail(TE_EINVAL, "null cluster descriptor");
  if (c->nocc < 1 || c->nvir < 1) return fail(TE_EINVAL, "nocc and nvir must be >= 1 (got %lld, %lld)",
                                              (long long)c->nocc, (long long)c->nvir);
  if (c->nocc > 2048 || c->nvir > 4096)
    return fail(TE_EUNSUPPORTED, "cluster too large (nocc <= 2048, nvir <= 4096)");
  if (!c->eps_o || !c->eps_v || (need_ovvv && !c->ovvv) || !c->ooov || !c->ovov || !c->t1 || !c->t2)
    return fail(TE_EINVAL, "null array pointer in cluster descriptor");
  if (p != TE_FP64 && p != TE_TF32 && p != TE_BF16X3 && p != TE_TF32X3 && p != TE_OZAKI)
    return fail(TE_EINVAL, "unknown precision mode %d", (int)p);
  return TE_OK;
}

// Host checks (descriptor, sizes, pointers), then the device-side value
// checks (finite entries, max eps_o < min eps_v) launched on s: no host
// synchronisation, the result is reported by te_sync.
static te_status validate(Handle* h, const te_cluster* c, te_precision p, cudaStream_t s, int64_t cluster = 0) {
  te_status st = host_check(h, c, p);
  if (st != TE_OK) return st;
  const cudaError_t e = launch_check_inputs(c, cluster, h->d_err, h->num_sms, s);
  ++h->n_launches;
  if (e != cudaSuccess) return fail(TE_ECUDA, "input check launch: %s", cudaGetErrorString(e));
  return TE_OK;
}

// ---------------------------------------------------------------------------
// FP64 path
// ---------------------------------------------------------------------------

struct Fp64Plan {
  int nslots;
  int64_t nbt;
  size_t bytes;
};

static int fp64_slots(const Handle* h, int64_t v, int64_t ntri) {
  const int64_t tiles = ((v * v + 63) / 64) * ((v + 63) / 64) * 3;
  int64_t want = (8LL * std::max(1, h->num_sms) + tiles - 1) / tiles;
  const int64_t mem_cap = std::max<int64_t>(1, (int64_t)(1536LL << 20) / (24 * v * v * v));
  want = std::min<int64_t>({want, mem_cap, 4096, std::max<int64_t>(1, ntri)});
  return (int)std::max<int64_t>(1, want);
}

static size_t fp64_carve(Carver& cv, int64_t o, int64_t v, int nslots, int64_t nbt, int64_t ntri,
                         Prepared* P, double** gbuf, double** partials, double** etri) {
  P->t2L = cv.take<double>(o * v * v * o);
  P->nooT = cv.take<double>(o * o * v * o);
  P->ovs = cv.take<double>(o * v * o * v);
  P->ovs32 = nullptr;
  P->t1_32 = nullptr;
  *gbuf = cv.take<double>((size_t)nslots * 3 * v * v * v);
  *partials = cv.take<double>((size_t)nslots * nbt);
  *etri = cv.take<double>((size_t)std::max<int64_t>(1, ntri));
  return cv.off;
}

static te_status run_fp64(Handle* h, const te_cluster* c, int64_t t_begin, int64_t t_end,
                          double* e_tri_out, double* e_total_out, cudaStream_t s) {
  const int64_t o = c->nocc, v = c->nvir;
  const int64_t ntri_all = num_unique_triples(o);
  const int64_t nt = t_end - t_begin;
  const int nslots = fp64_slots(h, v, nt);
  const int64_t nbt = energy_num_block_triples(v);
  Prepared P{};
  double *gbuf, *partials, *etri;
  Carver probe(nullptr);
  const size_t bytes = fp64_carve(probe, o, v, nslots, nbt, ntri_all, &P, &gbuf, &partials, &etri);
  te_status st = ensure_workspace(h, bytes);
  if (st != TE_OK) return st;
  st = ensure_triples(h, (int)o);
  if (st != TE_OK) return st;
  Carver cv(h->ws);
  fp64_carve(cv, o, v, nslots, nbt, ntri_all, &P, &gbuf, &partials, &etri);
  P.o = (int)o;
  P.v = (int)v;
  P.eps_o = c->eps_o;
  P.eps_v = c->eps_v;
  P.ovvv = c->ovvv;
  P.t2 = c->t2;
  P.t1 = c->t1;
  cudaError_t e = launch_prep_fp64(c, &P, s);
  h->n_launches += 3;
  if (e != cudaSuccess) return fail(TE_ECUDA, "prep launch: %s", cudaGetErrorString(e));
  double* out = e_tri_out ? e_tri_out : etri;
  for (int64_t t0 = t_begin; t0 < t_end; t0 += nslots) {
    const int ns = (int)std::min<int64_t>(nslots, t_end - t0);
    size_t pm = prof_begin(h, 0, s);
    e = launch_gemm_fp64(&P, h->d_triples, t0, ns, gbuf, s);
    prof_end(h, pm, s);
    h->gemm_flops += 2.0 * 3.0 * ns * (double)v * v * v * (2.0 * v + 2.0 * o);
    if (e == cudaSuccess) {
      pm = prof_begin(h, 1, s);
      e = launch_energy_f64(&P, h->d_triples, t0, ns, gbuf, partials, nbt, s);
      prof_end(h, pm, s);
    }
    if (e == cudaSuccess)
      e = launch_reduce_triples(partials, nbt, h->d_triples, t0, ns, out + (t0 - t_begin), s);
    h->n_launches += 3;
    if (e != cudaSuccess) return fail(TE_ECUDA, "fp64 launch: %s", cudaGetErrorString(e));
  }
  if (e_total_out) {
    ++h->n_launches;
    e = launch_reduce_total(out, nt, e_total_out, s);
    if (e != cudaSuccess) return fail(TE_ECUDA, "reduction launch: %s", cudaGetErrorString(e));
  }
  return TE_OK;
}

size_t prof_begin(Handle* h, int kind, cudaStream_t s) {
  if (kind == 0) ++h->n_gemm;
  else ++h->n_energy;
  if (!h->profiling || h->capturing) return SIZE_MAX;
  while (h->ev_pool.size() < h->ev_used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return SIZE_MAX;
    }
    h->ev_pool.push_back(e);
  }
  const size_t i = h->ev_used;
  h->ev_used += 2;
  cudaEventRecord(h->ev_pool[i], s);
  h->ev_marks.emplace_back(kind, i);
  return i;
}

void prof_end(Handle* h, size_t start, cudaStream_t s) {
  if (start != SIZE_MAX) cudaEventRecord(h->ev_pool[start + 1], s);
}

std::string tune_header(const Handle* h) {
  char buf[96];
  std::snprintf(buf, sizeof buf, "tenergy-autotune 1 sms=%d cc=%d.%d", h->num_sms, h->cc_major, h->cc_minor);
  return buf;
}

// Entries of a file written for another kind of GPU, and malformed lines, are
// skipped; the tuner checks each entry against its candidates before use.
static void tune_load(Handle* h) {
  FILE* f = std::fopen(h->tune_path.c_str(), "r");
  if (!f) return;
  char line[256];
  if (std::fgets(line, sizeof line, f)) {
    std::string first(line);
    while (!first.empty() && (first.back() == '\n' || first.back() == '\r')) first.pop_back();
    if (first == tune_header(h)) {
      while (std::fgets(line, sizeof line, f)) {
        int o, v, mode, tb, nnt;
        char extra;
        if (std::sscanf(line, "%d %d %d %d %d %c", &o, &v, &mode, &tb, &nnt, &extra) == 5)
          h->tune_file[std::make_tuple(o, v, mode)] = std::make_pair(tb, nnt);
      }
    }
  }
  std::fclose(f);
}

void tune_save(Handle* h) {
  if (h->tune_path.empty()) return;
  auto all = h->tune_file;
  for (const auto& kv : h->tuned) all[kv.first] = kv.second;
  const std::string tmp = h->tune_path + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  bool ok = std::fprintf(f, "%s\n", tune_header(h).c_str()) > 0;
  for (const auto& kv : all)
    ok = ok && std::fprintf(f, "%d %d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first),
                            std::get<2>(kv.first), kv.second.first, kv.second.second) > 0;
  ok = (std::fclose(f) == 0) && ok;
  if (!ok || std::rename(tmp.c_str(), h->tune_path.c_str()) != 0) std::remove(tmp.c_str());
}

te_status ensure_workspace_public(Handle* h, size_t bytes) { return ensure_workspace(h, bytes); }
te_status ensure_triples_public(Handle* h, int nocc) { return ensure_triples(h, nocc); }

// The descriptor and factors of t_energy_df; then the device value checks
// (Bov and Bvv instead of ovvv).
static te_status validate_df(Handle* h, const te_cluster* c, const te_df* df, te_precision p, cudaStream_t s) {
  te_status st = host_check(h, c, p, false);
  if (st != TE_OK) return st;
  if (!df) return fail(TE_EINVAL, "null density-fitting factor descriptor");
  if (df->naux < 1 || df->naux > (1LL << 20))
    return fail(TE_EINVAL, "naux must be in [1, 2^20] (got %lld)", (long long)df->naux);
  if (!df->Bov || !df->Bvv) return fail(TE_EINVAL, "null density-fitting factor pointer");
  if (p == TE_FP64)
    return fail(TE_EUNSUPPORTED, "ovvv from density-fitting factors needs a tensor-core mode (TE_OZAKI, "
                                 "TE_BF16X3, TE_TF32X3 or TE_TF32)");
  if (c->nvir > 2047) return fail(TE_EUNSUPPORTED, "ovvv from density-fitting factors needs nvir <= 2047");
  const cudaError_t e = launch_check_inputs(c, 0, h->d_err, h->num_sms, s, df);
  ++h->n_launches;
  if (e != cudaSuccess) return fail(TE_ECUDA, "input check launch: %s", cudaGetErrorString(e));
  return TE_OK;
}

static te_status run_any(Handle* h, const te_cluster* c, te_precision p, int64_t t_begin,
                         int64_t t_end, double* e_tri_out, double* e_total_out, cudaStream_t s) {
  if (p == TE_FP64) return run_fp64(h, c, t_begin, t_end, e_tri_out, e_total_out, s);
  return run_tc(h, c, p, t_begin, t_end, e_tri_out, e_total_out, s);
}

}  // namespace te

using namespace te;

extern "C" {

te_status te_create(te_handle* out, int device, const char* autotune_cache_path) {
  if (!out) return fail(TE_EINVAL, "null handle pointer");
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return fail(TE_ECUDA, "no CUDA device available");
  }
  if (device < 0 || device >= ndev) return fail(TE_EINVAL, "device %d out of range [0,%d)", device, ndev);
  DeviceGuard g(device);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess)
    return fail(TE_ECUDA, "cudaGetDeviceProperties failed");
  Handle* h = new Handle();
  h->device = device;
  h->num_sms = prop.multiProcessorCount;
  h->smem_optin = prop.sharedMemPerBlockOptin;
  h->cc_major = prop.major;
  h->cc_minor = prop.minor;
  if (cudaMalloc(&h->d_err, sizeof(unsigned int) * 4) != cudaSuccess ||
      cudaMemset(h->d_err, 0, sizeof(unsigned int) * 4) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(TE_ENOMEM, "error-word allocation failed");
  }
  const char* lg = std::getenv("TE_LOG");
  h->log = lg && *lg && std::strcmp(lg, "0") != 0;
  if (autotune_cache_path && *autotune_cache_path) {
    h->tune_path = autotune_cache_path;
    tune_load(h);
  }
  *out = reinterpret_cast<te_handle>(h);
  return TE_OK;
}

te_status te_destroy(te_handle hh) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return TE_OK;
  DeviceGuard g(h->device);
  cudaDeviceSynchronize();
  if (h->ws) cudaFree(h->ws);
  if (h->d_triples) cudaFree(h->d_triples);
  if (h->d_err) cudaFree(h->d_err);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  drop_graphs(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  destroy_tc_state(h);
  delete h;
  return TE_OK;
}

te_status t_energy_triples(te_handle hh, const te_cluster* c, te_precision p, int64_t t_begin,
                           int64_t t_end, double* e_triples, te_stream_t ss) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(ss);
  if (!h) return fail(TE_EINVAL, "null handle");
  DeviceGuard g(h->device);
  te_status st = validate(h, c, p, s);
  if (st != TE_OK) return st;
  const int64_t nt = num_unique_triples(c->nocc);
  if (t_begin < 0 || t_end > nt || t_begin > t_end)
    return fail(TE_EINVAL, "triple range [%lld,%lld) outside [0,%lld)", (long long)t_begin,
                (long long)t_end, (long long)nt);
  if (t_begin == t_end) return TE_OK;
  if (!e_triples) return fail(TE_EINVAL, "null e_triples");
  return run_any(h, c, p, t_begin, t_end, e_triples, nullptr, s);
}

te_status t_energy(te_handle hh, const te_cluster* c, te_precision p, double* e_out, te_stream_t ss) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(ss);
  if (!h) return fail(TE_EINVAL, "null handle");
  if (!e_out) return fail(TE_EINVAL, "null e_out");
  DeviceGuard g(h->device);
  te_status st = validate(h, c, p, s);
  if (st != TE_OK) return st;
  const int64_t nt = num_unique_triples(c->nocc);
  if (nt == 0) {
    if (cudaMemsetAsync(e_out, 0, sizeof(double), s) != cudaSuccess)
      return fail(TE_ECUDA, "memset failed");
    return TE_OK;
  }
  return run_any(h, c, p, 0, nt, nullptr, e_out, s);
}

te_status t_energy_df(te_handle hh, const te_cluster* c, const te_df* df, te_precision p, double* e_out,
                      te_stream_t ss) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(ss);
  if (!h) return fail(TE_EINVAL, "null handle");
  if (!e_out) return fail(TE_EINVAL, "null e_out");
  DeviceGuard g(h->device);
  te_status st = validate_df(h, c, df, p, s);
  if (st != TE_OK) return st;
  const int64_t nt = num_unique_triples(c->nocc);
  if (nt == 0) {
    if (cudaMemsetAsync(e_out, 0, sizeof(double), s) != cudaSuccess) return fail(TE_ECUDA, "memset failed");
    return TE_OK;
  }
  return run_tc(h, c, p, 0, nt, nullptr, e_out, s, df);
}

te_status t_energy_df_triples(te_handle hh, const te_cluster* c, const te_df* df, te_precision p, int64_t t_begin,
                              int64_t t_end, double* e_triples, te_stream_t ss) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(ss);
  if (!h) return fail(TE_EINVAL, "null handle");
  DeviceGuard g(h->device);
  te_status st = validate_df(h, c, df, p, s);
  if (st != TE_OK) return st;
  const int64_t nt = num_unique_triples(c->nocc);
  if (t_begin < 0 || t_end > nt || t_begin > t_end)
    return fail(TE_EINVAL, "triple range [%lld,%lld) outside [0,%lld)", (long long)t_begin, (long long)t_end,
                (long long)nt);
  if (t_begin == t_end) return TE_OK;
  if (!e_triples) return fail(TE_EINVAL, "null e_triples");
  return run_tc(h, c, p, t_begin, t_end, e_triples, nullptr, s, df);
}

te_status te_df_workspace_bytes(te_handle hh, const te_cluster* c, const te_df* df, te_precision p,
                                size_t* bytes) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !c || !df || !bytes) return fail(TE_EINVAL, "null argument");
  if (c->nocc < 1 || c->nvir < 1 || df->naux < 1) return fail(TE_EINVAL, "nocc, nvir and naux must be >= 1");
  if (p == TE_FP64) return fail(TE_EUNSUPPORTED, "ovvv from density-fitting factors needs a tensor-core mode");
  return tc_workspace_bytes(h, c, p, bytes, df);
}

te_status t_energy_batched(te_handle hh, const te_cluster* cs, int64_t n, te_precision p,
                           double* e_out, te_stream_t ss) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(ss);
  if (!h) return fail(TE_EINVAL, "null handle");
  if (n < 0) return fail(TE_EINVAL, "negative batch size");
  if (n == 0) return TE_OK;
  if (!cs || !e_out) return fail(TE_EINVAL, "null cluster array or e_out");
  DeviceGuard g(h->device);
  for (int64_t x = 0; x < n; ++x) {
    te_status st = host_check(h, cs + x, p);
    if (st != TE_OK) {
      char msg[600];  // the message buffer holds at most 511 characters, plus the prefix
      snprintf(msg, sizeof(msg), "cluster %lld: %.511s", (long long)x, te_last_error());
      return fail(st, "%s", msg);
    }
  }
  // a replay of a captured batch needs no further checks of the descriptors
  for (auto& ge : h->graphs) {
    if (ge.precision != (int)p || ge.e_out != e_out || (int64_t)ge.clusters.size() != n) continue;
    if (std::memcmp(ge.clusters.data(), cs, sizeof(te_cluster) * n) != 0) continue;
    // the graph begins with every member's input check
    if (cudaGraphLaunch(ge.exec, s) != cudaSuccess)
      return fail(TE_ECUDA, "graph launch: %s", cudaGetErrorString(cudaGetLastError()));
    h->n_launches += ge.launches;
    return TE_OK;
  }
  te_status st = TE_OK;
  int64_t maxo = 1;
  for (int64_t x = 0; x < n; ++x) maxo = std::max<int64_t>(maxo, cs[x].nocc);
  st = ensure_triples(h, (int)maxo);
  if (st != TE_OK) return st;
  if (p != TE_FP64) {  // tile shapes tuned per (nocc, nvir) before the capture
    for (int64_t x = 0; x < n; ++x) {
      st = tc_autotune(h, cs + x, p, s);
      if (st != TE_OK) return st;
    }
  }
  // one workspace for the whole batch: float64 runs the members one after
  // another; the tensor-core modes hold every member's operands and one G pool
  size_t need = 0;
  if (p == TE_FP64) {
    for (int64_t x = 0; x < n; ++x) {
      size_t b = 0;
      st = te_workspace_bytes(hh, cs + x, p, &b);
      if (st != TE_OK) return st;
      need = std::max(need, b);
    }
  } else {
    st = tc_batched_bytes(h, cs, n, p, &need);
    if (st != TE_OK) return st;
  }
  st = ensure_workspace(h, need);
  if (st != TE_OK) return st;
  // capture the batch's launches into one CUDA graph on an internal stream
  if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(TE_ECUDA, "stream creation failed");
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(TE_ECUDA, "stream synchronise failed");
  if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return fail(TE_ECUDA, "begin capture: %s", cudaGetErrorString(cudaGetLastError()));
  h->capturing = true;
  const int64_t l0 = h->n_launches;
  for (int64_t x = 0; x < n && st == TE_OK; ++x) st = validate(h, cs + x, p, h->cap_stream, x);
  if (st == TE_OK && p != TE_FP64) st = run_tc_batched(h, cs, n, p, e_out, h->cap_stream);
  for (int64_t x = 0; x < n && st == TE_OK && p == TE_FP64; ++x) {
    const int64_t nt = num_unique_triples(cs[x].nocc);
    if (nt == 0) {
      if (cudaMemsetAsync(e_out + x, 0, sizeof(double), h->cap_stream) != cudaSuccess)
        st = fail(TE_ECUDA, "memset failed");
      ++h->n_launches;
    } else {
      st = run_any(h, cs + x, p, 0, nt, nullptr, e_out + x, h->cap_stream);
    }
  }
  h->capturing = false;
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(h->cap_stream, &graph);
  if (st != TE_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (ec != cudaSuccess || !graph) return fail(TE_ECUDA, "end capture: %s", cudaGetErrorString(ec));
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) return fail(TE_ECUDA, "graph instantiate: %s", cudaGetErrorString(ei));
  if (h->graphs.size() >= 4) {
    cudaGraphExecDestroy(h->graphs.front().exec);
    h->graphs.erase(h->graphs.begin());
  }
  Handle::GraphEntry ge;
  ge.clusters.assign(cs, cs + n);
  ge.precision = (int)p;
  ge.e_out = e_out;
  ge.exec = exec;
  ge.launches = h->n_launches - l0;
  h->graphs.push_back(ge);
  if (cudaGraphLaunch(exec, s) != cudaSuccess)
    return fail(TE_ECUDA, "graph launch: %s", cudaGetErrorString(cudaGetLastError()));
  return TE_OK;
}

// The adjoint over the canonical triples [t_begin, t_end) of one cluster.
static te_status vjp_range(Handle* h, const te_cluster* c, te_precision p, int64_t t_begin, int64_t t_end,
                           double gE, double* e_out, te_cluster_grad* gr, cudaStream_t s, int64_t cluster) {
  if (!gr) return fail(TE_EINVAL, "null gradient descriptor");
  if (!(gE == gE) || gE > 1e300 || gE < -1e300) return fail(TE_EINVAL, "non-finite gE");
  if (h->capturing) return fail(TE_EINVAL, "the adjoint cannot run inside the library's graph capture");
  te_status st = validate(h, c, p, s, cluster);
  if (st != TE_OK) return st;
  const int64_t nt = num_unique_triples(c->nocc);
  if (t_begin < 0 || t_end > nt || t_begin > t_end)
    return fail(TE_EINVAL, "triple range [%lld,%lld) outside [0,%lld)", (long long)t_begin, (long long)t_end,
                (long long)nt);
  // float64: DFMA contractions; the tensor-core modes: exact-slice contractions
  if (p == TE_FP64) return run_vjp_fp64(h, c, t_begin, t_end, gE, e_out, gr, s);
  if (h->cc_major != 10 && h->cc_major != 11)
    return fail(TE_EUNSUPPORTED, "the tensor-core adjoint needs an sm_100-family GPU");
  return run_vjp_tc(h, c, t_begin, t_end, gE, e_out, gr, s);
}

te_status t_energy_vjp(te_handle hh, const te_cluster* c, te_precision p, double gE, double* e_out,
                       te_cluster_grad* gr, te_stream_t ss) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return fail(TE_EINVAL, "null handle");
  if (!c) return fail(TE_EINVAL, "null cluster descriptor");
  DeviceGuard g(h->device);
  const int64_t nt = c->nocc >= 1 ? num_unique_triples(c->nocc) : 0;
  return vjp_range(h, c, p, 0, nt, gE, e_out, gr, reinterpret_cast<cudaStream_t>(ss), 0);
}

te_status t_energy_vjp_triples(te_handle hh, const te_cluster* c, te_precision p, int64_t t_begin,
                               int64_t t_end, double gE, double* e_out, te_cluster_grad* gr, te_stream_t ss) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return fail(TE_EINVAL, "null handle");
  DeviceGuard g(h->device);
  return vjp_range(h, c, p, t_begin, t_end, gE, e_out, gr, reinterpret_cast<cudaStream_t>(ss), 0);
}

te_status t_energy_vjp_batched(te_handle hh, const te_cluster* cs, int64_t n, te_precision p, const double* gE,
                               double* e_out, te_cluster_grad* grads, te_stream_t ss) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return fail(TE_EINVAL, "null handle");
  if (n < 0) return fail(TE_EINVAL, "negative batch size");
  if (n == 0) return TE_OK;
  if (!cs || !grads) return fail(TE_EINVAL, "null cluster or gradient array");
  DeviceGuard g(h->device);
  for (int64_t x = 0; x < n; ++x) {  // every descriptor before any launch
    te_status st = host_check(h, cs + x, p);
    if (st == TE_OK && gE && !(gE[x] == gE[x] && gE[x] < 1e300 && gE[x] > -1e300))
      st = fail(TE_EINVAL, "non-finite gE");
    if (st != TE_OK) {
      char msg[600];
      snprintf(msg, sizeof(msg), "cluster %lld: %.511s", (long long)x, te_last_error());
      return fail(st, "%s", msg);
    }
  }
  // the workspace of the largest member, once
  size_t need = 0;
  int64_t maxo = 1;
  for (int64_t x = 0; x < n; ++x) {
    need = std::max(need, p == TE_FP64 ? vjp_fp64_bytes(cs[x].nocc, cs[x].nvir)
                                       : vjp_tc_bytes(cs[x].nocc, cs[x].nvir, h->num_sms));
    maxo = std::max<int64_t>(maxo, cs[x].nocc);
  }
  te_status st = ensure_workspace(h, need);
  if (st == TE_OK) st = ensure_triples(h, (int)maxo);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(ss);
  for (int64_t x = 0; x < n && st == TE_OK; ++x) {
    const int64_t nt = num_unique_triples(cs[x].nocc);
    st = vjp_range(h, cs + x, p, 0, nt, gE ? gE[x] : 1.0, e_out ? e_out + x : nullptr, grads + x, s, x);
    if (st != TE_OK) {
      char msg[600];
      snprintf(msg, sizeof(msg), "cluster %lld: %.511s", (long long)x, te_last_error());
      return fail(st, "%s", msg);
    }
  }
  return st;
}

te_status t_energy_frag(te_handle hh, const te_cluster* c, const double* cf, te_precision p, double* e_out,
                        double* e_triples, te_stream_t ss) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(ss);
  if (!h) return fail(TE_EINVAL, "null handle");
  if (!cf) return fail(TE_EINVAL, "null projector");
  if (!e_out && !e_triples) return fail(TE_EINVAL, "no output");
  if (p != TE_FP64 && p != TE_OZAKI)
    return fail(TE_EUNSUPPORTED, "the projected energy runs in TE_FP64 or TE_OZAKI (got %d)", (int)p);
  if (h->capturing) return fail(TE_EINVAL, "t_energy_frag cannot run inside a graph capture");
  DeviceGuard g(h->device);
  te_status st = validate(h, c, p, s);
  if (st != TE_OK) return st;
  if (p == TE_OZAKI && h->cc_major != 10 && h->cc_major != 11)
    return fail(TE_EUNSUPPORTED, "exact-slice contractions need an sm_100-family GPU");
  return run_frag(h, c, cf, p, e_out, e_triples, s);
}

te_status te_sync(te_handle hh, te_stream_t ss) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return fail(TE_EINVAL, "null handle");
  DeviceGuard g(h->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(ss);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(TE_ECUDA, "stream synchronise: %s", cudaGetErrorString(e));
  unsigned int err[4] = {0, 0, 0, 0};
  if (cudaMemcpy(err, h->d_err, sizeof(err), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(TE_ECUDA, "error word read failed");
  if (err[0] != 0) {
    cudaMemset(h->d_err, 0, sizeof(err));
    if (err[0] & ERR_WAIT_TIMEOUT)
      return fail(TE_ETIMEOUT, "device wait expired (code %u, site %u, block %u)", err[0], err[1], err[2]);
    if (err[0] & ERR_BAD_INPUT) {
      static const char* what[11] = {"?", "eps_o", "eps_v", "ovvv", "ooov", "ovov", "t1", "t2", "", "Bov", "Bvv"};
      if (err[1] == 8)
        return fail(TE_EINVAL, "input check failed (cluster %u): max(eps_o) must be below min(eps_v)", err[2]);
      return fail(TE_EINVAL, "input check failed (cluster %u): non-finite value in %s", err[2],
                  what[(err[1] < 11 && err[1] != 8) ? err[1] : 0]);
    }
    return fail(TE_ECUDA, "device check failed (code %u, site %u, block %u)", err[0], err[1], err[2]);
  }
  return TE_OK;
}

te_status te_workspace_bytes(te_handle hh, const te_cluster* c, te_precision p, size_t* bytes) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !c || !bytes) return fail(TE_EINVAL, "null argument");
  if (c->nocc < 1 || c->nvir < 1) return fail(TE_EINVAL, "nocc and nvir must be >= 1");
  const int64_t o = c->nocc, v = c->nvir;
  const int64_t nt = num_unique_triples(o);
  if (p == TE_FP64) {
    Prepared P{};
    double *a, *b, *d;
    Carver probe(nullptr);
    *bytes = fp64_carve(probe, o, v, fp64_slots(h, v, nt), energy_num_block_triples(v), nt, &P, &a, &b, &d);
    return TE_OK;
  }
  return tc_workspace_bytes(h, c, p, bytes);
}

te_status te_reserve(te_handle hh, const te_cluster* c, te_precision p, int what) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !c) return fail(TE_EINVAL, "null argument");
  if (c->nocc < 1 || c->nvir < 1) return fail(TE_EINVAL, "nocc and nvir must be >= 1");
  if (what < 1 || what > (TE_RESERVE_ENERGY | TE_RESERVE_VJP | TE_RESERVE_FRAG))
    return fail(TE_EINVAL, "what must be a non-empty combination of TE_RESERVE_ENERGY, _VJP, _FRAG");
  if (p < TE_FP64 || p > TE_OZAKI) return fail(TE_EINVAL, "unknown precision %d", (int)p);
  DeviceGuard g(h->device);
  size_t need = 0;
  if (what & TE_RESERVE_ENERGY) {
    te_status st = te_workspace_bytes(hh, c, p, &need);
    if (st != TE_OK) return st;
  }
  if (what & TE_RESERVE_VJP)
    need = std::max(need, p == TE_FP64 ? vjp_fp64_bytes(c->nocc, c->nvir) : vjp_tc_bytes(c->nocc, c->nvir, h->num_sms));
  if (what & TE_RESERVE_FRAG) need = std::max(need, frag_bytes(c->nocc, c->nvir, p, h->num_sms));
  te_status st = ensure_workspace(h, need);
  if (st != TE_OK) return st;
  return ensure_triples(h, (int)c->nocc);
}

const char* te_last_error(void) { return g_last_error; }

te_status te_profile_enable(te_handle hh, int on) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return fail(TE_EINVAL, "null handle");
  h->profiling = on != 0;
  return TE_OK;
}

te_status te_profile_read(te_handle hh, te_profile* out, int reset) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !out) return fail(TE_EINVAL, "null argument");
  DeviceGuard g(h->device);
  if (cudaDeviceSynchronize() != cudaSuccess)
    return fail(TE_ECUDA, "synchronise: %s", cudaGetErrorString(cudaGetLastError()));
  double ms[2] = {0.0, 0.0};
  for (const auto& m : h->ev_marks) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, h->ev_pool[m.second], h->ev_pool[m.second + 1]) == cudaSuccess)
      ms[m.first] += t;
    else
      cudaGetLastError();
  }
  out->launches = h->n_launches;
  out->gemm_launches = h->n_gemm;
  out->gemm_ms = ms[0];
  out->energy_launches = h->n_energy;
  out->energy_ms = ms[1];
  out->gemm_flops = h->gemm_flops;
  if (reset) {
    h->n_launches = h->n_gemm = h->n_energy = 0;
    h->gemm_flops = 0.0;
    h->ev_used = 0;
    h->ev_marks.clear();
  }
  return TE_OK;
}

te_status te_set_ozaki_bits(te_handle hh, int bits) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return fail(TE_EINVAL, "null handle");
  if (bits != 0 && bits != 6 && bits != 7) return fail(TE_EINVAL, "slice width must be 0, 6 or 7 (got %d)", bits);
  if (bits != h->ozaki_bits) {
    DeviceGuard g(h->device);
    drop_graphs(h);  // captured batches bake in the slice width
    h->ozaki_bits = bits;
  }
  return TE_OK;
}

te_status te_set_workspace_limit(te_handle hh, size_t bytes) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return fail(TE_EINVAL, "null handle");
  if (bytes && h->ws_bytes > bytes)
    return fail(TE_EINVAL, "the handle already holds %zu bytes of workspace, above %zu", h->ws_bytes, bytes);
  h->ws_limit = bytes;
  return TE_OK;
}

te_status te_set_wait_limit_ns(te_handle hh, uint64_t ns) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return fail(TE_EINVAL, "null handle");
  h->wait_limit_ns = ns ? ns : 4000000000ull;
  return TE_OK;
}

}  // extern "C"
