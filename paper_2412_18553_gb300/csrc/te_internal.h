// Internal declarations shared by the host-side translation units of
// libtenergy.  Nothing here is part of the C ABI (include/tenergy.h).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/tenergy.h"

namespace te {

// Device error word bits (written by kernels, read by te_sync).
enum : unsigned int {
  ERR_WAIT_TIMEOUT = 1u,   // a bounded mbarrier/flag wait expired
  ERR_BAD_TILE = 2u,       // a tile coordinate check failed (skipped access)
  ERR_BAD_INPUT = 4u,      // an input value check failed (non-finite, eps ordering)
};

// Device-side input value checks of one cluster (checks.cu): every entry
// finite and max(eps_o) < min(eps_v); a violation sets ERR_BAD_INPUT with the
// site (1..7 the array, 8 the eps ordering, 9 and 10 the density-fitting
// factors) and `cluster` in the error word.  With df, ovvv is not checked
// (not read) and Bov, Bvv are.
cudaError_t launch_check_inputs(const te_cluster* c, int64_t cluster, unsigned int* err, int num_sms,
                                cudaStream_t s, const te_df* df = nullptr);
// The same for the MP2 step's inputs (eps_o, eps_v, and the DF factor's ov
// block of nB entries, site 9).
cudaError_t launch_check_mp2(const double* eps_o, int64_t o, const double* eps_v, int64_t v, const double* Bov,
                             int64_t nB, int64_t cluster, unsigned int* err, int num_sms, cudaStream_t s);

// One occupied triple of the canonical unique list.
struct Triple {
  int i, j, k, m;  // i >= j >= k, m = number of distinct orderings (3 or 6)
};

// A view of the prepared operands of one cluster, as the kernels see them.
struct Prepared {
  int o, v;
  // float64 originals (caller-owned)
  const double* eps_o;
  const double* eps_v;
  const double* ovvv;
  const double* t2;
  const double* t1;
  // float64 prepared copies (handle workspace)
  double* t2L;   // [o][v][v][o]  t2L[q][a][b][l] = t2[l,q,a,b]
  double* nooT;  // [o][o][v][o]  nooT[p][r][g][l] = -ooov[p,l,r,g]
  double* ovs;   // [o][v][o][v]  1/2 (ovov[i,a,j,b] + ovov[j,b,i,a])
  float* ovs32;  // same, float32 (mixed modes)
  float* t1_32;  // t1 as float32 (mixed modes)
};

struct Handle {
  int device = 0;
  int num_sms = 0;
  int cc_major = 0, cc_minor = 0;
  size_t smem_optin = 0;
  uint64_t wait_limit_ns = 4000000000ull;
  int ozaki_bits = 0;                // exact-slice width: 0 automatic, 6 or 7
  unsigned int* d_err = nullptr;     // device error word
  // workspace (grows, never shrinks until destroy)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  size_t ws_limit = 0;  // most workspace bytes the handle may hold (0: no limit)
  bool log = false;     // TE_LOG=1: tile plans and autotune decisions on stderr
  // triple table cache
  Triple* d_triples = nullptr;
  int triples_nocc = -1;
  size_t triples_cap = 0;
  void* tc = nullptr;  // tensor-core path state (tensor maps cache), owned
  // launch accounting / profiling
  int64_t n_launches = 0, n_gemm = 0, n_energy = 0;
  double gemm_flops = 0.0;
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, size_t>> ev_marks;  // (kind 0 gemm / 1 energy, start event index)
  bool capturing = false;                         // inside a CUDA graph capture (no profiling events)
  // CUDA graphs of whole batches, keyed by the batch signature
  struct GraphEntry {
    std::vector<te_cluster> clusters;
    int precision;
    double* e_out;
    cudaGraphExec_t exec;
    int64_t launches;
  };
  std::vector<GraphEntry> graphs;
  cudaStream_t cap_stream = nullptr;
  // autotuned tile shapes: (nocc, nvir, mode) -> (TB, n_nt)
  std::map<std::tuple<int, int, int>, std::pair<int, int>> tuned;
  // the autotune cache file and the entries read from it (checked against the
  // tuner's candidates before use)
  std::string tune_path;
  std::map<std::tuple<int, int, int>, std::pair<int, int>> tune_file;
};

void drop_graphs(Handle* h);

// autotune cache file: first line of the format for this handle's GPU; write
// the file from tune_file and tuned (no-op without a path)
std::string tune_header(const Handle* h);
void tune_save(Handle* h);

// Profiling helpers: begin/end a timed launch of `kind` on stream s.
size_t prof_begin(Handle* h, int kind, cudaStream_t s);
void prof_end(Handle* h, size_t start, cudaStream_t s);

// thread-local last error message
void set_error(const char* fmt, ...);
te_status fail(te_status st, const char* fmt, ...);

// enumerate canonical unique triples
std::vector<Triple> unique_triples(int nocc);
int64_t num_unique_triples(int64_t nocc);

// launch wrappers (defined in the .cu files)
cudaError_t launch_prep_fp64(const te_cluster* c, Prepared* P, cudaStream_t s);
cudaError_t launch_gemm_fp64(const Prepared* P, const Triple* d_triples, int64_t t0,
                             int nslots, double* gbuf, cudaStream_t s);

// energy over G buffers: T = float (mixed) or double (fp64)
cudaError_t launch_energy_f64(const Prepared* P, const Triple* d_triples, int64_t t0,
                              int nslots, const double* gbuf, double* partials,
                              int64_t nbt, cudaStream_t s);
cudaError_t launch_energy_f32(const Prepared* P, const Triple* d_triples, int64_t t0,
                              int nslots, const float* gbuf, int ldz, double* partials,
                              int64_t nbt, cudaStream_t s);
// writes e_out[slot] = (m/3) * sum of the slot's partials, for triples t0 .. t0+nslots-1
cudaError_t launch_reduce_triples(const double* partials, int64_t nbt, const Triple* d_triples,
                                  int64_t t0, int nslots, double* e_out, cudaStream_t s);
cudaError_t launch_reduce_total(const double* e_triples, int64_t n, double* e_out,
                                cudaStream_t s);

// adjoint of E(T) in float64 (vjp.cu)
// over the canonical triples [t_begin, t_end): the gradient of the sum of their shares
te_status run_vjp_fp64(Handle* h, const te_cluster* c, int64_t t_begin, int64_t t_end, double gE,
                       double* e_out, te_cluster_grad* g, cudaStream_t s);
// fragment-projected E(T) (vjp.cu): cf device [nocc][nocc]; precision TE_FP64 or
// exact slices; per-triple shares to e_triples (nullable), total to e_out (nullable)
size_t frag_bytes(int64_t o, int64_t v, te_precision p, int num_sms);
te_status run_frag(Handle* h, const te_cluster* c, const double* cf, te_precision p, double* e_out,
                   double* e_triples, cudaStream_t s);
// workspace bytes of the two adjoints (vjp.cu)
size_t vjp_fp64_bytes(int64_t o, int64_t v);
size_t vjp_tc_bytes(int64_t o, int64_t v, int num_sms);
// the same with the contractions on the tensor cores in exact BF16 slices (vjp.cu)
te_status run_vjp_tc(Handle* h, const te_cluster* c, int64_t t_begin, int64_t t_end, double gE,
                     double* e_out, te_cluster_grad* g, cudaStream_t s);

constexpr int ENERGY_TB = 8;  // virtual block edge of the energy kernel
inline int64_t energy_num_blocks(int64_t v) { return (v + ENERGY_TB - 1) / ENERGY_TB; }
inline int64_t energy_num_block_triples(int64_t v) {
  int64_t nb = energy_num_blocks(v);
  return nb * (nb + 1) * (nb + 2) / 6;
}

}  // namespace te
