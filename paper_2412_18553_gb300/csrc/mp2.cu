// The MP2 step that precedes (T) in the SIE workflow, for a batch of clusters
// (supplement section on bath-natural-orbital construction):
//
//   (ia|jb)   = sum_P B[P,i,a] B[P,j,b]                       (density fitting)
//   t_ij^ab   = -(ia|jb) / D_ij^ab,  D_ij^ab = e_a + e_b - e_i - e_j
//   gamma_ab  = 2 sum_ij sum_c t_ij^ac (2 t_ij^bc - t_ij^cb)
//   gamma_ij  = 2 delta_ij - 2 sum_k sum_ab t_ik^ab (2 t_jk^ab - t_jk^ba)
//   populations: the eigenvalues of gamma_oo and gamma_vv (BNO populations)
//
// The three contractions are GEMMs over two-index views (strided.h).  The
// (ia|jb) contraction runs in float64 on the DFMA units or, in the exact-slice
// mode, in exact BF16 slices on the tensor cores (Bov scaled by one power of
// two and cut into four 7-bit slices; K blocks of at most 1024 keep the
// level-0/1 sums exact).  The density contractions run in float64 in both
// modes: their K spans the amplitudes' whole dynamic range (o^2 v and o v^2
// terms), which one scale per array would resolve only to ~1e-6 of the
// largest entry; they cost o/naux and o/v of the first.  With T~ = 2t - t^(ab
// swapped), both density blocks are single contractions against T~:
//   gamma_vv[a,b] = 2 sum_{(ij),c} t[ij,a,c] T~[ij,b,c]
//   gamma_oo[i,j] = 2 delta_ij - 2 sum_{k,(ab)} t[i,k,ab] T~[j,k,ab]
// The eigenvalues come from the cyclic Jacobi method in the parallel
// (round-robin) ordering, one block per matrix, float64 throughout, with the
// matrix in shared memory up to order 168; one launch takes the matrices of
// up to 32 clusters, whose density blocks stay in the workspace until then.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "strided.h"
#include "te_internal.h"

namespace te {

te_status ensure_workspace_public(Handle* h, size_t bytes);

namespace {

static int grid_of(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>(1, (n + 255) / 256), 8192); }

// t[i,j,a,b] = -ovov[i,a,j,b] / D, T~[i,j,a,b] = 2 t[i,j,a,b] - t[i,j,b,a]
// (D is symmetric in a, b, so t[i,j,b,a] = -ovov[i,b,j,a] / D)
__global__ void k_mp2_amplitudes(const double* __restrict__ ovov, const double* __restrict__ eps_o,
                                 const double* __restrict__ eps_v, int o, int v, double* __restrict__ t2,
                                 double* __restrict__ tt) {
  const int64_t n = (int64_t)o * o * v * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(idx % v);
    int64_t r = idx / v;
    const int a = (int)(r % v);
    r /= v;
    const int j = (int)(r % o);
    const int i = (int)(r / o);
    const double D = (eps_v[a] + eps_v[b]) - (eps_o[i] + eps_o[j]);
    const double t = -ovov[(((int64_t)i * v + a) * o + j) * v + b] / D;
    const double ts = -ovov[(((int64_t)i * v + b) * o + j) * v + a] / D;
    t2[idx] = t;
    tt[idx] = 2.0 * t - ts;
  }
}

// gamma_oo starts at 2 on the diagonal, 0 elsewhere
__global__ void k_two_identity(double* __restrict__ g, int o) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < o * o; idx += gridDim.x * blockDim.x)
    g[idx] = (idx / o == idx % o) ? 2.0 : 0.0;
}

// One symmetric matrix for the eigensolver: the source (n x n), the output
// eigenvalues (n, ascending), the padded order m (n rounded up to even; the
// padding row and column are zero and never rotate) and a global working copy
// (m x m) for an order too large for shared memory (null otherwise).
struct EigJob {
  double* a;
  const double* src;
  double* out;
  int n, m;
};

// Orders up to this one keep their working copy in shared memory:
// 168^2 doubles plus 84 pairs' rotations fit the 227 KB of one block.
constexpr int kJacobiSmemM = 168;

struct EigJobs {
  int count;
  EigJob j[64];
};

// Shared memory of one job: rotations of its m / 2 pairs, then its working
// copy unless it has a global one.
__host__ __device__ inline size_t jacobi_rot_bytes(int m) { return ((size_t)(m / 2) * 20 + 15) & ~size_t(15); }
__host__ __device__ inline size_t jacobi_smem_bytes(const EigJob& j) {
  return jacobi_rot_bytes(j.m) + (j.a ? 0 : (size_t)j.m * j.m * 8);
}

// Parallel-order cyclic Jacobi: in step s of a sweep the index at position 0
// stays and the others rotate; pair k is (label(k), label(m-1-k)) with
// label(0) = 0, label(x) = 1 + (x - 1 + s) mod (m - 1).  The m/2 rotations of a
// step act on disjoint index pairs, so they are applied at once: rows p, q of
// every pair, then columns p, q.  The matrix taken is the symmetric part of the
// block ((A + A^T) / 2): a density computed in exact slices is symmetric only
// to about 1e-9 of its scale, and an orthogonal similarity cannot remove an
// antisymmetric part.  Sweeps repeat until the off-diagonal mass is below
// 1e-30 of the matrix's, stops decreasing (rounding floor), or 60 sweeps have
// run.  Then the diagonal is sorted.  Dynamic shared memory: the rotations
// (cosines, sines, then the p and q indices, m / 2 each), then the working
// copy when the job has no global one.
__global__ void __launch_bounds__(512, 1) k_jacobi(const __grid_constant__ EigJobs J) {
  const EigJob& jb = J.j[blockIdx.x];
  const int n = jb.n, m = jb.m;
  extern __shared__ __align__(16) unsigned char jac_smem[];
  double* cs = reinterpret_cast<double*>(jac_smem);
  double* sn = cs + m / 2;
  unsigned short* pp = reinterpret_cast<unsigned short*>(sn + m / 2);
  unsigned short* qq = pp + m / 2;
  double* A = jb.a ? jb.a : reinterpret_cast<double*>(jac_smem + jacobi_rot_bytes(m));
  __shared__ double red[32];
  __shared__ int done;
  __shared__ double prev_off;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) prev_off = -1.0;
  for (int64_t e = tid; e < (int64_t)m * m; e += nt) {
    const int r = (int)(e / m), c = (int)(e % m);
    A[e] = (r < n && c < n) ? 0.5 * (jb.src[(int64_t)r * n + c] + jb.src[(int64_t)c * n + r]) : 0.0;
  }
  __syncthreads();
  const int half = m / 2;
  for (int sweep = 0; sweep < 60; ++sweep) {
    // convergence test: off-diagonal and total squared mass
    double off = 0.0, tot = 0.0;
    for (int64_t e = tid; e < (int64_t)m * m; e += nt) {
      const double x = A[e];
      tot += x * x;
      if (e / m != e % m) off += x * x;
    }
    for (int d = 16; d > 0; d >>= 1) {
      off += __shfl_down_sync(0xffffffffu, off, d);
      tot += __shfl_down_sync(0xffffffffu, tot, d);
    }
    if ((tid & 31) == 0) {
      red[tid >> 5] = off;
      if (tid == 0) done = 0;
    }
    __syncthreads();
    if (tid == 0) {
      double so = 0.0;
      for (int w = 0; w < (nt >> 5); ++w) so += red[w];
      red[0] = so;
    }
    __syncthreads();
    const double off_all = red[0];
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = tot;
    __syncthreads();
    if (tid == 0) {
      double st = 0.0;
      for (int w = 0; w < (nt >> 5); ++w) st += red[w];
      done = (off_all <= 1e-30 * st || (prev_off >= 0.0 && off_all >= prev_off)) ? 1 : 0;
      prev_off = off_all;
    }
    __syncthreads();
    if (done) break;
    for (int s = 0; s < m - 1; ++s) {
      for (int k = tid; k < half; k += nt) {
        auto label = [&](int x) { return x == 0 ? 0 : 1 + (x - 1 + s) % (m - 1); };
        const int p = label(k), q = label(m - 1 - k);
        const double apq = A[(int64_t)p * m + q];
        double c = 1.0, t = 0.0;
        if (apq != 0.0) {
          const double theta = (A[(int64_t)q * m + q] - A[(int64_t)p * m + p]) / (2.0 * apq);
          const double at = fabs(theta);
          t = at > 1e150 ? 0.5 / theta : copysign(1.0, theta) / (at + sqrt(at * at + 1.0));
          c = 1.0 / sqrt(t * t + 1.0);
        }
        pp[k] = (unsigned short)p;
        qq[k] = (unsigned short)q;
        cs[k] = c;
        sn[k] = t * c;
      }
      __syncthreads();
      for (int64_t e = tid; e < (int64_t)half * m; e += nt) {  // rows p, q of every pair
        const int k = (int)(e / m), col = (int)(e % m);
        const int64_t rp = (int64_t)pp[k] * m + col, rq = (int64_t)qq[k] * m + col;
        const double ap = A[rp], aq = A[rq], c = cs[k], s_ = sn[k];
        A[rp] = c * ap - s_ * aq;
        A[rq] = s_ * ap + c * aq;
      }
      __syncthreads();
      for (int64_t e = tid; e < (int64_t)half * m; e += nt) {  // columns p, q of every pair
        const int k = (int)(e % half), row = (int)(e / half);
        const int64_t cp = (int64_t)row * m + pp[k], cq = (int64_t)row * m + qq[k];
        const double ap = A[cp], aq = A[cq], c = cs[k], s_ = sn[k];
        A[cp] = c * ap - s_ * aq;
        A[cq] = s_ * ap + c * aq;
      }
      __syncthreads();
    }
  }
  // eigenvalues ascending: each by its rank (ties by index)
  for (int i = tid; i < n; i += nt) {
    const double di = A[(int64_t)i * m + i];
    int rank = 0;
    for (int j2 = 0; j2 < n; ++j2) {
      const double dj = A[(int64_t)j2 * m + j2];
      rank += (dj < di || (dj == di && j2 < i)) ? 1 : 0;
    }
    jb.out[rank] = di;
  }
}

}  // namespace


// Doubles of split-K partial tiles for the three contractions.  The
// exact-slice GEMM splits K into blocks of at most 1024 (exactness) and, for
// outputs with few tiles, into about two blocks per SM; the float64 GEMM fits
// its split count to the capacity it is given.
static int64_t mp2_scratch(int64_t o, int64_t v, int64_t naux, bool oz, int num_sms) {
  const int64_t ov = o * v;
  const int64_t f64 = std::max<int64_t>(splitk_cap(o, v), 80LL * std::max(o * o, v * v));
  if (!oz) return f64;
  return std::max({gemm_oz_scratch(ov, ov, naux, num_sms), f64, (int64_t)1});  // (ia|jb) split K
}

static size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

// Bytes of workspace one cluster uses while its contractions run (the largest
// is allocated; the next cluster reuses it).
static size_t mp2_bytes(int64_t o, int64_t v, int64_t naux, bool oz, int num_sms) {
  const size_t ovov = (size_t)o * v * o * v, t2n = (size_t)o * o * v * v;
  size_t b = al256(ovov * 8) + 2 * al256(t2n * 8);                       // ovov, t2 (own copy), T~
  b += al256((size_t)mp2_scratch(o, v, naux, oz, num_sms) * 8);          // split-K partial tiles
  if (oz) b += al256((size_t)naux * o * v * 8) + al256(64);              // slices of Bov (4 x 2 B per element), scale
  return b;
}

// Bytes one cluster keeps until its group's eigensolver launch: the gamma
// blocks (when the caller did not ask for them) and global working copies for
// orders above kJacobiSmemM.
static size_t mp2_keep_bytes(int64_t o, int64_t v) {
  const int64_t mo = (o + 1) / 2 * 2, mv = (v + 1) / 2 * 2;
  size_t b = al256((size_t)o * o * 8) + al256((size_t)v * v * 8);
  if (mo > kJacobiSmemM) b += al256((size_t)mo * mo * 8);
  if (mv > kJacobiSmemM) b += al256((size_t)mv * mv * 8);
  return b;
}

// Clusters per eigensolver launch: two matrices each, 64 jobs.
constexpr int64_t kMp2Group = 32;

static cudaError_t launch_jacobi(EigJobs* jobs, cudaStream_t s) {
  size_t bytes = 16;
  for (int k = 0; k < jobs->count; ++k) bytes = std::max(bytes, jacobi_smem_bytes(jobs->j[k]));
  cudaError_t e = cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k_jacobi<<<jobs->count, 512, bytes, s>>>(*jobs);
  jobs->count = 0;
  return cudaGetLastError();
}

}  // namespace te

using namespace te;

extern "C" te_status t_mp2_bno_batched(te_handle hh, const te_mp2_cluster* cs, const te_mp2_out* outs, int64_t n,
                                       te_precision p, te_stream_t ss) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(ss);
  if (!h) return fail(TE_EINVAL, "null handle");
  if (n < 0) return fail(TE_EINVAL, "negative batch size");
  if (n == 0) return TE_OK;
  if (!cs || !outs) return fail(TE_EINVAL, "null cluster or output array");
  if (p != TE_FP64 && p != TE_OZAKI)
    return fail(TE_EUNSUPPORTED, "the MP2 step runs in TE_FP64 or TE_OZAKI (got %d)", (int)p);
  if (h->capturing) return fail(TE_EINVAL, "the MP2 step cannot run inside the library's graph capture");
  if (p == TE_OZAKI && h->cc_major != 10 && h->cc_major != 11)
    return fail(TE_EUNSUPPORTED, "exact-slice contractions need an sm_100-family GPU");
  const bool oz = p == TE_OZAKI;
  size_t need_tr = 0, need_keep = 0, group_keep = 0;
  for (int64_t x = 0; x < n; ++x) {  // every descriptor before any launch
    const te_mp2_cluster& c = cs[x];
    if (c.nocc < 1 || c.nvir < 1 || c.naux < 1)
      return fail(TE_EINVAL, "cluster %lld: nocc, nvir and naux must be >= 1", (long long)x);
    if (c.nocc > 2048 || c.nvir > 4094 || c.naux > (1LL << 20))
      return fail(TE_EUNSUPPORTED, "cluster %lld too large (nocc <= 2048, nvir <= 4094)", (long long)x);
    if (!c.eps_o || !c.eps_v || !c.Bov) return fail(TE_EINVAL, "cluster %lld: null input pointer", (long long)x);
    const te_mp2_out& q = outs[x];
    if (!q.t2 && !q.gamma_oo && !q.gamma_vv && !q.pop_o && !q.pop_v)
      return fail(TE_EINVAL, "cluster %lld: no output requested", (long long)x);
    need_tr = std::max(need_tr, mp2_bytes(c.nocc, c.nvir, c.naux, oz, h->num_sms));
    if (x % kMp2Group == 0) group_keep = 0;
    group_keep += mp2_keep_bytes(c.nocc, c.nvir);
    need_keep = std::max(need_keep, group_keep);
  }
  const size_t need = need_keep + need_tr + 1024;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != h->device) cudaSetDevice(h->device);
  struct Restore {
    int prev, dev;
    ~Restore() {
      if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    }
  } restore{prev, h->device};
  te_status st = ensure_workspace_public(h, need);
  if (st != TE_OK) return st;
  EigJobs* jobs = new EigJobs;
  std::memset(jobs, 0, sizeof(*jobs));
  cudaError_t e = cudaSuccess;
  char* const ws0 = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(h->ws) + 255) & ~uintptr_t(255));
  char* keep = ws0;                       // kept blocks of the current group
  char* const transient = ws0 + need_keep;  // one cluster's contractions
  for (int64_t x = 0; x < n && e == cudaSuccess; ++x) {
    const te_mp2_cluster& c = cs[x];
    const te_mp2_out& q = outs[x];
    const int64_t o = c.nocc, v = c.nvir, P = c.naux;
    const int64_t ov = o * v, t2n = o * o * v * v;
    if (x % kMp2Group == 0) keep = ws0;
    auto take_from = [](char*& base, size_t bytes) {
      char* r = base;
      base += al256(bytes);
      return r;
    };
    char* base = transient;
    auto take = [&](size_t bytes) { return take_from(base, bytes); };
    double* ovov = reinterpret_cast<double*>(take((size_t)ov * ov * 8));
    double* t2 = reinterpret_cast<double*>(take((size_t)t2n * 8));
    double* tt = reinterpret_cast<double*>(take((size_t)t2n * 8));
    double* goo = reinterpret_cast<double*>(take_from(keep, (size_t)o * o * 8));
    double* gvv = reinterpret_cast<double*>(take_from(keep, (size_t)v * v * 8));
    const int mo = (int)((o + 1) / 2 * 2), mv = (int)((v + 1) / 2 * 2);
    double* eo_work = mo > kJacobiSmemM ? reinterpret_cast<double*>(take_from(keep, (size_t)mo * mo * 8)) : nullptr;
    double* ev_work = mv > kJacobiSmemM ? reinterpret_cast<double*>(take_from(keep, (size_t)mv * mv * 8)) : nullptr;
    const int64_t cap = mp2_scratch(o, v, P, oz, h->num_sms);
    const int64_t cap64 = std::min(cap, mp2_scratch(o, v, P, false, h->num_sms));
    double* scratch = reinterpret_cast<double*>(take((size_t)cap * 8));
    if (q.t2) t2 = q.t2;
    if (q.gamma_oo) goo = q.gamma_oo;
    if (q.gamma_vv) gvv = q.gamma_vv;
    // input values: finite, max eps_o < min eps_v (reported by te_sync)
    e = launch_check_mp2(c.eps_o, o, c.eps_v, v, c.Bov, P * ov, x, h->d_err, h->num_sms, s);
    ++h->n_launches;
    // (ia|jb) = sum_P B[P,i,a] B[P,j,b]: rows (i,a), columns (j,b), K = P
    if (e == cudaSuccess) e = cudaMemsetAsync(ovov, 0, (size_t)ov * ov * 8, s);
    if (!oz) {
      if (e == cudaSuccess)
        e = gemm_strided(GemmView{c.Bov, c.Bov, ovov, o, v, ov, P, 1, v, 1, ov, 0, ov, 0, 1, v * ov, ov, 1, 1.0},
                         h->num_sms, scratch, cap, s, &h->n_launches);
    } else {
      __nv_bfloat16* bs = reinterpret_cast<__nv_bfloat16*>(take((size_t)P * ov * 8));
      unsigned long long* mx = reinterpret_cast<unsigned long long*>(take(64));
      int* ex = reinterpret_cast<int*>(mx + 3);
      if (e == cudaSuccess) e = slice_planes(c.Bov, P * ov, 4, mx, ex, bs, s, &h->n_launches);
      if (e == cudaSuccess)
        e = gemm_oz(OzView{bs, bs, P * ov, P * ov, ovov, o, v, ov, P, 1, v, 1, ov, 0, ov, 0, 1, v * ov, ov, 1, 1.0,
                           ex, ex, 0},
                    h->num_sms, scratch, cap, s, &h->n_launches);
    }
    // amplitudes, then the two density contractions in float64 in both modes:
    // their K (o^2 v and o v^2 terms) spans the amplitudes' whole dynamic
    // range, which one power-of-two scale per array would not resolve
    {
      if (e == cudaSuccess) {
        k_mp2_amplitudes<<<grid_of(t2n), 256, 0, s>>>(ovov, c.eps_o, c.eps_v, (int)o, (int)v, t2, tt);
        ++h->n_launches;
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaMemsetAsync(gvv, 0, (size_t)v * v * 8, s);
      if (e == cudaSuccess)
        e = gemm_strided(GemmView{t2, tt, gvv, v, 1, v, o * o, v, v, 0, v * v, 1, v * v, 1, v, v, 0, 1, 2.0},
                         h->num_sms, scratch, cap64, s, &h->n_launches);
      if (e == cudaSuccess) {
        k_two_identity<<<grid_of(o * o), 256, 0, s>>>(goo, (int)o);
        ++h->n_launches;
        e = cudaGetLastError();
      }
      if (e == cudaSuccess)
        e = gemm_strided(
            GemmView{t2, tt, goo, o, 1, o, o, v * v, o * v * v, 0, v * v, 1, v * v, 1, o * v * v, o, 0, 1, -2.0},
            h->num_sms, scratch, cap64, s, &h->n_launches);
    }
    // populations: one eigensolver block per requested matrix, launched
    // once per group of clusters (their blocks stay in the kept region)
    if (e == cudaSuccess) {
      if (q.pop_o) jobs->j[jobs->count++] = EigJob{eo_work, goo, q.pop_o, (int)o, mo};
      if (q.pop_v) jobs->j[jobs->count++] = EigJob{ev_work, gvv, q.pop_v, (int)v, mv};
      if (jobs->count > 0 && ((x + 1) % kMp2Group == 0 || x + 1 == n)) {
        e = launch_jacobi(jobs, s);
        ++h->n_launches;
      }
    }
  }
  delete jobs;
  if (e != cudaSuccess) return fail(TE_ECUDA, "MP2 step launch: %s", cudaGetErrorString(e));
  return TE_OK;
}
