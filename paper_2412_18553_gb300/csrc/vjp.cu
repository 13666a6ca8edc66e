// Adjoint of E(T): dE/d(eps_o, eps_v, ovvv, ooov, ovov, t1, t2), in float64
// (DFMA contractions) or with the contractions on the tensor cores in exact
// BF16 slices (the exact-slice mode's scheme), epilogue and sums in float64.
//
// E = sum over unique occupied triples t of (m_t/3) e_t,
//   e_t = sum_{abc} W~[abc] R[V][abc] / D[abc],  V = W~ + Y,
// with R acting on the virtual indices at fixed ijk (equal to R on the
// occupied ones at fixed abc).  R's coefficient pattern (4, 3-cycles +1,
// transpositions -2) is symmetric and D is invariant under permutations of
// abc, so with w_t = gE m_t / 3:
//   dW~ = w_t R[2 W~ + Y] / D,   dY = w_t R[W~] / D,   dD = -w_t W~ R[V] / D^2.
// W~[a,b,c] = G0[a,b,c] + G1[b,c,a] + G2[c,a,b] gives dG0[x,y,z] = dW~[x,y,z],
// dG1[x,y,z] = dW~[z,x,y], dG2[x,y,z] = dW~[y,z,x]; each G block
//   G(p,q,r)[x,y,z] = sum_d ovvv[p,x,y,d] t2[r,q,z,d] + sum_d ovvv[q,y,x,d] t2[r,p,z,d]
//                   - sum_l t2[l,p,y,x] ooov[q,l,r,z] - sum_l t2[l,q,x,y] ooov[p,l,r,z]
// back-propagates through eight GEMMs (two per K segment).  Y = ovs(ia,jb) t1(kc)
// + ovs(jb,kc) t1(ia) + ovs(ia,kc) t1(jb) with ovs = (ovov + ovov^T)/2 gives the
// ovov and t1 parts.  Triples are processed one after another on the stream
// and every accumulation has a fixed order, so the gradient is deterministic.
#include <atomic>
#include <cuda_bf16.h>

#include <algorithm>
#include <initializer_list>
#include <vector>

#include "strided.h"
#include "tc_path.h"
#include "te_internal.h"
#include "view_tc.h"

namespace te {

// ---------------------------------------------------------------------------
// per-triple adjoint of the energy epilogue, one thread per ordered (a,b,c)
// ---------------------------------------------------------------------------

// orbit index t = a(a+1)(a+2)/6 + b(b+1)/2 + c -> (a, b, c), a >= b >= c
// (FP32 estimates, exact integer fix-ups)
__device__ __forceinline__ void orbit_abc(int64_t t, int* pa, int* pb, int* pc) {
  int a = (int)cbrtf(6.0f * (float)t);
  while (a > 0 && (int64_t)a * (a + 1) * (a + 2) / 6 > t) --a;
  while ((int64_t)(a + 1) * (a + 2) * (a + 3) / 6 <= t) ++a;
  const int64_t rem = t - (int64_t)a * (a + 1) * (a + 2) / 6;
  int b = (int)sqrtf(2.0f * (float)rem);
  while (b > 0 && (int64_t)b * (b + 1) / 2 > rem) --b;
  while ((int64_t)(b + 1) * (b + 2) / 2 <= rem) ++b;
  *pa = a;
  *pb = b;
  *pc = (int)(rem - (int64_t)b * (b + 1) / 2);
}

// blocks of the adjoint epilogue: a fixed number per device, so the orbits
// each block takes, and every partial sum, do not depend on the cluster
int adjoint_grid(int num_sms) { return std::min(4 * std::max(1, num_sms), 8192); }

// Threads stride over the orbits a >= b >= c (v(v+1)(v+2)/6 of them): W~ and Y
// are formed once per orbit and every distinct element of the orbit gets its
// dW~, dY and dD.  1/D is Newton's iteration x <- x (2 - D x) from an FP32
// seed, twice (relative error below 2^-90 before rounding): float64 division
// costs several times more on GB300's float64 units.  Each block writes its
// energy and dD partial sums to epart, dpart[blockIdx.x].
__global__ void __launch_bounds__(256) k_adjoint(AdjArgs A) {
  __shared__ double red[8], redd[8];
  const int64_t v = A.v;
  const int64_t norb = v * (v + 1) * (v + 2) / 6;
  const double eo = A.eps_o[A.i] + A.eps_o[A.j] + A.eps_o[A.k];
  double contrib = 0.0, dsum = 0.0, wmax = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < norb; t += (int64_t)gridDim.x * blockDim.x) {
    int a, b, c;
    orbit_abc(t, &a, &b, &c);
    double W[6], Y[6], RW[6], RY[6];
    int64_t idx[6];
    orbit_values(A, a, b, c, W, Y);
    orbit_index(v, a, b, c, idx);
    r_orbit(W, RW);
    r_orbit(Y, RY);
    const unsigned distinct = orbit_distinct(a, b, c);
    const double D = eo - A.eps_v[a] - A.eps_v[b] - A.eps_v[c];
    double rD = (double)__frcp_rn((float)D);
    rD = fma(rD, fma(-D, rD, 1.0), rD);
    rD = fma(rD, fma(-D, rD, 1.0), rD);
    const double q = A.w * rD;
#pragma unroll
    for (int n = 0; n < 6; ++n) {
      if (!(distinct >> n & 1u)) continue;
      const double RV = RW[n] + RY[n];
      const double dw = q * (2.0 * RW[n] + RY[n]);
      const double dd = -q * W[n] * RV * rD;
      A.dW[idx[n]] = dw;
      A.dY[idx[n]] = q * RW[n];
      A.dD[idx[n]] = dd;
      dsum += dd;
      contrib += W[n] * RV * rD;
      wmax = fmax(wmax, fabs(dw));
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    contrib += __shfl_down_sync(0xffffffffu, contrib, off);
    dsum += __shfl_down_sync(0xffffffffu, dsum, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = contrib;
    redd[threadIdx.x >> 5] = dsum;
  }
  if (A.dwmax) {
    double m = wmax;
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(A.dwmax, (unsigned long long)__double_as_longlong(m));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0, sd = 0.0;
    for (int w = 0; w < 8; ++w) {
      s += red[w];
      sd += redd[w];
    }
    A.epart[blockIdx.x] = s;
    A.dpart[blockIdx.x] = sd;
  }
}

// ---------------------------------------------------------------------------
// generic strided float64 GEMM:  C[m,n] += alpha sum_k A[m,k] B[k,n]
// m = (m1, m2), k = (k1, k2), each index with its own stride.  Outputs with
// few tiles (the contractions over a virtual pair, K = v^2) split K over
// blockIdx.z into fixed ranges; the partial tiles go to a scratch array and
// are added in split order by k_splitk_add, so the result is deterministic.
// ---------------------------------------------------------------------------


constexpr int GT = 64, GK = 16;

// (k1, k2) of k = k1 K2 + k2, advanced by GK per step without division
struct KCursor {
  int k1, k2;
  __device__ __forceinline__ void init(int k, int K2) {
    k1 = k / K2;
    k2 = k - k1 * K2;
  }
  __device__ __forceinline__ void step(int K2) {
    k2 += GK;
    while (k2 >= K2) {
      k2 -= K2;
      ++k1;
    }
  }
};

__global__ void __launch_bounds__(256) k_gemm_strided(GemmView g, int kchunk, double* __restrict__ part) {
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  const int tid = threadIdx.x;
  const int M = (int)(g.M1 * g.M2), K = (int)(g.K1 * g.K2), K2 = (int)g.K2;
  const int m0 = blockIdx.x * GT, n0 = blockIdx.y * GT;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  const int tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  // loader: 64 rows (m or n) x 16 k; thread (lr, lk .. lk+3)
  const int lr = tid >> 2, lk = (tid & 3) * 4;
  const int am = m0 + lr;
  const bool am_ok = am < M;
  const int64_t a_row = am_ok ? (int64_t)(am / (int)g.M2) * g.a_m1 + (int64_t)(am % (int)g.M2) * g.a_m2 : 0;
  const int bn = n0 + lr;
  const bool bn_ok = bn < (int)g.N;
  const int64_t b_col = bn_ok ? (int64_t)bn * g.b_n : 0;
  KCursor cur[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) cur[u].init(kb + lk + u, K2);
  for (int k0 = kb; k0 < ke; k0 += GK) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool k_ok = k0 + lk + u < ke;
      const int64_t ka = (int64_t)cur[u].k1 * g.a_k1 + (int64_t)cur[u].k2 * g.a_k2;
      const int64_t kbo = (int64_t)cur[u].k1 * g.b_k1 + (int64_t)cur[u].k2 * g.b_k2;
      As[lk + u][lr] = (am_ok && k_ok) ? g.A[a_row + ka] : 0.0;
      Bs[lk + u][lr] = (bn_ok && k_ok) ? g.B[b_col + kbo] : 0.0;
      cur[u].step(K2);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][ty * 4 + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx * 4 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int m = m0 + ty * 4 + a;
    if (m >= M) continue;
    if (part) {  // split K: this split's tile, row-major [M][N]
      double* prow = part + ((int64_t)blockIdx.z * M + m) * g.N;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int n = n0 + tx * 4 + b;
        if (n < g.N) prow[n] = acc[a][b];
      }
    } else {
      const int64_t crow = (int64_t)(m / (int)g.M2) * g.c_m1 + (int64_t)(m % (int)g.M2) * g.c_m2;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int n = n0 + tx * 4 + b;
        if (n < g.N) g.C[crow + n * g.c_n] += g.alpha * acc[a][b];
      }
    }
  }
}

// C[m,n] += alpha sum_z part[z][m][n], z in order
__global__ void k_splitk_add(GemmView g, int nsplit, const double* __restrict__ part) {
  const int M = (int)(g.M1 * g.M2);
  const int64_t MN = (int64_t)M * g.N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < MN; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;  // in split order; unrolled so that many loads are in flight
#pragma unroll 16
    for (int z = 0; z < nsplit; ++z) s += part[z * MN + e];
    const int m = (int)(e / g.N), n = (int)(e % g.N);
    const int64_t crow = (int64_t)(m / (int)g.M2) * g.c_m1 + (int64_t)(m % (int)g.M2) * g.c_m2;
    g.C[crow + n * g.c_n] += g.alpha * s;
  }
}

// Split count for a GEMM of `tiles` output tiles and K steps: about two
// blocks per SM, each split at least 8 K steps; the scratch holds `cap`
// doubles.
static int num_splits(int64_t tiles, int64_t K, int64_t MN, int num_sms, int64_t cap) {
  const int64_t steps = (K + GK - 1) / GK;
  int64_t want = (2LL * num_sms + tiles - 1) / tiles;
  want = std::min<int64_t>(want, std::max<int64_t>(1, steps / 8));
  want = std::min<int64_t>(want, std::max<int64_t>(1, cap / std::max<int64_t>(1, MN)));
  return (int)std::max<int64_t>(1, want);
}

cudaError_t gemm_strided(const GemmView& g, int num_sms, double* scratch, int64_t scratch_cap, cudaStream_t s,
                         int64_t* launches) {
  const int64_t M = g.M1 * g.M2, K = g.K1 * g.K2;
  const int64_t tm = (M + GT - 1) / GT, tn = (g.N + GT - 1) / GT;
  const int ns = num_splits(tm * tn, K, M * g.N, num_sms, scratch_cap);
  const int64_t steps = (K + GK - 1) / GK;
  const int kchunk = (int)(((steps + ns - 1) / ns) * GK);
  const int nsplit = (int)((K + kchunk - 1) / kchunk);
  dim3 grid((unsigned)tm, (unsigned)tn, (unsigned)nsplit);
  k_gemm_strided<<<grid, 256, 0, s>>>(g, kchunk, nsplit > 1 ? scratch : nullptr);
  ++*launches;
  if (nsplit > 1) {
    const int64_t MN = M * g.N;
    k_splitk_add<<<(unsigned)std::min<int64_t>((MN + 255) / 256, 4096), 256, 0, s>>>(g, nsplit, scratch);
    ++*launches;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// exact-slice strided GEMM on the tensor cores (mma.sync, BF16 -> FP32):
//   C[m,n] (+)= alpha 2^(ea + eb) sum_k A[m,k] B[k,n]
// A and B are NS BF16 slice planes each (slice s at base + s * plane; NS = 4,
// or 5 for 35-bit operands), read through the same two-index strided views as
// the float64 kernel.  The slice products a_i b_j with i + j <= NS - 1 (ten,
// or fifteen) go to three FP32 accumulators:
// level 0 and level 1 exactly (K <= 1024 per block keeps their partial sums
// integer multiples of the level's unit below 2^24), the higher levels
// approximately; each block's sums go to float64 once, at its end.
// ---------------------------------------------------------------------------


constexpr int OZ_BM = 64, OZ_BN = 64, OZ_BK = 32, OZ_KMAX = 1024;
constexpr int OZ_THREADS = 256;  // eight warps, each 32 x 16 outputs
constexpr int OZ_LD = OZ_BK + 8;  // padded row (bf16): conflict-free fragment loads

__device__ __forceinline__ void mma_bf16_16816(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Tiles of 64 x 64 outputs, 32 k per stage, two stages in flight (cp.async).
// Each operand tile sits in shared memory k-major ([row][k]) when its view is
// contiguous along k, else row-major ([k][row]) when contiguous along its rows
// (columns); 16-byte chunks of eight BF16 values are copied asynchronously
// where the view allows, element by element otherwise.
template <bool AK, bool BK, int NS>
struct OzTile {
  static constexpr int A = AK ? OZ_BM * OZ_LD : OZ_BK * (OZ_BM + 8);
  static constexpr int B = BK ? OZ_BN * OZ_LD : OZ_BK * (OZ_BN + 8);
  static constexpr int STAGE = NS * (A + B);  // elements
  static constexpr size_t BYTES = 2 * STAGE * sizeof(__nv_bfloat16);
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// four 8 x 8 BF16 matrices from shared memory, as stored / transposed
__device__ __forceinline__ void ldsm_x4(uint32_t* r, const __nv_bfloat16* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"((uint32_t)__cvta_generic_to_shared(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t* r, const __nv_bfloat16* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"((uint32_t)__cvta_generic_to_shared(p)));
}

// Eight elements (rows r + e step_r, k + e step_k) of every slice, element by
// element, zero outside the view: ragged edges and views without a
// contiguous index.  Rolled loops, so the pipelined loop stays small enough
// for the instruction cache.
__device__ __forceinline__ void oz_fill_slow(const __nv_bfloat16* __restrict__ src, int64_t ps, __nv_bfloat16* dst,
                                          int dps, int ns, int r, int k, int step_r, int step_k, int R, int ke,
                                          int R2, int64_t r1s, int64_t r2s, int K2, int64_t k1s, int64_t k2s) {
#pragma unroll 1
  for (int e = 0; e < 8; ++e) {
    const int rr = r + e * step_r, kk = k + e * step_k;
    const bool ok = rr < R && kk < ke;
    const int64_t off =
        ok ? (int64_t)(rr / R2) * r1s + (int64_t)(rr % R2) * r2s + (int64_t)(kk / K2) * k1s + (int64_t)(kk % K2) * k2s
           : 0;
#pragma unroll 1
    for (int sl = 0; sl < ns; ++sl) dst[sl * dps + e] = ok ? src[off + sl * ps] : __float2bfloat16_rn(0.f);
  }
}

template <bool AK, bool BK, int NS>
__global__ void __launch_bounds__(OZ_THREADS, 2) k_gemm_oz2(OzView g, int kchunk, double* __restrict__ part,
                                                            int a_vec, int b_vec) {
  using T = OzTile<AK, BK, NS>;
  extern __shared__ __align__(16) unsigned char oz_smem[];
  __nv_bfloat16* smem = reinterpret_cast<__nv_bfloat16*>(oz_smem);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int M = (int)(g.M1 * g.M2), N = (int)g.N, K2 = (int)g.K2;
  const int m0 = blockIdx.x * OZ_BM, n0 = blockIdx.y * OZ_BN;
  const int kb = blockIdx.z * kchunk, ke = min((int)(g.K1 * g.K2), kb + kchunk);
  const int nst = (ke - kb + OZ_BK - 1) / OZ_BK;

  auto a_row = [&](int m) { return (int64_t)(m / (int)g.M2) * g.a_m1 + (int64_t)(m % (int)g.M2) * g.a_m2; };
  auto a_kof = [&](int k) { return (int64_t)(k / K2) * g.a_k1 + (int64_t)(k % K2) * g.a_k2; };
  auto b_kof = [&](int k) { return (int64_t)(k / K2) * g.b_k1 + (int64_t)(k % K2) * g.b_k2; };
  // 256 chunks of 8 elements per slice and operand, OZ_CH per thread; the row
  // (column) part of a chunk's offset is the same at every stage
  constexpr int OZ_CH = 256 / OZ_THREADS;
  int64_t a_roff[OZ_CH];
#pragma unroll
  for (int c2 = 0; c2 < OZ_CH; ++c2) {
    const int c = tid + OZ_THREADS * c2;
    const int m = AK ? m0 + (c >> 2) : m0 + (c & 7) * 8;
    a_roff[c2] = m < M ? a_row(m) : 0;
  }

  // one 8-element chunk: elements e = 0..7 along the tile's contiguous direction
  auto load_stage = [&](int buf, int k0) {
    __nv_bfloat16* As = smem + buf * T::STAGE;
    __nv_bfloat16* Bs = As + NS * T::A;
#pragma unroll
    for (int c2 = 0; c2 < OZ_CH; ++c2) {
      const int c = tid + OZ_THREADS * c2;
      // ---- A ----
      {
        int m, k, step_m, step_k;  // first element and the step between the 8
        __nv_bfloat16* dst0;
        if (AK) {
          m = m0 + (c >> 2);
          k = k0 + (c & 3) * 8;
          step_m = 0;
          step_k = 1;
          dst0 = As + (c >> 2) * OZ_LD + (c & 3) * 8;
        } else {
          k = k0 + (c >> 3);
          m = m0 + (c & 7) * 8;
          step_m = 1;
          step_k = 0;
          dst0 = As + (c >> 3) * (OZ_BM + 8) + (c & 7) * 8;
        }
        const bool full = a_vec && (AK ? (m < M && k + 8 <= ke) : (k < ke && m + 8 <= M));
        if (full) {
          const __nv_bfloat16* src = g.A + a_roff[c2] + a_kof(k);
#pragma unroll
          for (int sl = 0; sl < NS; ++sl) cp_async16(dst0 + sl * T::A, src + sl * g.a_ps);
        } else {
          oz_fill_slow(g.A, g.a_ps, dst0, T::A, NS, m, k, step_m, step_k, M, ke, (int)g.M2, g.a_m1, g.a_m2, K2,
                       g.a_k1, g.a_k2);
        }
      }
      // ---- B ----
      {
        int n, k, step_n, step_k;
        __nv_bfloat16* dst0;
        if (BK) {
          n = n0 + (c >> 2);
          k = k0 + (c & 3) * 8;
          step_n = 0;
          step_k = 1;
          dst0 = Bs + (c >> 2) * OZ_LD + (c & 3) * 8;
        } else {
          k = k0 + (c >> 3);
          n = n0 + (c & 7) * 8;
          step_n = 1;
          step_k = 0;
          dst0 = Bs + (c >> 3) * (OZ_BN + 8) + (c & 7) * 8;
        }
        const bool full = b_vec && (BK ? (n < N && k + 8 <= ke) : (k < ke && n + 8 <= N));
        if (full) {
          const __nv_bfloat16* src = g.B + (int64_t)n * g.b_n + b_kof(k);
#pragma unroll
          for (int sl = 0; sl < NS; ++sl) cp_async16(dst0 + sl * T::B, src + sl * g.b_ps);
        } else {
          oz_fill_slow(g.B, g.b_ps, dst0, T::B, NS, n, k, step_n, step_k, N, ke, 1, g.b_n, 0, K2, g.b_k1, g.b_k2);
        }
      }
    }
  };

  const int wm = (warp & 1) * 32, wn = (warp >> 1) * 16;
  const int gq = lane >> 2, tq = lane & 3;
  float acc[3][2][2][4];
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[l][i][j][q] = 0.f;

  if (nst > 0) load_stage(0, kb);
  cp_async_commit();
  for (int st = 0; st < nst; ++st) {
    if (st + 1 < nst) load_stage((st + 1) & 1, kb + (st + 1) * OZ_BK);
    cp_async_commit();
    cp_async_wait1();  // every group but the newest: this stage's copies have landed
    __syncthreads();
    const __nv_bfloat16* As = smem + (st & 1) * T::STAGE;
    const __nv_bfloat16* Bs = As + NS * T::A;
#pragma unroll
    for (int kk = 0; kk < OZ_BK; kk += 16) {
      // ldmatrix: lane l addresses row (l & 7) of 8 x 8 matrix (l >> 3)
      const int lr = lane & 7, lm = lane >> 3;
      uint32_t bf[NS][2][2];
#pragma unroll
      for (int sl = 0; sl < NS; ++sl) {
        // matrices: (cols 0-7, k kk), (cols 0-7, k kk+8), (cols 8-15, k kk), (cols 8-15, k kk+8)
        const __nv_bfloat16* b = Bs + sl * T::B;
        uint32_t t[4];
        const int cb = wn + (lm >> 1) * 8;
        if (BK) ldsm_x4(t, b + (cb + lr) * OZ_LD + kk + (lm & 1) * 8);
        else ldsm_x4_t(t, b + (kk + lr + (lm & 1) * 8) * (OZ_BN + 8) + cb);
        bf[sl][0][0] = t[0];
        bf[sl][0][1] = t[1];
        bf[sl][1][0] = t[2];
        bf[sl][1][1] = t[3];
      }
#pragma unroll
      for (int sa = 0; sa < NS; ++sa) {
        uint32_t af[2][4];  // A slice sa, loaded when its products are due
        const __nv_bfloat16* a = As + sa * T::A;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int r = wm + i * 16;
          // matrices: (rows r, k kk), (rows r+8, k kk), (rows r, k kk+8), (rows r+8, k kk+8)
          if (AK) ldsm_x4(af[i], a + (r + lr + (lm & 1) * 8) * OZ_LD + kk + (lm >> 1) * 8);
          else ldsm_x4_t(af[i], a + (kk + lr + (lm >> 1) * 8) * (OZ_BM + 8) + r + (lm & 1) * 8);
        }
#pragma unroll
        for (int sb = 0; sb < NS - sa; ++sb) {
          const int lev = sa + sb == 0 ? 0 : (sa + sb == 1 ? 1 : 2);
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) mma_bf16_16816(acc[lev][i][j], af[i], bf[sb][j]);
        }
      }
    }
    __syncthreads();  // the buffer is refilled two stages on
  }
  const double scale = ldexp(g.alpha, *g.ea + *g.eb);
  // this thread's four output rows (i, half h) and their offsets in C
  int64_t crow[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int m = m0 + wm + i * 16 + gq + hh * 8;
      crow[i][hh] = m < M ? (int64_t)(m / (int)g.M2) * g.c_m1 + (int64_t)(m % (int)g.M2) * g.c_m2 : 0;
    }
  // Per 16-row half: every old value of C is loaded before any store, so the
  // loads overlap (a store could otherwise alias the next load).
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    double val[2][4], old[2][4];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + wm + i * 16 + gq + (q >> 1) * 8;
        const int n = n0 + wn + j * 8 + 2 * tq + (q & 1);
        val[j][q] = scale * (((double)acc[0][i][j][q] + (double)acc[1][i][j][q]) + (double)acc[2][i][j][q]);
        old[j][q] = (!part && !g.overwrite && m < M && n < N) ? g.C[crow[i][q >> 1] + n * g.c_n] : 0.0;
      }
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + wm + i * 16 + gq + (q >> 1) * 8;
        const int n = n0 + wn + j * 8 + 2 * tq + (q & 1);
        if (m >= M || n >= N) continue;
        if (part) part[((int64_t)blockIdx.z * M + m) * N + n] = val[j][q];
        else g.C[crow[i][q >> 1] + n * g.c_n] = old[j][q] + val[j][q];
      }
  }
}

// C[m,n] += sum_z part[z][m][n], z in order (alpha is already applied)
__global__ void k_splitk_add_oz(OzView g, int nsplit, const double* __restrict__ part) {
  const int M = (int)(g.M1 * g.M2);
  const int64_t MN = (int64_t)M * g.N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < MN; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;  // in split order; unrolled so that many loads are in flight
#pragma unroll 16
    for (int z = 0; z < nsplit; ++z) s += part[z * MN + e];
    const int m = (int)(e / g.N), n = (int)(e % g.N);
    double* cp = g.C + (int64_t)(m / (int)g.M2) * g.c_m1 + (int64_t)(m % (int)g.M2) * g.c_m2 + n * g.c_n;
    *cp = g.overwrite ? s : *cp + s;
  }
}

template <bool AK, bool BK, int NS>
static cudaError_t launch_oz2(const OzView& g, dim3 grid, int kchunk, double* part, int av, int bv, cudaStream_t s) {
  const size_t bytes = OzTile<AK, BK, NS>::BYTES;
  static std::atomic<unsigned long long> opted{0};  // devices this instantiation may use `bytes` on
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(opted.load() & bit)) {
    e = cudaFuncSetAttribute(k_gemm_oz2<AK, BK, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    opted.fetch_or(bit);
  }
  k_gemm_oz2<AK, BK, NS><<<grid, OZ_THREADS, bytes, s>>>(g, kchunk, part, av, bv);
  return cudaGetLastError();
}

// K in splits of at most OZ_KMAX (exactness), more when the output has few
// tiles: the K chunk per split (a multiple of OZ_BK)
static int oz_kchunk(int64_t M, int64_t N, int64_t K, int num_sms) {
  const int64_t tm = (M + OZ_BM - 1) / OZ_BM, tn = (N + OZ_BN - 1) / OZ_BN;
  const int64_t steps = (K + OZ_BK - 1) / OZ_BK;
  int64_t ns = std::max<int64_t>((K + OZ_KMAX - 1) / OZ_KMAX, (2LL * num_sms + tm * tn - 1) / (tm * tn));
  ns = std::min<int64_t>(ns, std::max<int64_t>(1, steps / 4));
  ns = std::max<int64_t>(ns, (K + OZ_KMAX - 1) / OZ_KMAX);
  return (int)(((steps + ns - 1) / ns) * OZ_BK);
}

int64_t gemm_oz_scratch(int64_t M, int64_t N, int64_t K, int num_sms) {
  const int kchunk = oz_kchunk(M, N, K, num_sms);
  const int64_t nsplit = (K + kchunk - 1) / kchunk;
  return nsplit > 1 ? nsplit * M * N : 0;
}

cudaError_t gemm_oz(const OzView& g, int num_sms, double* scratch, int64_t scratch_cap, cudaStream_t s,
                           int64_t* launches) {
  const int64_t M = g.M1 * g.M2, K = g.K1 * g.K2;
  const int64_t tm = (M + OZ_BM - 1) / OZ_BM, tn = (g.N + OZ_BN - 1) / OZ_BN;
  const int kchunk = oz_kchunk(M, g.N, K, num_sms);
  const int nsplit = (int)((K + kchunk - 1) / kchunk);
  if (nsplit > 1 && (int64_t)nsplit * M * g.N > scratch_cap) return cudaErrorInvalidValue;
  dim3 grid((unsigned)tm, (unsigned)tn, (unsigned)nsplit);
  // tile orientation per operand: k-major if the view is contiguous along k,
  // else row-major if contiguous along its rows (columns), else k-major
  // element by element
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  const bool a_k = g.a_ps % 8 == 0 && al16(g.A) &&
                   ((g.K2 == 1 && g.a_k1 == 1) || (g.K2 % 8 == 0 && g.a_k2 == 1 && g.a_k1 % 8 == 0)) &&
                   (g.a_m1 % 8 == 0 || g.M1 == 1) && (g.a_m2 % 8 == 0 || g.M2 == 1);
  const bool a_m = !a_k && g.a_ps % 8 == 0 && al16(g.A) &&
                   ((g.M2 == 1 && g.a_m1 == 1) || (g.M2 % 8 == 0 && g.a_m2 == 1 && g.a_m1 % 8 == 0)) &&
                   g.a_k1 % 8 == 0 && (g.K2 == 1 || g.a_k2 % 8 == 0);
  const bool b_k = g.b_ps % 8 == 0 && al16(g.B) &&
                   ((g.K2 == 1 && g.b_k1 == 1) || (g.K2 % 8 == 0 && g.b_k2 == 1 && g.b_k1 % 8 == 0)) && g.b_n % 8 == 0;
  const bool b_n = !b_k && g.b_ps % 8 == 0 && al16(g.B) && g.b_n == 1 && g.b_k1 % 8 == 0 &&
                   (g.K2 == 1 || g.b_k2 % 8 == 0);
  double* pp = nsplit > 1 ? scratch : nullptr;
  const bool AK = !a_m, BK = !b_n;
  const int av = (a_k || a_m) ? 1 : 0, bv = (b_k || b_n) ? 1 : 0;
  cudaError_t err;
  if (g.ns == 5) {
    if (AK && BK) err = launch_oz2<true, true, 5>(g, grid, kchunk, pp, av, bv, s);
    else if (AK) err = launch_oz2<true, false, 5>(g, grid, kchunk, pp, av, bv, s);
    else if (BK) err = launch_oz2<false, true, 5>(g, grid, kchunk, pp, av, bv, s);
    else err = launch_oz2<false, false, 5>(g, grid, kchunk, pp, av, bv, s);
  } else if (g.ns == 0 || g.ns == 4) {
    if (AK && BK) err = launch_oz2<true, true, 4>(g, grid, kchunk, pp, av, bv, s);
    else if (AK) err = launch_oz2<true, false, 4>(g, grid, kchunk, pp, av, bv, s);
    else if (BK) err = launch_oz2<false, true, 4>(g, grid, kchunk, pp, av, bv, s);
    else err = launch_oz2<false, false, 4>(g, grid, kchunk, pp, av, bv, s);
  } else {
    return cudaErrorInvalidValue;
  }
  if (err != cudaSuccess) return err;
  ++*launches;
  if (nsplit > 1) {
    const int64_t MN = M * g.N;
    k_splitk_add_oz<<<(unsigned)std::min<int64_t>((MN + 255) / 256, 4096), 256, 0, s>>>(g, nsplit, scratch);
    ++*launches;
  }
  return cudaGetLastError();
}

// max |x| as the bit pattern of a non-negative double (they order as integers)
__global__ void k_maxabs_bits(const double* __restrict__ x, int64_t n, unsigned long long* out) {
  double m = 0.0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[idx]));
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// NS 7-bit BF16 slices of x (slice s at planes + s n): x = 2^e sum_s m_s
// 2^-7(s+1) + r, 2^e > max |x|, |r| <= 2^(e - 7 NS - 1)
template <int NS>
__global__ void k_slice_planes(const double* __restrict__ x, int64_t n, const unsigned long long* __restrict__ xmax,
                               int* __restrict__ e_out, __nv_bfloat16* __restrict__ planes) {
  const double mx = __longlong_as_double((long long)*xmax);
  int ex = 0;
  if (mx > 0.0) frexp(mx, &ex);
  if (blockIdx.x == 0 && threadIdx.x == 0) *e_out = ex;
  const double sc = ldexp(1.0, -ex);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double t = x[i] * sc;  // |t| < 1
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      t = t * 128.0;
      const double m = rint(t);
      t = t - m;
      planes[k * n + i] = __float2bfloat16_rn((float)(m * (1.0 / (double)(1ull << (7 * (k + 1))))));
    }
  }
}

cudaError_t slice_planes(const double* x, int64_t n, int ns, unsigned long long* mx, int* ex,
                         __nv_bfloat16* planes, cudaStream_t s, int64_t* launches) {
  if (ns != 4 && ns != 5) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(mx, 0, 8, s);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<int64_t>(std::max<int64_t>(1, (n + 255) / 256), 8192);
  k_maxabs_bits<<<std::min(grid, 1024), 256, 0, s>>>(x, n, mx);
  if (ns == 5) k_slice_planes<5><<<grid, 256, 0, s>>>(x, n, mx, ex, planes);
  else k_slice_planes<4><<<grid, 256, 0, s>>>(x, n, mx, ex, planes);
  *launches += 2;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Y and denominator reductions for one triple
// ---------------------------------------------------------------------------

// dOVS[P1][x][P2][y] += sum_z dY[perm(x,y,z)] t1[P3][z]   (one of the three Y terms)
// mode 0: ovs(i,a,j,b) t1(k,c): out (a,b), sum over c; t1 row k
// mode 1: ovs(j,b,k,c) t1(i,a): out (b,c), sum over a; t1 row i
// mode 2: ovs(i,a,k,c) t1(j,b): out (a,c), sum over b; t1 row j
__global__ void k_dovs(int mode, int o, int v, int i, int j, int k, const double* __restrict__ dY,
                       const double* __restrict__ t1, double* __restrict__ dOVS) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)v * v) return;
  const int x = (int)(idx / v), y = (int)(idx % v);
  const int64_t V = v;
  double s = 0.0;
  int P1, P2, P3;
  if (mode == 0) {
    P1 = i; P2 = j; P3 = k;
    for (int c = 0; c < v; ++c) s += dY[(x * V + y) * V + c] * t1[(int64_t)P3 * v + c];
  } else if (mode == 1) {
    P1 = j; P2 = k; P3 = i;
    for (int a = 0; a < v; ++a) s += dY[(a * V + x) * V + y] * t1[(int64_t)P3 * v + a];
  } else {
    P1 = i; P2 = k; P3 = j;
    for (int b = 0; b < v; ++b) s += dY[(x * V + b) * V + y] * t1[(int64_t)P3 * v + b];
  }
  dOVS[(((int64_t)P1 * v + x) * o + P2) * v + y] += s;
}

// fixed-order block sum of 256 threads' values; the result is valid in thread 0
__device__ __forceinline__ double block_sum256(double s, double* red) {
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < 8; ++w) t += red[w];
  return t;
}

// dt1[P3][z] += sum over the other two indices of dY * ovs (one of the three
// Y terms); one block per z
__global__ void __launch_bounds__(256) k_dt1(int mode, int o, int v, int i, int j, int k,
                                              const double* __restrict__ dY, const double* __restrict__ ovs,
                                              double* __restrict__ dt1) {
  __shared__ double red[8];
  const int z = blockIdx.x;
  const int64_t V = v, n = V * V;
  auto OV = [&](int P1, int a, int P2, int b) { return ovs[(((int64_t)P1 * v + a) * o + P2) * v + b]; };
  double s = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    const int p = (int)(e / v), q = (int)(e % v);
    if (mode == 0) s += dY[(p * V + q) * V + z] * OV(i, p, j, q);       // t1(k,c): dY[a,b,c] ovs(i,a,j,b)
    else if (mode == 1) s += dY[(z * V + p) * V + q] * OV(j, p, k, q);  // t1(i,a): dY[a,b,c] ovs(j,b,k,c)
    else s += dY[(p * V + z) * V + q] * OV(i, p, k, q);                 // t1(j,b): dY[a,b,c] ovs(i,a,k,c)
  }
  const double t = block_sum256(s, red);
  if (threadIdx.x == 0) {
    const int row = mode == 0 ? k : (mode == 1 ? i : j);
    dt1[(int64_t)row * v + z] += t;
  }
}

// deps_v[x] -= sum_bc dD[x,b,c] + sum_ac dD[a,x,c] + sum_ab dD[a,b,x]; one block per x
__global__ void __launch_bounds__(256) k_deps_v(int v, const double* __restrict__ dD, double* __restrict__ deps_v) {
  __shared__ double red[8];
  const int x = blockIdx.x;
  const int64_t V = v, n = V * V;
  double s = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    const int p = (int)(e / v), q = (int)(e % v);
    s += dD[(x * V + p) * V + q] + dD[(p * V + x) * V + q] + dD[(p * V + q) * V + x];
  }
  const double t = block_sum256(s, red);
  if (threadIdx.x == 0) deps_v[x] -= t;
}

// deps_o[i], [j], [k] += sum_abc dD, from the adjoint kernel's per-block sums
// (fixed-order block sum)
__global__ void __launch_bounds__(256) k_deps_o(int64_t n, const double* __restrict__ dpart, int i, int j, int k,
                                                 double* __restrict__ deps_o) {
  __shared__ double red[8];
  double s = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) s += dpart[e];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    deps_o[i] += t;
    deps_o[j] += t;
    deps_o[k] += t;
  }
}

// dovov[P1,x,P2,y] = (dOVS[P1,x,P2,y] + dOVS[P2,y,P1,x]) / 2
__global__ void k_dovov(int o, int v, const double* __restrict__ dOVS, double* __restrict__ dovov) {
  const int64_t n = (int64_t)o * v * o * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(idx % v);
    int64_t rest = idx / v;
    const int P2 = (int)(rest % o);
    rest /= o;
    const int x = (int)(rest % v);
    const int P1 = (int)(rest / v);
    dovov[idx] = 0.5 * (dOVS[idx] + dOVS[(((int64_t)P2 * v + y) * o + P1) * v + x]);
  }
}

// sum of the adjoint kernel's per-block partials -> one per-triple share
__global__ void __launch_bounds__(256) k_sum_share(const double* __restrict__ part, int64_t n, double scale,
                                                    double* __restrict__ out) {
  __shared__ double red[8];
  double s = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) s += part[e];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    *out = t * scale;
  }
}

cudaError_t launch_sum_share(const double* part, int64_t n, double scale, double* out, cudaStream_t s) {
  k_sum_share<<<1, 256, 0, s>>>(part, n, scale, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// driver
// ---------------------------------------------------------------------------

struct VjpWork {
  double *t2L, *nooT, *ovs, *G, *dW, *dY, *dD, *dOVS, *epart, *dpart, *shares, *splitk;
};

// doubles of split-K scratch: room for the partial tiles of a v x v output
int64_t splitk_cap(int64_t o, int64_t v) { return 80 * std::max(v * v, o * v); }

size_t vjp_fp64_bytes(int64_t o, int64_t v) {
  const int64_t v3 = v * v * v, nt = num_unique_triples(o);
  const int64_t nblk = std::max<int64_t>((v3 + 255) / 256, 8192);  // at least adjoint_grid's largest
  auto a = [](int64_t n) { return ((size_t)n * 8 + 255) & ~size_t(255); };
  return a(o * v * v * o) + a(o * o * v * o) + a(o * v * o * v) + a(3 * v3) + 3 * a(v3) + a(o * v * o * v) +
         2 * a(nblk) + a(std::max<int64_t>(1, nt)) + a(splitk_cap(o, v)) + 1024;
}

te_status ensure_workspace_public(Handle* h, size_t bytes);
te_status ensure_triples_public(Handle* h, int nocc);

te_status run_vjp_fp64(Handle* h, const te_cluster* c, int64_t t_begin, int64_t t_end, double gE,
                       double* e_out, te_cluster_grad* g, cudaStream_t s) {
  const int o = (int)c->nocc, v = (int)c->nvir;
  const int64_t v2 = (int64_t)v * v, v3 = v2 * v, nt = num_unique_triples(o);
  te_status st = ensure_workspace_public(h, vjp_fp64_bytes(o, v));
  if (st != TE_OK) return st;
  st = ensure_triples_public(h, o);
  if (st != TE_OK) return st;
  char* p = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(h->ws) + 255) & ~uintptr_t(255));
  auto take = [&](int64_t n) {
    double* r = reinterpret_cast<double*>(p);
    p += ((size_t)n * 8 + 255) & ~size_t(255);
    return r;
  };
  VjpWork W;
  W.t2L = take((int64_t)o * v * v * o);
  W.nooT = take((int64_t)o * o * v * o);
  W.ovs = take((int64_t)o * v * o * v);
  W.G = take(3 * v3);
  W.dW = take(v3);
  W.dY = take(v3);
  W.dD = take(v3);
  W.dOVS = take((int64_t)o * v * o * v);
  const int64_t nblk = std::max<int64_t>((v3 + 255) / 256, adjoint_grid(h->num_sms));
  const int64_t agrid = adjoint_grid(h->num_sms);
  W.epart = take(nblk);
  W.dpart = take(nblk);
  W.shares = take(std::max<int64_t>(1, nt));
  W.splitk = take(splitk_cap(o, v));

  // gradient outputs start at zero
  auto zero = [&](double* ptr, int64_t n) {
    return ptr ? cudaMemsetAsync(ptr, 0, sizeof(double) * n, s) : cudaSuccess;
  };
  cudaError_t e = cudaSuccess;
  e = e ? e : zero(g->eps_o, o);
  e = e ? e : zero(g->eps_v, v);
  e = e ? e : zero(g->ovvv, (int64_t)o * v3);
  e = e ? e : zero(g->ooov, (int64_t)o * o * o * v);
  e = e ? e : zero(g->ovov, (int64_t)o * v * o * v);
  e = e ? e : zero(g->t1, (int64_t)o * v);
  e = e ? e : zero(g->t2, (int64_t)o * o * v2);
  e = e ? e : zero(W.dOVS, (int64_t)o * v * o * v);
  if (e != cudaSuccess) return fail(TE_ECUDA, "memset: %s", cudaGetErrorString(e));

  Prepared P{};
  P.o = o;
  P.v = v;
  P.eps_o = c->eps_o;
  P.eps_v = c->eps_v;
  P.ovvv = c->ovvv;
  P.t2 = c->t2;
  P.t1 = c->t1;
  P.t2L = W.t2L;
  P.nooT = W.nooT;
  P.ovs = W.ovs;
  e = launch_prep_fp64(c, &P, s);
  if (e != cudaSuccess) return fail(TE_ECUDA, "prep: %s", cudaGetErrorString(e));

  std::vector<Triple> trip = unique_triples(o);
  for (int64_t t = t_begin; t < t_end && e == cudaSuccess; ++t) {
    const Triple T = trip[t];
    e = launch_gemm_fp64(&P, h->d_triples, t, 1, W.G, s);
    if (e != cudaSuccess) break;
    AdjArgs A{};  // value-initialised: optional pointers (dwmax) are null unless set
    A.o = o; A.v = v; A.i = T.i; A.j = T.j; A.k = T.k;
    A.w = gE * (double)T.m / 3.0;
    A.G = W.G; A.ovs = W.ovs; A.t1 = c->t1; A.eps_o = c->eps_o; A.eps_v = c->eps_v;
    A.dW = W.dW; A.dY = W.dY; A.dD = W.dD; A.epart = W.epart; A.dpart = W.dpart;
    k_adjoint<<<(unsigned)agrid, 256, 0, s>>>(A);
    k_sum_share<<<1, 256, 0, s>>>(W.epart, agrid, (double)T.m / 3.0, W.shares + t);
    h->n_launches += 3;
    // back-propagation through the three G blocks; Gamma_g is a strided view of dW~
    for (int gi = 0; gi < 3 && e == cudaSuccess; ++gi) {
      int pp, qq, rr;
      if (gi == 0) { pp = T.i; qq = T.j; rr = T.k; }
      else if (gi == 1) { pp = T.j; qq = T.k; rr = T.i; }
      else { pp = T.k; qq = T.i; rr = T.j; }
      // Gamma[x,y,z] strides (gx, gy, gz)
      int64_t gx, gy, gz;
      if (gi == 0) { gx = v2; gy = v; gz = 1; }        // dW~[x,y,z]
      else if (gi == 1) { gx = v; gy = 1; gz = v2; }   // dW~[z,x,y]
      else { gx = 1; gy = v2; gz = v; }                // dW~[y,z,x]
      const double* t2rq = c->t2 + ((int64_t)rr * o + qq) * v2;
      const double* t2rp = c->t2 + ((int64_t)rr * o + pp) * v2;
      auto run = [&](GemmView gv) {
        if (e == cudaSuccess) e = gemm_strided(gv, h->num_sms, W.splitk, splitk_cap(o, v), s, &h->n_launches);
      };
      if (g->ovvv) {
        // (a) dovvv[p,x,y,d] += sum_z G[x,y,z] t2[r,q,z,d]
        run(GemmView{W.dW, t2rq, g->ovvv + (int64_t)pp * v3, v, v, v, v, 1, gx, gy, gz, 0, v, 0, 1, v2, v, 1, 1.0});
        // (b) dovvv[q,y,x,d] += sum_z G[x,y,z] t2[r,p,z,d]
        run(GemmView{W.dW, t2rp, g->ovvv + (int64_t)qq * v3, v, v, v, v, 1, gx, gy, gz, 0, v, 0, 1, v, v2, 1, 1.0});
      }
      if (g->t2) {
        // (c) dt2[r,q,z,d] += sum_xy G[x,y,z] ovvv[p,x,y,d]
        run(GemmView{W.dW, c->ovvv + (int64_t)pp * v3, g->t2 + ((int64_t)rr * o + qq) * v2, v, 1, v, v, v, gz, 0,
                     gx, gy, v2, v, 1, v, 0, 1, 1.0});
        // (d) dt2[r,p,z,d] += sum_xy G[x,y,z] ovvv[q,y,x,d]
        run(GemmView{W.dW, c->ovvv + (int64_t)qq * v3, g->t2 + ((int64_t)rr * o + pp) * v2, v, 1, v, v, v, gz, 0,
                     gx, gy, v, v2, 1, v, 0, 1, 1.0});
        // (e) dt2[l,p,y,x] -= sum_z G[x,y,z] ooov[q,l,r,z]
        run(GemmView{W.dW, c->ooov + ((int64_t)qq * o * o + rr) * v, g->t2 + (int64_t)pp * v2, v, v, o, v, 1, gx,
                     gy, gz, 0, 1, 0, (int64_t)o * v, 1, v, (int64_t)o * v2, -1.0});
        // (g) dt2[l,q,x,y] -= sum_z G[x,y,z] ooov[p,l,r,z]
        run(GemmView{W.dW, c->ooov + ((int64_t)pp * o * o + rr) * v, g->t2 + (int64_t)qq * v2, v, v, o, v, 1, gx,
                     gy, gz, 0, 1, 0, (int64_t)o * v, v, 1, (int64_t)o * v2, -1.0});
      }
      if (g->ooov) {
        // (f) dooov[q,l,r,z] -= sum_xy t2[l,p,y,x] G[x,y,z]
        run(GemmView{c->t2 + (int64_t)pp * v2, W.dW, g->ooov + ((int64_t)qq * o * o + rr) * v, o, 1, v, v, v,
                     (int64_t)o * v2, 0, 1, v, gx, gy, gz, (int64_t)o * v, 0, 1, -1.0});
        // (h) dooov[p,l,r,z] -= sum_xy t2[l,q,x,y] G[x,y,z]
        run(GemmView{c->t2 + (int64_t)qq * v2, W.dW, g->ooov + ((int64_t)pp * o * o + rr) * v, o, 1, v, v, v,
                     (int64_t)o * v2, 0, v, 1, gx, gy, gz, (int64_t)o * v, 0, 1, -1.0});
      }
    }
    if (e != cudaSuccess) break;
    // disconnected term and denominators
    const unsigned gb2 = (unsigned)((v2 + 255) / 256);
    for (int mode = 0; mode < 3; ++mode) {
      if (g->ovov) k_dovs<<<gb2, 256, 0, s>>>(mode, o, v, T.i, T.j, T.k, W.dY, c->t1, W.dOVS);
      if (g->t1) k_dt1<<<(unsigned)v, 256, 0, s>>>(mode, o, v, T.i, T.j, T.k, W.dY, W.ovs, g->t1);
    }
    if (g->eps_v) k_deps_v<<<(unsigned)v, 256, 0, s>>>(v, W.dD, g->eps_v);
    if (g->eps_o) k_deps_o<<<1, 256, 0, s>>>(agrid, W.dpart, T.i, T.j, T.k, g->eps_o);
    h->n_launches += 8;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && g->ovov) {
    k_dovov<<<1024, 256, 0, s>>>(o, v, W.dOVS, g->ovov);
    ++h->n_launches;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && e_out) {
    e = launch_reduce_total(W.shares + t_begin, t_end - t_begin, e_out, s);
    ++h->n_launches;
  }
  if (e != cudaSuccess) return fail(TE_ECUDA, "vjp launch: %s", cudaGetErrorString(e));
  return TE_OK;
}

}  // namespace te

namespace te {

// ---------------------------------------------------------------------------
// the adjoint with the contractions on the tensor cores (exact BF16 slices)
// ---------------------------------------------------------------------------

int64_t oz_scratch_cap(int64_t o, int64_t v, int num_sms) {
  const int64_t splits = std::max<int64_t>((v * v + OZ_KMAX - 1) / OZ_KMAX + 1, 2LL * num_sms);
  return splits * std::max(v * v, o * v);
}

// Slices per element in the exact-slice adjoint: four (28 bits) up to nvir =
// 200, five (35 bits) above.  Its back-contractions sum v (or v^2) products
// whose largest terms can sit far above the result, and the rows of t2 and
// ovvv away from the occupied-virtual boundary far below their scale; at
// nocc=48 nvir=560 four slices left errors of 2.7e-6 of d ovvv's largest entry.
static int adjoint_slices(int64_t v) { return v > 200 ? 5 : 4; }

// ---------------------------------------------------------------------------
// exact-slice adjoint on tcgen05 (view_tc.cu)
// ---------------------------------------------------------------------------

// Slices of three index permutations of dW~ into three layouts L[x][y][z]
// (z padded to vp), layout b of phase f holding the slices of dW~[pi(x, y, z)]:
//   phase 0: pi = (x,y,z), (z,x,y), (y,z,x);  phase 1: (z,y,x), (x,z,y), (y,x,z).
// With 2^e > max |dW~| (e written to *e_out), the slices are slice_digits'
// (integer arithmetic on the bits of dW~, no float64 operations).  A block handles one
// 32 x 32 tile of the (c, z) plane at one value of the third index, c being
// the index along which dW~ is contiguous for this permutation (or y when that
// is z), so both the reads and the writes are coalesced.
template <int NS>
__global__ void __launch_bounds__(256) k_dw_layouts(const double* __restrict__ dW, int v, int vp, int phase,
                                                    const unsigned long long* __restrict__ dwmax,
                                                    int* __restrict__ e_out, __nv_bfloat16* __restrict__ out,
                                                    int64_t lay_elems) {
  __shared__ double tile[32][33];
  const double mx = __longlong_as_double((long long)*dwmax);
  int ex = 0;
  if (mx > 0.0) frexp(mx, &ex);
  if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 && threadIdx.y == 0) *e_out = ex;
  const int perm = phase * 3 + (int)blockIdx.z;
  const int64_t V = v, V2 = V * V, plane = V2 * vp;
  // source strides of the output indices (x, y, z)
  int64_t sx, sy, sz;
  switch (perm) {
    case 0: sx = V2; sy = V; sz = 1; break;
    case 1: sx = V; sy = 1; sz = V2; break;
    case 2: sx = 1; sy = V2; sz = V; break;
    case 3: sx = 1; sy = V; sz = V2; break;
    case 4: sx = V2; sy = 1; sz = V; break;
    default: sx = V; sy = V2; sz = 1; break;
  }
  // c: the tile's other index (0 = x, 1 = y); w: the block's fixed index
  const int cidx = (sx == 1) ? 0 : 1;
  const int64_t sc_ = cidx == 0 ? sx : sy, sw = cidx == 0 ? sy : sx;
  const int ntz = (v + 31) / 32;
  const int c0 = (int)(blockIdx.x / ntz) * 32, z0 = (int)(blockIdx.x % ntz) * 32;
  const int w = blockIdx.y;
  const int tx = threadIdx.x, ty = threadIdx.y;
  // load: threads along c when dW~ is contiguous along c, else along z
  for (int i = ty; i < 32; i += 8) {
    const int cc = sz == 1 ? c0 + i : c0 + tx, zz = sz == 1 ? z0 + tx : z0 + i;
    if (cc < v && zz < v) {
      const double x = dW[w * sw + cc * sc_ + zz * sz];
      if (sz == 1) tile[i][tx] = x;
      else tile[tx][i] = x;
    }
  }
  __syncthreads();
  __nv_bfloat16* o = out + blockIdx.z * lay_elems;
  for (int i = ty; i < 32; i += 8) {
    const int cc = c0 + i, zz = z0 + tx;
    if (cc >= v || zz >= v) continue;
    float d[NS];
    slice_digits<NS>(tile[i][tx], ex, d);
    const int64_t xi = cidx == 0 ? cc : w, yi = cidx == 0 ? w : cc;
    const int64_t at = (xi * V + yi) * vp + zz;
#pragma unroll
    for (int k = 0; k < NS; ++k) o[k * plane + at] = __float2bfloat16_rn(ldexpf(d[k], -7 * (k + 1)));
  }
}

static int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

struct VjpTcSizes {
  int ns, vp;
  size_t lay;         // elements of one dW~ layout (ns planes of v v vp)
  size_t region;      // bytes: G, dY and dD, later the three layouts
  size_t ovt, t2t, t2p, noo;  // bytes of the operand copies
  int64_t part_cap;   // doubles of split-K partials
};

static VjpTcSizes vjp_tc_sizes(int64_t o, int64_t v, int num_sms) {
  VjpTcSizes z;
  z.ns = adjoint_slices(v);
  z.vp = (int)rup(v, 16);
  const int64_t v3 = v * v * v, vp = z.vp, NS = z.ns;
  auto a = [](size_t b) { return (b + 1023) & ~size_t(1023); };
  z.lay = (size_t)NS * v * v * vp;
  z.region = std::max(a((size_t)3 * v3 * 8) + 2 * a((size_t)v3 * 8), 3 * a(z.lay * 2));
  z.ovt = a((size_t)NS * v * v * vp * 2);
  z.t2t = a((size_t)6 * NS * v * vp * 2);
  z.t2p = a((size_t)3 * NS * o * v * vp * 2);
  z.noo = a((size_t)NS * o * o * o * vp * 2);
  // partials of the split jobs of one launch (an upper bound over the launches)
  const int64_t ntv = vt_ntile(v), nto = vt_ntile(o);
  const int64_t rows_xy = ((v + 7) / 8) * ((v + 15) / 16), rows_z = (v + 127) / 128;
  const int64_t pair_blk = 3 * vt_seg_blocks((int)v, (int)v, VT_SPLIT_CHUNKS);
  const int64_t one_blk = 4 * vt_seg_blocks(1, (int)v, VT_SPLIT_CHUNKS);
  const int64_t d_ovvv = vt_split_doubles(rows_xy * ((v + ntv - 1) / ntv), one_blk, v * v * v, num_sms);
  const int64_t d_t2s = vt_split_doubles(rows_xy * ((o + nto - 1) / nto), one_blk, v * v * o, num_sms);
  const int64_t d_ooov = vt_split_doubles(rows_z * ((o + nto - 1) / nto), pair_blk, v * o, num_sms);
  const int64_t d_t2 = vt_split_doubles(rows_z * ((v + ntv - 1) / ntv), pair_blk, v * v, num_sms);
  z.part_cap = std::max(3 * (d_ovvv + d_t2s + d_ooov), 3 * (d_t2 + d_ooov)) + 1024;
  return z;
}

size_t vjp_tc_bytes(int64_t o, int64_t v, int num_sms) {
  const int64_t v3 = v * v * v, nt = num_unique_triples(o);
  const int64_t nblk = std::max<int64_t>((v3 + 255) / 256, 8192);  // at least adjoint_grid's largest
  const VjpTcSizes z = vjp_tc_sizes(o, v, num_sms);
  auto a = [](int64_t n) { return ((size_t)n * 8 + 1023) & ~size_t(1023); };
  return tc_slices_bytes((int)o, (int)v, z.ns) + 1024 + a(o * v * o * v) + z.region + a(v3) + a(o * v * o * v) +
         2 * a(nblk) + a(std::max<int64_t>(1, nt)) + a(4) + z.ovt + z.t2t + z.t2p + z.noo + a(z.part_cap) + 4096;
}

// The contractions of one triple (g = 0, 1, 2 the G blocks with occupied
// indices (p, q, r) = (i, j, k), (j, k, i), (k, i, j); dG_g the views of dW~):
//   G:  G_g[x,y,z] = S1 + S2 + S3 + S4 (four K segments, the forward's form)
//   (a) dovvv[p,x,y,d] += sum_z dG[x,y,z] t2[r,q,z,d]    (b) dovvv[q,y,x,d] += sum_z dG[x,y,z] t2[r,p,z,d]
//   (c) dt2[r,q,z,d] += sum_xy dG[x,y,z] ovvv[p,x,y,d]   (d) dt2[r,p,z,d] += sum_xy dG[x,y,z] ovvv[q,y,x,d]
//   (e) dt2[l,p,y,x] -= sum_z dG[x,y,z] ooov[q,l,r,z]    (g) dt2[l,q,x,y] -= sum_z dG[x,y,z] ooov[p,l,r,z]
//   (f) dooov[q,l,r,z] -= sum_xy t2[l,p,y,x] dG[x,y,z]   (h) dooov[p,l,r,z] -= sum_xy t2[l,q,x,y] dG[x,y,z]
// Every operand is read along a contiguous K index: dG_g comes in the layouts
// L1_g[x][y][z] (K = z), L2_g[z][x][y] (K = (x, y)) and L3_g[z][y][x] (K =
// (y, x)), the index permutations of dW~ that k_dw_layouts writes; t2, ovvv
// and ooov enter as transposed slice copies (t2T[d][z] per pair (r, q),
// ovvvT[d][x][y] per slab, t2P[l][x][y] per occupied index, nooTT[q][r][l][z]).
// Outputs of the same launch are disjoint: the contributions to one output
// slab (or pair block) are the segments of one job.
te_status run_vjp_tc(Handle* h, const te_cluster* c, int64_t t_begin, int64_t t_end, double gE,
                     double* e_out, te_cluster_grad* g, cudaStream_t s) {
  const int o = (int)c->nocc, v = (int)c->nvir;
  const int64_t v2 = (int64_t)v * v, v3 = v2 * v, nt = num_unique_triples(o);
  te_status st = ensure_workspace_public(h, vjp_tc_bytes(o, v, h->num_sms));
  if (st != TE_OK) return st;
  st = ensure_triples_public(h, o);
  if (st != TE_OK) return st;
  const VjpTcSizes Z = vjp_tc_sizes(o, v, h->num_sms);
  const int ns = Z.ns;
  const int64_t vp = Z.vp;
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(h->ws) + 1023) & ~uintptr_t(1023));
  SliceSet S;
  st = tc_prepare_slices(c, base, &S, h->num_sms, s, ns);
  if (st != TE_OK) return st;
  char* p = base + ((tc_slices_bytes(o, v, ns) + 1023) & ~size_t(1023));
  auto takeb = [&](size_t bytes) {
    char* r = p;
    p += (bytes + 1023) & ~size_t(1023);
    return r;
  };
  auto take = [&](int64_t n) { return reinterpret_cast<double*>(takeb((size_t)n * 8)); };
  VjpWork W;
  W.t2L = nullptr;
  W.nooT = nullptr;
  W.ovs = take((int64_t)o * v * o * v);
  char* region = takeb(Z.region);
  W.G = reinterpret_cast<double*>(region);
  W.dY = reinterpret_cast<double*>(region + (((size_t)3 * v3 * 8 + 1023) & ~size_t(1023)));
  W.dD = W.dY + ((((size_t)v3 * 8 + 1023) & ~size_t(1023)) / 8);
  W.dW = take(v3);
  W.dOVS = take((int64_t)o * v * o * v);
  const int64_t nblk = std::max<int64_t>((v3 + 255) / 256, adjoint_grid(h->num_sms));
  const int64_t agrid = adjoint_grid(h->num_sms);
  W.epart = take(nblk);
  W.dpart = take(nblk);
  W.shares = take(std::max<int64_t>(1, nt));
  unsigned long long* dwmax = reinterpret_cast<unsigned long long*>(take(4));
  int* dwexp = reinterpret_cast<int*>(dwmax + 1);
  using bf = __nv_bfloat16;
  bf* ovT = reinterpret_cast<bf*>(takeb(Z.ovt));
  bf* t2T = reinterpret_cast<bf*>(takeb(Z.t2t));
  bf* t2P = reinterpret_cast<bf*>(takeb(Z.t2p));
  bf* nooTT = reinterpret_cast<bf*>(takeb(Z.noo));
  double* part = take(Z.part_cap);
  const size_t lay_stride = ((Z.lay * 2 + 1023) & ~size_t(1023)) / 2;  // elements between layouts
  bf* lay = reinterpret_cast<bf*>(region);

  auto zero = [&](double* ptr, int64_t n) {
    return ptr ? cudaMemsetAsync(ptr, 0, sizeof(double) * n, s) : cudaSuccess;
  };
  cudaError_t e = cudaSuccess;
  e = e ? e : zero(g->eps_o, o);
  e = e ? e : zero(g->eps_v, v);
  e = e ? e : zero(g->ovvv, (int64_t)o * v3);
  e = e ? e : zero(g->ooov, (int64_t)o * o * o * v);
  e = e ? e : zero(g->ovov, (int64_t)o * v * o * v);
  e = e ? e : zero(g->t1, (int64_t)o * v);
  e = e ? e : zero(g->t2, (int64_t)o * o * v2);
  e = e ? e : zero(W.dOVS, (int64_t)o * v * o * v);
  if (e != cudaSuccess) return fail(TE_ECUDA, "memset: %s", cudaGetErrorString(e));

  Prepared P{};  // float64 ovs for the disconnected term
  P.o = o;
  P.v = v;
  P.eps_o = c->eps_o;
  P.eps_v = c->eps_v;
  P.ovvv = c->ovvv;
  P.t2 = c->t2;
  P.t1 = c->t1;
  P.t2L = W.t2L;
  P.nooT = W.nooT;
  P.ovs = W.ovs;
  e = launch_prep_fp64(c, &P, s);
  if (e != cudaSuccess) return fail(TE_ECUDA, "prep: %s", cudaGetErrorString(e));

  const bf* sO = static_cast<const bf*>(S.ovvv);
  const bf* sT = static_cast<const bf*>(S.t2);
  const bf* sL = static_cast<const bf*>(S.t2L);
  const bf* sN = static_cast<const bf*>(S.nooT);
  const int64_t op = S.op, O = o, V = v, NS = ns;
  // nooTT[q][r][l][z] = nooT[q][r][z][l] = -ooov[q,l,r,z], once per call
  e = vt_transpose(sN, S.nooT_plane, S.nooT_pr, op, nooTT, O * O * O * vp, O * vp, vp, ns, o * o, v, o, s);
  if (e != cudaSuccess) return fail(TE_ECUDA, "transpose: %s", cudaGetErrorString(e));
  ++h->n_launches;

  // tensor maps, encoded once: rows (x, y) in tiles of 8 x 16, rows z alone in tiles of 128
  const int NTv = vt_ntile(v), NTo = vt_ntile(o);
  VtBank bank;
  bank.n = 0;
  auto add = [&](const void* b0, std::initializer_list<int64_t> dims, std::initializer_list<int64_t> str,
                 VtRoles r, int rows2, int rows1, int* idx) {
    VtView w;
    w.base = b0;
    int q = 0;
    for (int64_t d : dims) w.dims[q++] = (uint64_t)d;
    q = 0;
    for (int64_t x : str) w.stride[q++] = (uint64_t)x;
    w.roles = r;
    return vt_bank_add(&bank, w, rows2, rows1, idx);
  };
  const VtRoles XY{0, 1, 2, -1, 3};       // k2 | rows y, x | slice
  const VtRoles ROW{0, 1, -1, -1, 2};     // k2 | rows | slice
  const VtRoles ZK{0, 2, -1, 1, 3};       // k2 | k1 | rows | slice
  int m_g[6], m_l1n[3], m_l1t[3], m_lz[3], m_t2T, m_noo, m_ovT, m_t2P;
  const int64_t U1 = 1;
  if ((st = vt_slice_maps(&bank, S, o, v, NTv, m_g)) != TE_OK) return st;
  const int m_on = m_g[0], m_ot = m_g[1], m_ln = m_g[2], m_lt = m_g[3], m_t2 = m_g[4], m_no = m_g[5];
  const int64_t lplane = V * V * vp;
  for (int b = 0; b < 3; ++b) {
    const bf* lb = lay + b * lay_stride;
    if ((st = add(lb, {U1 * v, U1 * v, U1 * v, U1 * NS, 1}, {1, U1 * vp, V * vp, lplane, 0}, XY, 16, 8,
                  &m_l1n[b])) != TE_OK)
      return st;
    if ((st = add(lb, {U1 * v, U1 * v, U1 * v, U1 * NS, 1}, {1, V * vp, U1 * vp, lplane, 0}, XY, 16, 8,
                  &m_l1t[b])) != TE_OK)
      return st;
    if ((st = add(lb, {U1 * v, U1 * v, U1 * v, U1 * NS, 1}, {1, U1 * vp, V * vp, lplane, 0}, ZK, 128, 1,
                  &m_lz[b])) != TE_OK)
      return st;
  }
  if ((st = add(t2T, {U1 * v, U1 * v, U1 * NS, 6, 1}, {1, U1 * vp, V * vp, NS * V * vp, 0}, ROW, NTv, 1, &m_t2T)) !=
      TE_OK)
    return st;
  if ((st = add(nooTT, {U1 * v, U1 * O, U1 * O, U1 * O, U1 * NS}, {1, U1 * vp, O * vp, O * O * vp, O * O * O * vp},
                VtRoles{0, 1, -1, -1, 4}, NTo, 1, &m_noo)) != TE_OK)
    return st;
  if ((st = add(ovT, {U1 * v, U1 * v, U1 * v, U1 * NS, 1}, {1, U1 * vp, V * vp, V * V * vp, 0}, ZK, NTv, 1,
                &m_ovT)) != TE_OK)
    return st;
  if ((st = add(t2P, {U1 * v, U1 * v, U1 * O, U1 * NS, 3}, {1, U1 * vp, V * vp, O * V * vp, NS * O * V * vp}, ZK,
                NTo, 1, &m_t2P)) != TE_OK)
    return st;
  // layout buffers: phase 0 holds L1_g in buffer g and L2_g in buffer (g + 2) % 3; phase 1 holds L3_g in buffer g
  const int l2buf[3] = {2, 0, 1};

  auto eO = [&](int p_) { return S.e_ovvv + p_; };
  auto eT = [&](int r_, int q_) { return S.e_t2 + ((int64_t)r_ * o + q_); };
  auto eL = [&](int q_) { return S.e_t2L + q_; };
  auto eN = [&](int p_, int r_) { return S.e_nooT + ((int64_t)p_ * o + r_); };

  std::vector<Triple> trip = unique_triples(o);
  int slab = -1;  // the ovvv slab whose transpose ovT holds
  auto launch = [&](VtBuild& b) -> te_status {
    te_status q = vt_finish(&b, h->num_sms, part, Z.part_cap, nullptr);
    if (q != TE_OK) return q;
    return vt_launch(h, &b, s);
  };
  auto need_slab = [&](int sb) -> cudaError_t {
    if (slab == sb) return cudaSuccess;
    slab = sb;
    ++h->n_launches;
    return vt_transpose(sO + (int64_t)sb * S.ovvv_p, S.ovvv_plane, V * vp, vp, ovT, V * V * vp, vp, V * vp, ns, v, v,
                        v, s);
  };
  for (int64_t t = t_begin; t < t_end; ++t) {
    const Triple T = trip[t];
    const int PQR[3][3] = {{T.i, T.j, T.k}, {T.j, T.k, T.i}, {T.k, T.i, T.j}};
    // t2T slots: the (r, q) pairs the (a) and (b) contractions read
    int pr[6][2], npair = 0;
    auto pair_slot = [&](int r_, int q_) {
      for (int x = 0; x < npair; ++x)
        if (pr[x][0] == r_ && pr[x][1] == q_) return x;
      pr[npair][0] = r_;
      pr[npair][1] = q_;
      return npair++;
    };
    int sl_rq[3], sl_rp[3];
    for (int gi = 0; gi < 3; ++gi) {
      sl_rq[gi] = pair_slot(PQR[gi][2], PQR[gi][1]);
      sl_rp[gi] = pair_slot(PQR[gi][2], PQR[gi][0]);
    }
    // t2P slots: the distinct occupied indices of the triple
    int occ[3], nocc_ = 0;
    auto occ_slot = [&](int x_) {
      for (int q = 0; q < nocc_; ++q)
        if (occ[q] == x_) return q;
      occ[nocc_] = x_;
      return nocc_++;
    };
    occ_slot(T.i);
    occ_slot(T.j);
    occ_slot(T.k);
    for (int x = 0; x < npair && e == cudaSuccess; ++x)
      e = vt_transpose(sT + ((int64_t)pr[x][0] * o + pr[x][1]) * S.t2_rq, S.t2_plane, 0, vp, t2T + x * NS * V * vp,
                       V * vp, 0, vp, ns, 1, v, v, s);
    for (int x = 0; x < nocc_ && e == cudaSuccess; ++x)
      e = vt_transpose(sL + (int64_t)occ[x] * S.t2L_q, S.t2L_plane, V * op, op, t2P + x * NS * O * V * vp, O * V * vp,
                       vp, V * vp, ns, v, v, o, s);
    h->n_launches += npair + nocc_;
    if (e != cudaSuccess) break;

    // forward G blocks, float64 [g][x][y][z]
    {
      VtBuild b;
      vt_begin(&b, ns);
      for (int gi = 0; gi < 3; ++gi) {
        const int pp = PQR[gi][0], qq = PQR[gi][1], rr = PQR[gi][2];
        VtJob* J = vt_job(&b, v, v, v, 8, 16, NTv, W.G + gi * v3, v2, v, 1, 1);
        const int f_p[5] = {0, 0, 0, 0, pp}, f_q[5] = {0, 0, 0, 0, qq};
        const int t_qr[5] = {0, 0, 0, qq, rr}, t_pr[5] = {0, 0, 0, pp, rr};
        const int n_rq[5] = {0, 0, 0, rr, qq}, n_rp[5] = {0, 0, 0, rr, pp};
        vt_seg(J, vt_use(&b, bank, m_on), vt_use(&b, bank, m_t2), 1, v, f_p, t_qr, eO(pp), eT(rr, qq), 1.0);
        vt_seg(J, vt_use(&b, bank, m_ot), vt_use(&b, bank, m_t2), 1, v, f_q, t_pr, eO(qq), eT(rr, pp), 1.0);
        vt_seg(J, vt_use(&b, bank, m_lt), vt_use(&b, bank, m_no), 1, o, f_p, n_rq, eL(pp), eN(qq, rr), 1.0);
        vt_seg(J, vt_use(&b, bank, m_ln), vt_use(&b, bank, m_no), 1, o, f_q, n_rp, eL(qq), eN(pp, rr), 1.0);
      }
      if ((st = launch(b)) != TE_OK) return st;
    }
    AdjArgs A{};  // value-initialised: optional pointers (dwmax) are null unless set
    A.o = o; A.v = v; A.i = T.i; A.j = T.j; A.k = T.k;
    A.w = gE * (double)T.m / 3.0;
    A.G = W.G; A.ovs = W.ovs; A.t1 = c->t1; A.eps_o = c->eps_o; A.eps_v = c->eps_v;
    A.dW = W.dW; A.dY = W.dY; A.dD = W.dD; A.epart = W.epart; A.dpart = W.dpart; A.dwmax = dwmax;
    cudaMemsetAsync(dwmax, 0, 8, s);
    k_adjoint<<<(unsigned)agrid, 256, 0, s>>>(A);
    k_sum_share<<<1, 256, 0, s>>>(W.epart, agrid, (double)T.m / 3.0, W.shares + t);
    // the Y and denominator parts; G, dY and dD are dead afterwards and their
    // memory takes the dW~ layouts
    const unsigned gb2 = (unsigned)((v2 + 255) / 256);
    for (int mode = 0; mode < 3; ++mode) {
      if (g->ovov) k_dovs<<<gb2, 256, 0, s>>>(mode, o, v, T.i, T.j, T.k, W.dY, c->t1, W.dOVS);
      if (g->t1) k_dt1<<<(unsigned)v, 256, 0, s>>>(mode, o, v, T.i, T.j, T.k, W.dY, W.ovs, g->t1);
    }
    if (g->eps_v) k_deps_v<<<(unsigned)v, 256, 0, s>>>(v, W.dD, g->eps_v);
    if (g->eps_o) k_deps_o<<<1, 256, 0, s>>>(agrid, W.dpart, T.i, T.j, T.k, g->eps_o);
    const int nt32 = (v + 31) / 32;
    const dim3 lgrid((unsigned)(nt32 * nt32), (unsigned)v, 3), lblk(32, 8);
    if (ns == 5) k_dw_layouts<5><<<lgrid, lblk, 0, s>>>(W.dW, v, (int)vp, 0, dwmax, dwexp, lay, (int64_t)lay_stride);
    else k_dw_layouts<4><<<lgrid, lblk, 0, s>>>(W.dW, v, (int)vp, 0, dwmax, dwexp, lay, (int64_t)lay_stride);
    h->n_launches += 11;
    if ((e = cudaGetLastError()) != cudaSuccess) break;

    // d ovvv (a, b), d t2 slabs from ooov (e, g), d ooov (h): layouts L1, L2
    {
      VtBuild b;
      vt_begin(&b, ns);
      int dist[3], nd = 0;
      for (int x_ : {T.i, T.j, T.k}) {
        bool seen = false;
        for (int q = 0; q < nd; ++q) seen |= dist[q] == x_;
        if (!seen) dist[nd++] = x_;
      }
      for (int q = 0; q < nd && g->ovvv; ++q) {
        const int sb = dist[q];
        VtJob* J = vt_job(&b, v, v, v, 8, 16, NTv, g->ovvv + (int64_t)sb * v3, v2, v, 1, 0);
        for (int gi = 0; gi < 3; ++gi) {
          const int pp = PQR[gi][0], qq = PQR[gi][1], rr = PQR[gi][2];
          const int f_rq[5] = {0, 0, 0, sl_rq[gi], 0}, f_rp[5] = {0, 0, 0, sl_rp[gi], 0};
          if (pp == sb) vt_seg(J, vt_use(&b, bank, m_l1n[gi]), vt_use(&b, bank, m_t2T), 1, v, nullptr, f_rq, dwexp,
                               eT(rr, qq), 1.0);
          if (qq == sb) vt_seg(J, vt_use(&b, bank, m_l1t[gi]), vt_use(&b, bank, m_t2T), 1, v, nullptr, f_rp, dwexp,
                               eT(rr, pp), 1.0);
        }
      }
      for (int q = 0; q < nd && g->t2; ++q) {
        const int sb = dist[q];
        // element dt2[l][sb][X][Y]: rows (X, Y), columns l
        VtJob* J = vt_job(&b, v, v, o, 8, 16, NTo, g->t2 + (int64_t)sb * v2, v, 1, (int64_t)o * v2, 0);
        for (int gi = 0; gi < 3; ++gi) {
          const int pp = PQR[gi][0], qq = PQR[gi][1], rr = PQR[gi][2];
          const int f_rq[5] = {0, 0, rr, qq, 0}, f_rp[5] = {0, 0, rr, pp, 0};
          // (e): X = y, Y = x: transposed rows; B = nooTT = -ooov
          if (pp == sb) vt_seg(J, vt_use(&b, bank, m_l1t[gi]), vt_use(&b, bank, m_noo), 1, v, nullptr, f_rq, dwexp,
                               eN(qq, rr), 1.0);
          if (qq == sb) vt_seg(J, vt_use(&b, bank, m_l1n[gi]), vt_use(&b, bank, m_noo), 1, v, nullptr, f_rp, dwexp,
                               eN(pp, rr), 1.0);
        }
      }
      if (g->ooov) {
        bool done[3] = {false, false, false};
        for (int gi = 0; gi < 3; ++gi) {
          if (done[gi]) continue;
          const int P_ = PQR[gi][0], R_ = PQR[gi][2];
          VtJob* J = vt_job(&b, 1, v, o, 1, 128, NTo, g->ooov + ((int64_t)P_ * o * o + R_) * v, 0, 1, (int64_t)o * v, 0);
          for (int g2 = gi; g2 < 3; ++g2) {
            if (done[g2] || PQR[g2][0] != P_ || PQR[g2][2] != R_) continue;
            done[g2] = true;
            const int f_q[5] = {0, 0, 0, 0, occ_slot(PQR[g2][1])};
            vt_seg(J, vt_use(&b, bank, m_lz[l2buf[g2]]), vt_use(&b, bank, m_t2P), v, v, nullptr, f_q, dwexp,
                   eL(PQR[g2][1]), -1.0);
          }
        }
      }
      if (b.P.njobs && (st = launch(b)) != TE_OK) return st;
    }
    // d t2 pair blocks from ovvv (c): layouts L2, one slab transpose per launch
    const int order[3] = {T.i, T.j, T.k};
    for (int q = 0; q < 3 && g->t2; ++q) {
      const int sb = order[q];
      if ((q == 1 && sb == order[0]) || (q == 2 && (sb == order[0] || sb == order[1]))) continue;
      VtBuild b;
      vt_begin(&b, ns);
      bool done[3] = {false, false, false};
      for (int gi = 0; gi < 3; ++gi) {
        if (done[gi] || PQR[gi][0] != sb) continue;
        const int R_ = PQR[gi][2], Q_ = PQR[gi][1];
        VtJob* J = vt_job(&b, 1, v, v, 1, 128, NTv, g->t2 + ((int64_t)R_ * o + Q_) * v2, 0, v, 1, 0);
        for (int g2 = gi; g2 < 3; ++g2) {
          if (done[g2] || PQR[g2][0] != sb || PQR[g2][2] != R_ || PQR[g2][1] != Q_) continue;
          done[g2] = true;
          vt_seg(J, vt_use(&b, bank, m_lz[l2buf[g2]]), vt_use(&b, bank, m_ovT), v, v, nullptr, nullptr, dwexp, eO(sb),
                 1.0);
        }
      }
      if (!b.P.njobs) continue;
      if ((e = need_slab(sb)) != cudaSuccess) break;
      if ((st = launch(b)) != TE_OK) return st;
    }
    if (e != cudaSuccess) break;
    // phase 1 layouts: L3_g
    if (ns == 5) k_dw_layouts<5><<<lgrid, lblk, 0, s>>>(W.dW, v, (int)vp, 1, dwmax, dwexp, lay, (int64_t)lay_stride);
    else k_dw_layouts<4><<<lgrid, lblk, 0, s>>>(W.dW, v, (int)vp, 1, dwmax, dwexp, lay, (int64_t)lay_stride);
    ++h->n_launches;
    // d t2 pair blocks from ovvv (d), slabs in reverse order (the last slab of
    // (c) is still transposed), and d ooov (f) in the first launch: layouts L3
    bool first = true;
    for (int q = 2; q >= 0; --q) {
      const int sb = order[q];
      if ((q == 1 && sb == order[2]) || (q == 0 && (sb == order[2] || sb == order[1]))) continue;
      VtBuild b;
      vt_begin(&b, ns);
      bool done[3] = {false, false, false};
      for (int gi = 0; gi < 3 && g->t2; ++gi) {
        if (done[gi] || PQR[gi][1] != sb) continue;
        const int R_ = PQR[gi][2], P_ = PQR[gi][0];
        VtJob* J = vt_job(&b, 1, v, v, 1, 128, NTv, g->t2 + ((int64_t)R_ * o + P_) * v2, 0, v, 1, 0);
        for (int g2 = gi; g2 < 3; ++g2) {
          if (done[g2] || PQR[g2][1] != sb || PQR[g2][2] != R_ || PQR[g2][0] != P_) continue;
          done[g2] = true;
          vt_seg(J, vt_use(&b, bank, m_lz[g2]), vt_use(&b, bank, m_ovT), v, v, nullptr, nullptr, dwexp, eO(sb), 1.0);
        }
      }
      const bool need = b.P.njobs > 0;
      if (first && g->ooov) {
        bool done2[3] = {false, false, false};
        for (int gi = 0; gi < 3; ++gi) {
          if (done2[gi]) continue;
          const int Q_ = PQR[gi][1], R_ = PQR[gi][2];
          VtJob* J = vt_job(&b, 1, v, o, 1, 128, NTo, g->ooov + ((int64_t)Q_ * o * o + R_) * v, 0, 1, (int64_t)o * v, 0);
          for (int g2 = gi; g2 < 3; ++g2) {
            if (done2[g2] || PQR[g2][1] != Q_ || PQR[g2][2] != R_) continue;
            done2[g2] = true;
            const int f_p[5] = {0, 0, 0, 0, occ_slot(PQR[g2][0])};
            vt_seg(J, vt_use(&b, bank, m_lz[g2]), vt_use(&b, bank, m_t2P), v, v, nullptr, f_p, dwexp,
                   eL(PQR[g2][0]), -1.0);
          }
        }
      }
      first = false;
      if (!b.P.njobs) continue;
      if (need && (e = need_slab(sb)) != cudaSuccess) break;
      if ((st = launch(b)) != TE_OK) return st;
    }
    if (e != cudaSuccess) break;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && g->ovov) {
    k_dovov<<<1024, 256, 0, s>>>(o, v, W.dOVS, g->ovov);
    ++h->n_launches;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && e_out) {
    e = launch_reduce_total(W.shares + t_begin, t_end - t_begin, e_out, s);
    ++h->n_launches;
  }
  if (e != cudaSuccess) return fail(TE_ECUDA, "vjp launch: %s", cudaGetErrorString(e));
  return TE_OK;
}

}  // namespace te
