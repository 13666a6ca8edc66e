// Tensor-core path (TF32, BF16x3, TF32x3, OZAKI) for the W~ contractions.
//
// The same three G blocks as the float64 path (see gemm_fp64.cu):
//   W~_{ijk}[a,b,c] = G(i,j,k)[a,b,c] + G(j,k,i)[b,c,a] + G(k,i,j)[c,a,b]
// each one GEMM  D[(x,y), z] = sum_K A[(x,y), K] B[z, K]  with four K segments
//   S1 ovvv[p,x,y,:] . t2[r,q,z,:]     S2 ovvv[q,y,x,:] . t2[r,p,z,:]
//   S3 t2L[p,y,x,:] . nooT[q,r,z,:]    S4 t2L[q,x,y,:] . nooT[p,r,z,:]
// run on tcgen05: TMA brings 128-row A tiles (TA values of x times TB of y)
// and NT-row B tiles into swizzled shared memory; one thread issues
// tcgen05.mma into FP32 accumulators in tensor memory; four epilogue warps
// drain TMEM into the G buffer.
//
// Operand forms, prepared once per call:
//  * TF32, BF16X3, TF32X3: x = hi + lo, hi and lo the nearest 11-bit (TF32)
//    or 8-bit (BF16) significands (Veltkamp splitting); the products
//    hi*hi + hi*lo + lo*hi (hi*hi only for TF32) share one accumulator.
//  * OZAKI (Ozaki, Ogita, Oishi, Rump 2012, error-free slicing): each array
//    is scaled by 2^-s (s from its largest magnitude, chosen so that every
//    segment of the K axis has the same unit) and cut into four slices
//    m_k 2^-7k, |m_k| <= 128, exact in BF16.  Slice products are then exact
//    multiples of 2^-7(k+l); the level-2 product and the two level-3
//    products each go to their own accumulator, where every partial sum is
//    an integer multiple of the level's unit below 2^24 units - exact, so the
//    tensor core's FP32 accumulation cannot round them.  The seven products
//    of levels 4 and 5 share a third accumulator.  The epilogue adds the
//    three with an exact two-sum and stores G as an FP32 pair (hi, lo).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <cstring>

#include "energy_tc.h"
#include "ptx_sm100.cuh"
#include "strided.h"
#include "tc_path.h"

namespace te {

// TC_OZAKI: four 7-bit slices, ten slice products (K = 2 (v + o) <= 1024).
// TC_OZAKI6: five 6-bit slices, fifteen slice products (K <= 4096); chosen
// for the same user mode when the K axis is too long for 7-bit slices.
// TC_SLICE4, TC_SLICE5: four or five 7-bit slices, the operand form of the
// strided exact-slice GEMMs (no contraction kernel of their own), cut from the
// integer N = round(x 2^(7 NS - s)) in balanced base-128 digits.
enum TcMode { TC_TF32 = 0, TC_BF16X3 = 1, TC_TF32X3 = 2, TC_OZAKI = 3, TC_OZAKI6 = 4, TC_SLICE5 = 5, TC_SLICE4 = 6 };

constexpr int OZ_K_MAX7 = 1024;  // K * 2^14 < 2^24: exact level-2/3 sums with 7-bit slices
constexpr int OZ_K_MAX6 = 4096;  // K * 2^12 < 2^24 with 6-bit slices

// ozaki_bits: 0 = 7-bit slices when K allows, else 6-bit; 6 or 7 forces one.
static int tc_mode_of(te_precision p, int o, int v, int ozaki_bits) {
  switch (p) {
    case TE_TF32: return TC_TF32;
    case TE_BF16X3: return TC_BF16X3;
    case TE_TF32X3: return TC_TF32X3;
    default:
      if (ozaki_bits == 6) return TC_OZAKI6;
      if (ozaki_bits == 7) return TC_OZAKI;
      return 2 * (v + o) <= OZ_K_MAX7 ? TC_OZAKI : TC_OZAKI6;
  }
}

__host__ __device__ constexpr bool is_ozaki(int mode) {
  return mode == TC_OZAKI || mode == TC_OZAKI6 || mode == TC_SLICE5 || mode == TC_SLICE4;
}

template <int MODE>
struct ModeTraits {
  static constexpr bool tf32 = (MODE == TC_TF32 || MODE == TC_TF32X3);
  static constexpr int nparts =
      (MODE == TC_TF32) ? 1
                        : ((MODE == TC_OZAKI || MODE == TC_SLICE4) ? 4 : ((MODE == TC_OZAKI6 || MODE == TC_SLICE5) ? 5 : 2));
  static constexpr int nacc = is_ozaki(MODE) ? 3 : 1;   // accumulators per tile
  static constexpr int beta = MODE == TC_OZAKI6 ? 6 : 7;  // bits per slice
};

constexpr int MAX_PARTS = 5;

// ---------------------------------------------------------------------------
// operand preparation
// ---------------------------------------------------------------------------

// Round x to the nearest value with `bits` significant bits (Veltkamp split).
// __dmul_rn / __dsub_rn keep the compiler from contracting into an FMA.
template <int BITS>
__device__ __forceinline__ double round_sig(double x) {
  const double c = __dmul_rn(x, (double)((1ull << (53 - BITS)) + 1ull));
  return __dsub_rn(c, __dsub_rn(c, x));
}

struct Parts {
  void* p[MAX_PARTS];
};

// Element `idx` of every part plane.  For OZAKI, `scale` is 2^-s of the array.
template <int MODE>
__device__ __forceinline__ void split_store(double x, const Parts& parts, int64_t idx, double scale) {
  if (MODE == TC_BF16X3) {
    const double h = round_sig<8>(x);
    const double l = round_sig<8>(x - h);
    reinterpret_cast<__nv_bfloat16*>(parts.p[0])[idx] = __float2bfloat16_rn((float)h);
    reinterpret_cast<__nv_bfloat16*>(parts.p[1])[idx] = __float2bfloat16_rn((float)l);
  } else if (MODE == TC_SLICE4 || MODE == TC_SLICE5) {
    // integer digits of x 2^-s (slice_digits): no float64 arithmetic, against
    // five float64 operations per slice for the repeated rounding below
    constexpr int NS = ModeTraits<MODE>::nparts;
    const int e = 1023 - (int)((((unsigned long long)__double_as_longlong(scale)) >> 52) & 0x7FFull);  // scale = 2^-e
    float d[NS];
    slice_digits<NS>(x, e, d);
#pragma unroll
    for (int k = 0; k < NS; ++k)
      reinterpret_cast<__nv_bfloat16*>(parts.p[k])[idx] = __float2bfloat16_rn(ldexpf(d[k], -7 * (k + 1)));
  } else if (is_ozaki(MODE)) {
    constexpr int BETA = ModeTraits<MODE>::beta, NS = ModeTraits<MODE>::nparts;
    double t = x * scale;  // |t| < 1, exact power-of-two scaling
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      t = t * (double)(1 << BETA);
      const double m = rint(t);
      t = t - m;
      // m 2^-BETA(k+1) is exact in BF16 (|m| <= 2^BETA)
      reinterpret_cast<__nv_bfloat16*>(parts.p[k])[idx] =
          __float2bfloat16_rn((float)(m * (1.0 / (double)(1ull << (BETA * (k + 1))))));
    }
  } else {
    const double h = round_sig<11>(x);
    reinterpret_cast<float*>(parts.p[0])[idx] = (float)h;
    if (MODE == TC_TF32X3) reinterpret_cast<float*>(parts.p[1])[idx] = (float)round_sig<11>(x - h);
  }
}

__device__ __forceinline__ double scale_of(const int* exps, int which) {
  return exps ? ldexp(1.0, -exps[which]) : 1.0;
}

// Slice-interleaved operand planes: rows come in groups of G (one occupied
// index, or one occupied pair), and a group's slices are consecutive blocks,
// [group][slice][G rows][Kp].  parts.p[s] points at slice s of group 0, so a
// row's element for every slice sits at the same index from its part.
__device__ __forceinline__ int64_t slice_index(int64_t row, int64_t k, int64_t G, int NS, int64_t Kp) {
  return (row / G) * (NS * G * Kp) + (row % G) * Kp + k;
}

// dst[row][kp] = src[row][k] (k < K) or 0, rows x Kp, slice-interleaved by
// groups of G rows; gexp (nullable): one scale exponent per group instead of
// exps[which]
template <int MODE>
__global__ void k_split_rows(const double* __restrict__ src, Parts parts, int64_t rows, int K, int Kp, int64_t G,
                             const int* exps, int which, const int* __restrict__ gexp = nullptr) {
  const double sc = scale_of(exps, which);
  const int64_t n = rows * Kp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % Kp);
    const int64_t row = idx / Kp;
    const double x = k < K ? src[row * K + k] : 0.0;
    split_store<MODE>(x, parts, slice_index(row, k, G, ModeTraits<MODE>::nparts, Kp),
                      gexp ? ldexp(1.0, -gexp[row / G]) : sc);
  }
}

// t2L[q][x][y][l] = t2[l][q][x][y], l padded to op; gexp (nullable): one
// exponent per q
template <int MODE>
__global__ void k_split_t2L(const double* __restrict__ t2, Parts parts, int o, int v, int op, const int* exps,
                            int which, const int* __restrict__ gexp = nullptr) {
  const double sc = scale_of(exps, which);
  const int64_t n = (int64_t)o * v * v * op;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(idx % op);
    int64_t rest = idx / op;
    const int y = (int)(rest % v);
    rest /= v;
    const int x = (int)(rest % v);
    const int q = (int)(rest / v);
    const double val = l < o ? t2[(((int64_t)l * o + q) * v + x) * v + y] : 0.0;
    split_store<MODE>(val, parts, slice_index(idx / op, l, (int64_t)v * v, ModeTraits<MODE>::nparts, op),
                      gexp ? ldexp(1.0, -gexp[q]) : sc);
  }
}

// nooT[p][r][z][l] = -ooov[p][l][r][z], l padded to op; gexp (nullable): one
// exponent per (p, r), at p o + r
template <int MODE>
__global__ void k_split_noo(const double* __restrict__ ooov, Parts parts, int o, int v, int op, const int* exps,
                            int which, const int* __restrict__ gexp = nullptr) {
  const double sc = scale_of(exps, which);
  const int64_t n = (int64_t)o * o * v * op;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(idx % op);
    int64_t rest = idx / op;
    const int z = (int)(rest % v);
    rest /= v;
    const int r = (int)(rest % o);
    const int p = (int)(rest / o);
    const double val = l < o ? -ooov[(((int64_t)p * o + l) * o + r) * v + z] : 0.0;
    split_store<MODE>(val, parts, slice_index(idx / op, l, v, ModeTraits<MODE>::nparts, op),
                      gexp ? ldexp(1.0, -gexp[p * o + r]) : sc);
  }
}

// ovs32[i][a][j][b] = 1/2 (ovov[i,a,j,b] + ovov[j,b,i,a]), b padded to vq
__global__ void k_ovs32(const double* __restrict__ ovov, float* __restrict__ ovs32, int o, int v, int vq) {
  const int64_t n = (int64_t)o * v * o * vq;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(idx % vq);
    int64_t rest = idx / vq;
    const int j = (int)(rest % o);
    rest /= o;
    const int a = (int)(rest % v);
    const int i = (int)(rest / v);
    float val = 0.f;
    if (b < v)
      val = (float)(0.5 * (ovov[(((int64_t)i * v + a) * o + j) * v + b] +
                           ovov[(((int64_t)j * v + b) * o + i) * v + a]));
    ovs32[idx] = val;
  }
}

// t1_32[i][a] = t1[i][a] as float32, a padded to vq
__global__ void k_small_copies(const double* __restrict__ t1, float* __restrict__ t1_32, int o, int v, int vq) {
  const int64_t n = (int64_t)o * vq;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx % vq);
    const int i = (int)(idx / vq);
    t1_32[idx] = a < v ? (float)t1[(int64_t)i * v + a] : 0.f;
  }
}

// max |x| of three arrays (bit patterns of non-negative doubles order as integers)
__global__ void k_maxabs(const double* __restrict__ a, int64_t na, const double* __restrict__ b, int64_t nb,
                         const double* __restrict__ c, int64_t nc, unsigned long long* out) {
  const double* src[3] = {a, b, c};
  const int64_t n[3] = {na, nb, nc};
  for (int w = 0; w < 3; ++w) {
    double m = 0.0;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n[w];
         idx += (int64_t)gridDim.x * blockDim.x)
      m = fmax(m, fabs(src[w][idx]));
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(out + w, (unsigned long long)__double_as_longlong(m));
  }
}

// Scale exponents: every segment of the K axis gets the unit 2^U.
// exps = {s_ovvv, s_t2, s_t2L, s_nooT, U}
__global__ void k_exponents(const unsigned long long* maxbits, int* exps) {
  int e[3];
  for (int w = 0; w < 3; ++w) {
    const double m = __longlong_as_double((long long)maxbits[w]);
    int ex = 0;
    if (m > 0.0) frexp(m, &ex);  // m < 2^ex
    e[w] = ex;
  }
  const int Eovvv = e[0], Et2 = e[1], Eooov = e[2];
  const int U = max(Eovvv + Et2, Et2 + Eooov);
  exps[0] = U - Et2;    // ovvv slices
  exps[1] = Et2;        // t2 slices
  exps[2] = U - Eooov;  // t2L slices
  exps[3] = Eooov;      // nooT slices
  exps[4] = U;
}

// max |x| per row group of the strided GEMMs' operands, one bit pattern per
// group (atomicMax of non-negative doubles).  Elements are enumerated group
// by group, in chunks of `chunk` per block iteration:
//   mode 0 ovvv[p][x][y][d]   group p       (groups of v^3)
//   mode 1 t2[r][q][z][d]     group r o + q (groups of v^2)
//   mode 2 t2[l][q][x][y]     group q       (the t2L view; groups of o v^2)
//   mode 3 ooov[p][l][r][z]   group p o + r (the nooT view; groups of o v)
__global__ void __launch_bounds__(256) k_group_maxabs(const double* __restrict__ src, int mode, int o, int v,
                                                      int64_t gsize, int64_t ngroups, int64_t chunk,
                                                      unsigned long long* __restrict__ out) {
  const int64_t cpg = (gsize + chunk - 1) / chunk;
  const int64_t v2 = (int64_t)v * v;
  __shared__ double red[8];
  for (int64_t cid = blockIdx.x; cid < ngroups * cpg; cid += gridDim.x) {
    const int64_t g = cid / cpg, i0 = (cid % cpg) * chunk, i1 = min(gsize, i0 + chunk);
    double m = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      int64_t a;
      if (mode <= 1) {
        a = g * gsize + i;
      } else if (mode == 2) {  // i = l v^2 + xy
        a = ((i / v2) * o + g) * v2 + i % v2;
      } else {                 // g = p o + r, i = l v + z
        const int64_t p = g / o, r = g % o;
        a = (((p * o) + i / v) * o + r) * v + i % v;
      }
      m = fmax(m, fabs(src[a]));
    }
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
      if (m > 0.0) atomicMax(out + g, (unsigned long long)__double_as_longlong(m));
    }
    __syncthreads();
  }
}

// exps[g] = e with 2^e > max of group g (0 for an all-zero group)
__global__ void k_group_exps(const unsigned long long* __restrict__ bits, int64_t n, int* __restrict__ exps) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const double m = __longlong_as_double((long long)bits[g]);
    int ex = 0;
    if (m > 0.0) frexp(m, &ex);
    exps[g] = ex;
  }
}

static int gridn(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>(1, (n + 255) / 256), 16384); }

// ---------------------------------------------------------------------------
// the GEMM kernel
// ---------------------------------------------------------------------------

// One 5-D map per operand view; the slice is a box dimension, so one copy
// brings every slice of a stage (the slices land part-contiguous in shared
// memory, as the MMA descriptors expect).
struct TcMaps {
  CUtensorMap a_nat;  // ovvv slices [p][s][x][y][Kp], dims (Kp, y, x, s, p): rows (x,y) of ovvv[p]
  CUtensorMap a_tr;   // the same with the y and x strides swapped: rows ovvv[q,y,x,:]
  CUtensorMap l_nat;  // t2L slices [q][s][x][y][op], natural
  CUtensorMap l_tr;   // t2L slices, transposed rows
  CUtensorMap b_t2;   // t2 slices [r][q][s][z][Kp], dims (Kp, z, s, q, r)
  CUtensorMap b_noo;  // nooT slices [p][r][s][z][op], dims (op, z, s, r, p)
};

// The maps of every cluster of a launch.
struct TcMapSet {
  TcMaps m[TC_MAX_CL];
};

// Per-cluster constants of a contraction launch.
struct TcCl {
  int o, v;
  int TA, TB, NT;
  int n_mx, n_my, n_nt;
  int kw_chunks, ko_chunks;
  int kw_elems, ko_elems;  // elements per chunk
  int cbo;                 // chunk bytes of the o-segments (the v-segments use TcParams::cbw)
  int64_t slot_floats;     // G floats per triple slot
  const int* exps;         // OZAKI scale exponents
};

struct TcParams {
  int ncl, npieces;
  int cbw;                 // chunk bytes of the v-segments
  int stages;
  uint32_t stage_bytes;    // stage stride: the largest cluster's A and B parts
  uint32_t a_part_bytes;   // 128 rows x cbw
  uint32_t tmem_cols;
  int nbuf;                // TMEM accumulator sets (1 or 2)
  int nt_max;              // largest N tile: stride of the accumulator sets
  int64_t total_tiles;
  const Triple* triples;
  unsigned int* err;
  unsigned long long wait_ns;
  TcCl cl[TC_MAX_CL];
  TcPiece pc[TC_MAX_PIECES];
};

__device__ __forceinline__ uint32_t layout_code(int cb) { return cb == 128 ? 2u : (cb == 64 ? 4u : 6u); }

__device__ __forceinline__ void record_abort(const TcParams& P, volatile int* abort_flag, unsigned site) {
  *abort_flag = 1;
  if (atomicOr(P.err, ERR_WAIT_TIMEOUT) == 0) {
    P.err[1] = site;
    P.err[2] = blockIdx.x;
  }
}

struct TileCoord {
  int cl, piece, slot, g, p, q, r, x0, y0, z0;
};

__device__ __forceinline__ TileCoord decode_tile(const TcParams& P, int64_t tt) {
  TileCoord c;
  int q = 0;  // pieces are in tile order
  while (q + 1 < P.npieces && P.pc[q + 1].tile0 <= tt) ++q;
  const TcPiece& pc = P.pc[q];
  const TcCl& C = P.cl[pc.cl];
  int64_t rest = tt - pc.tile0;
  const int nt = (int)(rest % C.n_nt);
  rest /= C.n_nt;
  const int my = (int)(rest % C.n_my);
  rest /= C.n_my;
  const int mx = (int)(rest % C.n_mx);
  rest /= C.n_mx;
  c.g = (int)(rest % 3);
  c.slot = (int)(rest / 3);
  c.cl = pc.cl;
  c.piece = q;
  const Triple T = P.triples[pc.t0 + c.slot];
  if (c.g == 0) { c.p = T.i; c.q = T.j; c.r = T.k; }
  else if (c.g == 1) { c.p = T.j; c.q = T.k; c.r = T.i; }
  else { c.p = T.k; c.q = T.i; c.r = T.j; }
  c.x0 = mx * C.TA;
  c.y0 = my * C.TB;
  c.z0 = nt * C.NT;
  return c;
}

// out[k] = v[k ^ h] for k < 8 (three conditional swap stages, no dynamic indexing)
__device__ __forceinline__ void xor_permute8(float* v, int h) {
  if (h & 1) {
#pragma unroll
    for (int k = 0; k < 8; k += 2) { const float t = v[k]; v[k] = v[k + 1]; v[k + 1] = t; }
  }
  if (h & 2) {
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if ((k & 2) == 0) { const float t = v[k]; v[k] = v[k + 2]; v[k + 2] = t; }
  }
  if (h & 4) {
#pragma unroll
    for (int k = 0; k < 4; ++k) { const float t = v[k]; v[k] = v[k + 4]; v[k + 4] = t; }
  }
}

__device__ __forceinline__ void store8(float* dst, const float* v) {
  float4* o4 = reinterpret_cast<float4*>(dst);
  o4[0] = make_float4(v[0], v[1], v[2], v[3]);
  o4[1] = make_float4(v[4], v[5], v[6], v[7]);
}

// Knuth's two-sum: s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Warp roles: 0 TMA producer, 1 MMA issuer (and TMEM owner), the rest
// epilogue: warp w drains TMEM lanes 32 (w % 4) .. +31 (the lane quarter its
// warp index may access) and every (GEMM_EPI_WARPS / 4)-th 16-column chunk,
// starting at chunk (w - 2) / 4.
#ifndef TE_GEMM_EPI_WARPS
#define TE_GEMM_EPI_WARPS 8
#endif
constexpr int GEMM_EPI_WARPS = TE_GEMM_EPI_WARPS;
constexpr int GEMM_EPI_GROUPS = GEMM_EPI_WARPS / 4;
constexpr int GEMM_THREADS = (2 + GEMM_EPI_WARPS) * 32;
// 16-column chunks one epilogue warp holds in registers with a single
// accumulator set (exact-slice N tiles of at most 160 columns)
constexpr int EPI_CHUNKS = 5;
constexpr int EPI_NT_MAX = 16 * GEMM_EPI_GROUPS * EPI_CHUNKS;

template <int MODE>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    k_gemm_tc(const __grid_constant__ TcMapSet maps, const __grid_constant__ TcParams P) {
  using MT = ModeTraits<MODE>;
  constexpr bool TF32 = MT::tf32;
  constexpr int NPART = MT::nparts;
  constexpr int NACC = MT::nacc;
  // TMEM accumulator sets: 2 when they fit (the epilogue of one tile then
  // overlaps the MMAs of the next), else 1
  const int NBUF = P.nbuf;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)P.stages * P.stage_bytes);
  uint64_t* empty = full + P.stages;
  uint64_t* tfull = empty + P.stages;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < P.stages; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      ptx::mbar_init(&tfull[a], 1);
      ptx::mbar_init(&tempty[a], GEMM_EPI_WARPS);
    }
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_barrier_init();
  }
  if (warp == 0 && lane < P.ncl) {
    const TcMaps& m = maps.m[lane];
    ptx::tma_prefetch_desc(&m.a_nat);
    ptx::tma_prefetch_desc(&m.a_tr);
    ptx::tma_prefetch_desc(&m.l_nat);
    ptx::tma_prefetch_desc(&m.l_tr);
    ptx::tma_prefetch_desc(&m.b_t2);
    ptx::tma_prefetch_desc(&m.b_noo);
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, P.tmem_cols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const uint32_t acc_stride = (uint32_t)(NACC * P.nt_max);  // TMEM columns between accumulator sets

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      uint32_t stage = 0, phase = 0;
      int pending[16];
      for (int s = 0; s < 16; ++s) pending[s] = -1;
      bool ok = true;
      for (int64_t tt = blockIdx.x; ok && tt < P.total_tiles; tt += gridDim.x) {
        const TileCoord c = decode_tile(P, tt);
        const TcCl& C = P.cl[c.cl];
        const TcMaps& mp = maps.m[c.cl];
        for (int seg = 0; ok && seg < 4; ++seg) {
          const bool wide = seg < 2;
          const int nch = wide ? C.kw_chunks : C.ko_chunks;
          const int cb = wide ? P.cbw : C.cbo;
          const int ce = wide ? C.kw_elems : C.ko_elems;
          const uint32_t bytes = (uint32_t)NPART * (128u * cb + (uint32_t)C.NT * cb);
          for (int ch = 0; ch < nch; ++ch) {
            if (*abort_flag || !ptx::mbar_wait(&empty[stage], phase ^ 1u, P.wait_ns)) {
              if (!*abort_flag) record_abort(P, abort_flag, 1);
              ok = false;
              break;
            }
            ptx::mbar_arrive_expect_tx(&full[stage], bytes);
            pending[stage] = (int)phase;
            unsigned char* sa = smem + (size_t)stage * P.stage_bytes;
            unsigned char* sb = sa + NPART * P.a_part_bytes;
            const int kc = ch * ce;
            if (seg == 0) {
              ptx::tma_load_5d(sa, &mp.a_nat, &full[stage], kc, c.y0, c.x0, 0, c.p);
              ptx::tma_load_5d(sb, &mp.b_t2, &full[stage], kc, c.z0, 0, c.q, c.r);
            } else if (seg == 1) {
              ptx::tma_load_5d(sa, &mp.a_tr, &full[stage], kc, c.y0, c.x0, 0, c.q);
              ptx::tma_load_5d(sb, &mp.b_t2, &full[stage], kc, c.z0, 0, c.p, c.r);
            } else if (seg == 2) {
              ptx::tma_load_5d(sa, &mp.l_tr, &full[stage], kc, c.y0, c.x0, 0, c.p);
              ptx::tma_load_5d(sb, &mp.b_noo, &full[stage], kc, c.z0, 0, c.r, c.q);
            } else {
              ptx::tma_load_5d(sa, &mp.l_nat, &full[stage], kc, c.y0, c.x0, 0, c.q);
              ptx::tma_load_5d(sb, &mp.b_noo, &full[stage], kc, c.z0, 0, c.r, c.p);
            }
            if (++stage == (uint32_t)P.stages) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
      }
      // copies still in flight must land before the CTA exits
      for (int s = 0; s < P.stages; ++s)
        if (pending[s] >= 0) ptx::mbar_wait(&full[s], (uint32_t)pending[s], P.wait_ns);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t fmt = TF32 ? 2u : 1u;
      uint32_t stage = 0, phase = 0, acc = 0, acc_phase = 0;
      bool ok = true;
      bool issued = false;
      for (int64_t tt = blockIdx.x; ok && tt < P.total_tiles; tt += gridDim.x) {
        const TileCoord c = decode_tile(P, tt);
        const TcCl& C = P.cl[c.cl];
        const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(C.NT >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
        if (*abort_flag || !ptx::mbar_wait(&tempty[acc], acc_phase ^ 1u, P.wait_ns)) {
          if (!*abort_flag) record_abort(P, abort_flag, 2);
          break;
        }
        ptx::tc_fence_after();
        const uint32_t d_tmem = tmem_base + acc * acc_stride;
        uint32_t first = 1;
        for (int seg = 0; ok && seg < 4; ++seg) {
          const bool wide = seg < 2;
          const int nch = wide ? C.kw_chunks : C.ko_chunks;
          const int cb = wide ? P.cbw : C.cbo;
          const uint32_t lay = layout_code(cb);
          const uint32_t sbo = 8u * (uint32_t)cb;
          for (int ch = 0; ch < nch; ++ch) {
            if (*abort_flag || !ptx::mbar_wait(&full[stage], phase, P.wait_ns)) {
              if (!*abort_flag) record_abort(P, abort_flag, 3);
              ok = false;
              break;
            }
            ptx::tc_fence_after();
            unsigned char* sa = smem + (size_t)stage * P.stage_bytes;
            const uint32_t a0 = ptx::smem_u32(sa);
            const uint32_t b0 = ptx::smem_u32(sa + NPART * P.a_part_bytes);
            for (int ks = 0; ks < cb / 32; ++ks) {
              uint64_t ad[NPART], bd[NPART];
#pragma unroll
              for (int k = 0; k < NPART; ++k) {
                // one box per operand lands the slices back to back: 128 (A) or NT (B) rows of cb bytes each
                ad[k] = ptx::smem_desc(a0 + k * (128u * (uint32_t)cb) + ks * 32, sbo, lay);
                bd[k] = ptx::smem_desc(b0 + k * ((uint32_t)C.NT * (uint32_t)cb) + ks * 32, sbo, lay);
              }
              const uint32_t acc_in = first ? 0u : 1u;
              if constexpr (is_ozaki(MODE)) {
                // slice products a_i b_j with i + j <= NPART - 1: level i + j = 0 and
                // level 1 each in an exact accumulator, the higher levels in a third
                const uint32_t d2 = d_tmem, d3 = d_tmem + C.NT, dr = d_tmem + 2 * C.NT;
                ptx::mma<false>(d2, ad[0], bd[0], idesc, acc_in);
                ptx::mma<false>(d3, ad[0], bd[1], idesc, acc_in);
                ptx::mma<false>(d3, ad[1], bd[0], idesc, 1);
                uint32_t rin = acc_in;
#pragma unroll
                for (int lev = 2; lev < NPART; ++lev)
#pragma unroll
                  for (int i = 0; i <= lev; ++i) {
                    ptx::mma<false>(dr, ad[i], bd[lev - i], idesc, rin);
                    rin = 1;
                  }
              } else {
                ptx::mma<TF32>(d_tmem, ad[0], bd[0], idesc, acc_in);
                if constexpr (NPART == 2) {
                  ptx::mma<TF32>(d_tmem, ad[0], bd[1], idesc, 1);
                  ptx::mma<TF32>(d_tmem, ad[1], bd[0], idesc, 1);
                }
              }
              first = 0;
            }
            issued = true;
            ptx::mma_commit(&empty[stage]);
            if (++stage == (uint32_t)P.stages) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
        if (!ok) break;
        ptx::mma_commit(&tfull[acc]);
        if (NBUF == 2) {
          acc ^= 1u;
          if (acc == 0) acc_phase ^= 1u;
        } else {
          acc_phase ^= 1u;
        }
      }
      // every issued MMA completes before TMEM is released
      if (issued) {
        ptx::mma_commit(drain);
        ptx::mbar_wait(drain, 0, P.wait_ns);
      }
    }
  } else {
    // ---------------- epilogue: TMEM -> G buffer ----------------
    const int quad = warp & 3;
    const int chunk0 = (warp - 2) >> 2;  // this warp's first 16-column chunk
    const int row = quad * 32 + lane;
    uint32_t acc = 0, acc_phase = 0;
    for (int64_t tt = blockIdx.x; tt < P.total_tiles; tt += gridDim.x) {
      const TileCoord c = decode_tile(P, tt);
      const TcCl& C = P.cl[c.cl];
      const TcPiece& pc = P.pc[c.piece];
      int got = 0;
      if (!*abort_flag) got = ptx::mbar_wait(&tfull[acc], acc_phase, P.wait_ns) ? 1 : 0;
      // the decision is warp-uniform: tcgen05.ld below is a .sync.aligned instruction
      if (!__all_sync(0xffffffffu, got)) {
        if (!*abort_flag && lane == 0) record_abort(P, abort_flag, 4);
        break;
      }
      ptx::tc_fence_after();
      float gscale = 1.f;
      if (is_ozaki(MODE)) gscale = ldexpf(1.f, C.exps[4]);
      const int x = c.x0 + row / C.TB;
      const int y = c.y0 + row % C.TB;
      const bool valid = x < C.v && y < C.v;
      // orbit-major G: [slot][bt][g][pid][CW planes][512], swizzled rows (see
      // energy_tc.h); this row is (x, y) = (X*8 + xl, Y*8 + yl)
      const int nb = (C.v + 7) >> 3;
      constexpr int CWF = is_ozaki(MODE) ? 2 : 1;
      float* const gslot = pc.gbuf + (int64_t)c.slot * C.slot_floats;
      const int roff = cube_row(x & 7, y & 7);
      const int zx = cube_zx(x & 7, y & 7);
      const uint32_t tbase = tmem_base + ((uint32_t)(quad * 32) << 16) + acc * acc_stride;
      if constexpr (is_ozaki(MODE) && GEMM_EPI_GROUPS == 2) {
        if (NBUF == 1) {
          // One accumulator set: copy it to registers as (hi, lo) pairs and
          // release it before the stores, so that the next tile's MMAs run
          // while this tile's G is written.  A warp holds at most
          // EPI_CHUNKS 16-column chunks (N tiles <= 160, checked on the
          // host).  lo is held rounded to BF16 (two per register): |lo| <=
          // ulp(hi) / 2, so the pair keeps 2^-33 of the value, far below the
          // 2^-28 of the exact-slice operands.
          float hv[EPI_CHUNKS][16];
          uint32_t lp[EPI_CHUNKS][8];
#pragma unroll
          for (int k = 0; k < EPI_CHUNKS; ++k) {
            const int c0 = 16 * chunk0 + 32 * k;
            if (c0 < C.NT) {
#pragma unroll
              for (int half = 0; half < 2; ++half) {  // 8 columns at a time: fewer live registers
                const int cc = c0 + 8 * half;
                float a2[8], a3[8], ar[8];
                ptx::tmem_ld8x3(tbase + cc, tbase + C.NT + cc, tbase + 2 * C.NT + cc, a2, a3, ar);
#pragma unroll
                for (int j = 0; j < 8; j += 2) {
                  float l2[2];
#pragma unroll
                  for (int q = 0; q < 2; ++q) {
                    float s, e;
                    two_sum(a2[j + q], a3[j + q], s, e);
                    const float lo = __fadd_rn(e, ar[j + q]);
                    const float hi = __fadd_rn(s, lo);
                    hv[k][8 * half + j + q] = hi * gscale;
                    l2[q] = __fsub_rn(lo, __fsub_rn(hi, s)) * gscale;
                  }
                  const __nv_bfloat162 b = __floats2bfloat162_rn(l2[0], l2[1]);
                  lp[k][4 * half + (j >> 1)] = *reinterpret_cast<const uint32_t*>(&b);
                }
              }
            }
          }
          ptx::tc_fence_before();
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(&tempty[acc]);
          acc_phase ^= 1u;
          if (valid) {
#pragma unroll
            for (int k = 0; k < EPI_CHUNKS; ++k) {
              const int c0 = 16 * chunk0 + 32 * k;
              if (c0 < C.NT) {
                const int z = c.z0 + c0;  // multiple of 16: two whole Z blocks
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                  const int Z = (z >> 3) + h2;
                  if (Z < nb) {
                    int64_t bt;
                    unsigned mask;
                    orbit_slots(x >> 3, y >> 3, Z, &bt, &mask);
                    float l8[8];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                      const uint32_t w = lp[k][4 * h2 + q];
                      l8[2 * q] = __uint_as_float(w << 16);
                      l8[2 * q + 1] = __uint_as_float(w & 0xffff0000u);
                    }
                    xor_permute8(hv[k] + 8 * h2, zx);
                    xor_permute8(l8, zx);
                    float* item = gslot + (bt * 18 + c.g * 6) * (512 * CWF);
                    for (int pid = 0; pid < 6; ++pid) {
                      if (!((mask >> pid) & 1u)) continue;
                      float* cube = item + pid * (512 * CWF);
                      store8(cube + roff, hv[k] + 8 * h2);
                      store8(cube + 512 + roff, l8);
                    }
                  }
                }
              }
            }
          }
          continue;
        }
      }
      for (int c0 = 16 * chunk0; c0 < C.NT; c0 += 16 * GEMM_EPI_GROUPS) {
        const int z = c.z0 + c0;  // multiple of 16: two whole Z blocks
        if constexpr (is_ozaki(MODE)) {
          float a2[16], a3[16], ar[16];
          ptx::tmem_ld16x3(tbase + c0, tbase + C.NT + c0, tbase + 2 * C.NT + c0, a2, a3, ar);
          if (valid) {
            float hv[16], lv[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              float s, e;
              two_sum(a2[j], a3[j], s, e);
              const float lo = __fadd_rn(e, ar[j]);
              const float hi = __fadd_rn(s, lo);
              hv[j] = hi * gscale;
              lv[j] = __fsub_rn(lo, __fsub_rn(hi, s)) * gscale;
            }
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
              const int Z = (z >> 3) + h2;
              if (Z < nb) {
                int64_t bt;
                unsigned mask;
                orbit_slots(x >> 3, y >> 3, Z, &bt, &mask);
                xor_permute8(hv + 8 * h2, zx);
                xor_permute8(lv + 8 * h2, zx);
                float* item = gslot + (bt * 18 + c.g * 6) * (512 * CWF);
                for (int pid = 0; pid < 6; ++pid) {
                  if (!((mask >> pid) & 1u)) continue;
                  float* cube = item + pid * (512 * CWF);
                  store8(cube + roff, hv + 8 * h2);
                  store8(cube + 512 + roff, lv + 8 * h2);
                }
              }
            }
          }
        } else {
          float vals[16];
          ptx::tmem_ld16(tbase + c0, vals);
          if (valid) {
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
              const int Z = (z >> 3) + h2;
              if (Z < nb) {
                int64_t bt;
                unsigned mask;
                orbit_slots(x >> 3, y >> 3, Z, &bt, &mask);
                xor_permute8(vals + 8 * h2, zx);
                float* item = gslot + (bt * 18 + c.g * 6) * 512;
                for (int pid = 0; pid < 6; ++pid)
                  if ((mask >> pid) & 1u) store8(item + pid * 512 + roff, vals + 8 * h2);
              }
            }
          }
        }
      }
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&tempty[acc]);
      if (NBUF == 2) {
        acc ^= 1u;
        if (acc == 0) acc_phase ^= 1u;
      } else {
        acc_phase ^= 1u;
      }
    }
  }

  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem_base, P.tmem_cols);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct TcState {
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
};

static TcState* tc_state(Handle* h) {
  if (!h->tc) h->tc = new TcState();
  return static_cast<TcState*>(h->tc);
}

void destroy_tc_state(Handle* h) {
  delete static_cast<TcState*>(h->tc);
  h->tc = nullptr;
}

static te_status get_encoder(TcState* st) {
  if (st->encode) return TE_OK;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
          cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return fail(TE_ECUDA, "cuTensorMapEncodeTiled entry point not available");
  }
  st->encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return TE_OK;
}

struct TcPlan {
  int mode, es, nparts, cw;
  int vp, op, vq;
  int TA, TB, NT, n_mx, n_my, n_nt;
  int kw_chunks, ko_chunks, kw_elems, ko_elems, cbw, cbo;
  int stages;
  uint32_t stage_bytes, a_part_bytes, b_part_bytes, tmem_cols;
  int nbuf;
  int nslots;
  int ldz;
  size_t smem;
};

static int round_up(int x, int m) { return (x + m - 1) / m * m; }

static TcPlan make_plan(const Handle* h, int o, int v, int mode, int64_t ntri, int force_tb = 0,
                        int force_nnt = 0) {
  TcPlan pl{};
  pl.mode = mode;
  const bool oz = is_ozaki(mode);
  pl.es = (mode == TC_BF16X3 || oz) ? 2 : 4;
  pl.nparts = mode == TC_TF32 ? 1 : (mode == TC_OZAKI ? 4 : (mode == TC_OZAKI6 ? 5 : 2));
  pl.cw = oz ? 2 : 1;
  const int nacc = oz ? 3 : 1;
  // TF32/BF16X3 (one accumulator) double-buffer at any N tile; the exact-slice
  // modes (three accumulators) take N tiles up to 160 single-buffered, and
  // double-buffer when 2 x 3 x NT <= 512 columns (NT <= 80)
  const int nbuf_max = oz ? 1 : 2;
  pl.vp = round_up(v, 16);
  pl.op = round_up(o, 16);
  pl.vq = round_up(v, 4);
  // M tile: TA x-values by TB y-values, TA*TB = 128, least padding
  int bestTB = 128;
  int64_t best = -1;
  for (int TB = 128; TB >= 16; TB /= 2) {
    const int TA = 128 / TB;
    const int64_t rows = (int64_t)round_up(v, TA) * round_up(v, TB);
    if (best < 0 || rows < best) {
      best = rows;
      bestTB = TB;
    }
  }
  if (!force_tb) {
    auto it = h->tuned.find(std::make_tuple(o, v, mode));
    if (it != h->tuned.end()) {
      force_tb = it->second.first;
      force_nnt = it->second.second;
    }
  }
  if (force_tb) bestTB = force_tb;
  pl.TB = bestTB;
  pl.TA = 128 / bestTB;
  pl.n_mx = (v + pl.TA - 1) / pl.TA;
  pl.n_my = (v + pl.TB - 1) / pl.TB;
  const int ntmax = std::min(256, (512 / (nacc * nbuf_max)) / 16 * 16);
  pl.n_nt = (v + ntmax - 1) / ntmax;
  // a tuned split: any count whose N tile fits three accumulators in TMEM (N <= 160)
  if (force_nnt > 0 && round_up((v + force_nnt - 1) / force_nnt, 16) <= (oz ? 160 : 256)) pl.n_nt = force_nnt;
  pl.NT = round_up((v + pl.n_nt - 1) / pl.n_nt, 16);
  pl.nbuf = (2 * nacc * pl.NT <= 512) ? 2 : 1;
  pl.cbw = oz ? 64 : 128;
  pl.kw_elems = pl.cbw / pl.es;
  pl.kw_chunks = (pl.vp + pl.kw_elems - 1) / pl.kw_elems;
  const int obytes = pl.op * pl.es;
  pl.cbo = obytes <= 32 ? 32 : (obytes <= 64 ? 64 : std::min(128, pl.cbw));
  pl.ko_elems = pl.cbo / pl.es;
  pl.ko_chunks = (pl.op + pl.ko_elems - 1) / pl.ko_elems;
  pl.a_part_bytes = 128u * (uint32_t)pl.cbw;
  pl.b_part_bytes = (uint32_t)pl.NT * (uint32_t)pl.cbw;
  pl.stage_bytes = (uint32_t)pl.nparts * (pl.a_part_bytes + pl.b_part_bytes);
  const size_t avail = h->smem_optin > 2048 ? h->smem_optin - 2048 : 0;
  pl.stages = (int)std::min<size_t>(8, avail / pl.stage_bytes);
  pl.smem = (size_t)pl.stages * pl.stage_bytes + 1024 + 256;
  uint32_t cols = 32;
  while (cols < (uint32_t)(nacc * pl.nbuf * pl.NT)) cols <<= 1;
  pl.tmem_cols = cols;
  pl.ldz = round_up(v, 4);
  const int64_t tiles = 3LL * pl.n_mx * pl.n_my * pl.n_nt;
  int64_t want = (4LL * std::max(1, h->num_sms) + tiles - 1) / tiles;
  const int64_t per_slot = g_slot_floats(v, pl.cw) * 4;
  const int64_t mem_cap = std::max<int64_t>(1, (int64_t)(6LL << 30) / per_slot);
  want = std::max<int64_t>(want, 4);  // fewer launches per cluster
  want = std::min<int64_t>({want, mem_cap, 1024, std::max<int64_t>(1, ntri)});
  pl.nslots = (int)std::max<int64_t>(1, want);
  return pl;
}

// ---------------------------------------------------------------------------
// host side: workspace, launch rounds
// ---------------------------------------------------------------------------

// One cluster's part of the workspace: the operand planes, the float32
// copies the energy kernel reads, the scale exponents and the per-triple
// shares.  The G pool and the energy partials are shared by a whole run.
struct TcBuffers {
  void *a[MAX_PARTS], *b[MAX_PARTS], *l[MAX_PARTS], *n[MAX_PARTS];
  float *ovs32, *t1_32;
  double* etri;
  unsigned long long* maxbits;
  int* exps;
};

static size_t tc_carve_cluster(char* base, const TcPlan& pl, int64_t o, int64_t v, int64_t ntri, TcBuffers* b) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> void* {
    off = (off + 1023) & ~size_t(1023);
    void* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  };
  const size_t es = (size_t)pl.es;
  const size_t na = (size_t)o * v * v * pl.vp, nb = (size_t)o * o * v * pl.vp;
  const size_t nl = (size_t)o * v * v * pl.op, nn = (size_t)o * o * v * pl.op;
  // one slice-interleaved block per array; part k points at slice k of the
  // first row group (groups: v^2 rows per occupied index for ovvv and t2L,
  // v rows per occupied pair for t2 and nooT)
  const size_t ns = (size_t)pl.nparts;
  char* A = static_cast<char*>(take(ns * na * es));
  char* B = static_cast<char*>(take(ns * nb * es));
  char* Lb = static_cast<char*>(take(ns * nl * es));
  char* Nb = static_cast<char*>(take(ns * nn * es));
  for (int k = 0; k < MAX_PARTS; ++k) {
    const bool use = k < pl.nparts && base;
    b->a[k] = use ? A + (size_t)k * v * v * pl.vp * es : nullptr;
    b->b[k] = use ? B + (size_t)k * v * pl.vp * es : nullptr;
    b->l[k] = use ? Lb + (size_t)k * v * v * pl.op * es : nullptr;
    b->n[k] = use ? Nb + (size_t)k * v * pl.op * es : nullptr;
  }
  b->ovs32 = static_cast<float*>(take((size_t)o * v * o * pl.vq * 4));
  b->t1_32 = static_cast<float*>(take((size_t)o * pl.vq * 4));
  b->etri = static_cast<double*>(take((size_t)std::max<int64_t>(1, ntri) * 8));
  b->maxbits = static_cast<unsigned long long*>(take(4 * 8));
  b->exps = static_cast<int*>(take(8 * 4));
  return (off + 1023) & ~size_t(1023);
}

// Workspace of one run: the clusters' parts, then the G pool, then the
// energy partials: per G slot of a launch, one float64 sum per block (one
// block per SM) and compute warp.
struct TcPool {
  int64_t pool_floats;
  int64_t max_slots;  // G slots per launch
};

static size_t tc_partial_bytes(const TcPool& q, int num_sms) {
  return (size_t)q.max_slots * std::max(1, num_sms) * ENERGY_TC_WARPS * sizeof(double);
}

static size_t tc_shared_bytes(const TcPool& q, int num_sms) {
  const size_t g = ((size_t)q.pool_floats * 4 + 1023) & ~size_t(1023);
  return g + tc_partial_bytes(q, num_sms) + 1024;
}

static te_status encode(TcState* st, CUtensorMap* m, const void* base, CUtensorMapDataType dt, int rank,
                        const uint64_t* dims, const uint64_t* strides_bytes, const uint32_t* box,
                        CUtensorMapSwizzle swz, const char* what) {
  cuuint64_t gd[5];
  cuuint64_t gs[4];
  cuuint32_t bd[5], e1[5];
  for (int i = 0; i < rank; ++i) {
    gd[i] = dims[i];
    bd[i] = box[i];
    e1[i] = 1;
    if (i < rank - 1) gs[i] = strides_bytes[i];
  }
  CUresult r = st->encode(m, dt, (cuuint32_t)rank, const_cast<void*>(base), gd, gs, bd, e1,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(TE_ECUDA, "tensor map encoding failed for %s (CUresult %d)", what, (int)r);
  return TE_OK;
}

static CUtensorMapSwizzle swz_of(int cb) {
  return cb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : (cb == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
}

static te_status build_maps(TcState* st, const TcPlan& pl, int o, int v, const TcBuffers& b, TcMaps* M) {
  std::memset(M, 0, sizeof(*M));
  const CUtensorMapDataType dt = pl.es == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const uint64_t es = (uint64_t)pl.es;
  const uint64_t vp = pl.vp, op = pl.op, V = v, O = o, NS = (uint64_t)pl.nparts;
  const uint32_t ns = (uint32_t)pl.nparts;
  te_status s;
  {  // ovvv slices [p][s][x][y][d]: dims (d, y, x, s, p)
    const uint64_t d[5] = {vp, V, V, NS, O};
    const uint64_t sn[4] = {vp * es, V * vp * es, V * V * vp * es, NS * V * V * vp * es};
    const uint32_t box[5] = {(uint32_t)pl.kw_elems, (uint32_t)pl.TB, (uint32_t)pl.TA, ns, 1};
    if ((s = encode(st, &M->a_nat, b.a[0], dt, 5, d, sn, box, swz_of(pl.cbw), "ovvv")) != TE_OK) return s;
    // transposed rows: element (d, y, x, s, q) at ovvv[q][s][y][x][d]
    const uint64_t stt[4] = {V * vp * es, vp * es, V * V * vp * es, NS * V * V * vp * es};
    if ((s = encode(st, &M->a_tr, b.a[0], dt, 5, d, stt, box, swz_of(pl.cbw), "ovvv^T")) != TE_OK) return s;
  }
  {  // t2L slices [q][s][x][y][l]: dims (l, y, x, s, q)
    const uint64_t d[5] = {op, V, V, NS, O};
    const uint64_t sn[4] = {op * es, V * op * es, V * V * op * es, NS * V * V * op * es};
    const uint32_t box[5] = {(uint32_t)pl.ko_elems, (uint32_t)pl.TB, (uint32_t)pl.TA, ns, 1};
    if ((s = encode(st, &M->l_nat, b.l[0], dt, 5, d, sn, box, swz_of(pl.cbo), "t2L")) != TE_OK) return s;
    const uint64_t stt[4] = {V * op * es, op * es, V * V * op * es, NS * V * V * op * es};
    if ((s = encode(st, &M->l_tr, b.l[0], dt, 5, d, stt, box, swz_of(pl.cbo), "t2L^T")) != TE_OK) return s;
  }
  {  // t2 slices [r][q][s][z][d]: dims (d, z, s, q, r)
    const uint64_t d[5] = {vp, V, NS, O, O};
    const uint64_t sn[4] = {vp * es, V * vp * es, NS * V * vp * es, O * NS * V * vp * es};
    const uint32_t box[5] = {(uint32_t)pl.kw_elems, (uint32_t)pl.NT, ns, 1, 1};
    if ((s = encode(st, &M->b_t2, b.b[0], dt, 5, d, sn, box, swz_of(pl.cbw), "t2")) != TE_OK) return s;
  }
  {  // nooT slices [p][r][s][z][l]: dims (l, z, s, r, p)
    const uint64_t d[5] = {op, V, NS, O, O};
    const uint64_t sn[4] = {op * es, V * op * es, NS * V * op * es, O * NS * V * op * es};
    const uint32_t box[5] = {(uint32_t)pl.ko_elems, (uint32_t)pl.NT, ns, 1, 1};
    if ((s = encode(st, &M->b_noo, b.n[0], dt, 5, d, sn, box, swz_of(pl.cbo), "nooT")) != TE_OK) return s;
  }
  return TE_OK;
}

struct EnergyMapsHost {
  CUtensorMap ovs, t1;
};

static te_status build_energy_maps(TcState* st, const TcPlan& pl, int o, int v, const TcBuffers& b,
                                   EnergyMapsHost* E) {
  std::memset(E, 0, sizeof(*E));
  const uint64_t V = v, O = o, vq = pl.vq;
  te_status s;
  {  // ovs32 [i][a][j][vq]: dims (b, j, a, i)
    const uint64_t d[4] = {V, O, V, O};
    const uint64_t sn[3] = {vq * 4, O * vq * 4, V * O * vq * 4};
    const uint32_t box[4] = {8, 1, 8, 1};
    if ((s = encode(st, &E->ovs, b.ovs32, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, d, sn, box,
                    CU_TENSOR_MAP_SWIZZLE_NONE, "ovs")) != TE_OK)
      return s;
  }
  {  // t1 [i][vq]: dims (a, i)
    const uint64_t d[2] = {V, O};
    const uint64_t sn[1] = {vq * 4};
    const uint32_t box[2] = {8, 1};
    if ((s = encode(st, &E->t1, b.t1_32, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, d, sn, box,
                    CU_TENSOR_MAP_SWIZZLE_NONE, "t1")) != TE_OK)
      return s;
  }
  return TE_OK;
}

// ---------------------------------------------------------------------------
// ovvv from density-fitting factors (t_energy_df):
//   ovvv[p,x,y,d] = sum_P Bov[P,p,x] Bvv[P,y,d]
// formed nst slabs at a time by the exact-slice strided GEMM (five 7-bit
// slices per factor, K blocks of at most 1024 accumulated in float64) into a
// float64 staging block, then cut into the contraction's operand form.
// ---------------------------------------------------------------------------

constexpr int DF_NS = 5;                                  // slices per factor
constexpr size_t DF_STAGE_BYTES = size_t(2) << 30;        // staging block limit
constexpr int64_t DF_KBLOCK = 1024;                       // exact level-0/1 sums

// Scratch of the formation.  It shares the region of the G pool, which the
// contraction only writes after every operand is ready (stream order).
struct DfScratch {
  __nv_bfloat16 *bov = nullptr, *bvv = nullptr;  // DF_NS planes each
  unsigned long long* mx = nullptr;              // max |Bov|, max |Bvv| (bits)
  int* ex = nullptr;                             // their scale exponents
  double* stage = nullptr;                       // nst slabs of v^3
  double* part = nullptr;                        // split-K partial tiles
  int64_t part_cap = 0;
  int nst = 0;
};

static size_t df_carve(char* base, int o, int v, int64_t naux, int num_sms, DfScratch* d) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    off = (off + 1023) & ~size_t(1023);
    char* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  };
  const size_t v3 = (size_t)v * v * v;
  d->nst = (int)std::max<size_t>(1, std::min<size_t>((size_t)o, DF_STAGE_BYTES / (v3 * 8)));
  d->bov = reinterpret_cast<__nv_bfloat16*>(take((size_t)DF_NS * naux * o * v * 2));
  d->bvv = reinterpret_cast<__nv_bfloat16*>(take((size_t)DF_NS * naux * v * v * 2));
  d->mx = reinterpret_cast<unsigned long long*>(take(16));
  d->ex = reinterpret_cast<int*>(take(8));
  d->stage = reinterpret_cast<double*>(take((size_t)d->nst * v3 * 8));
  // the largest split-K scratch over the slab counts and K blocks that occur
  int64_t cap = 0;
  const int64_t kcs[2] = {std::min<int64_t>(naux, DF_KBLOCK), naux % DF_KBLOCK};
  const int nes[2] = {d->nst, o % d->nst};
  for (int64_t kc : kcs)
    for (int ne : nes)
      if (kc > 0 && ne > 0) cap = std::max(cap, gemm_oz_scratch((int64_t)ne * v, (int64_t)v * v, kc, num_sms));
  d->part_cap = cap;
  d->part = reinterpret_cast<double*>(take((size_t)std::max<int64_t>(cap, 1) * 8));
  return (off + 1023) & ~size_t(1023);
}

// slabs p0 .. p0+ne-1 of ovvv into the staging block ([p - p0][x][y][d])
static cudaError_t df_form(const te_df* df, int o, int v, int p0, int ne, const DfScratch& d, int num_sms,
                           cudaStream_t s, int64_t* launches) {
  const int64_t P = df->naux, ov = (int64_t)o * v, vv = (int64_t)v * v;
  for (int64_t k0 = 0; k0 < P; k0 += DF_KBLOCK) {
    const int64_t kc = std::min<int64_t>(DF_KBLOCK, P - k0);
    // rows m = (p, x) contiguous in Bov[P][o][v]; columns n = (y, d) contiguous in Bvv[P][v][v]
    const OzView g{d.bov + k0 * ov + (int64_t)p0 * v, d.bvv + k0 * vv, P * ov, P * vv, d.stage,
                   (int64_t)ne * v, 1, vv, kc, 1,
                   1, 0, ov, 0,
                   vv, 0, 1,
                   vv, 0, 1,
                   1.0, d.ex, d.ex + 1, k0 == 0 ? 1 : 0, DF_NS};
    const cudaError_t e = gemm_oz(g, num_sms, d.part, d.part_cap, s, launches);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Operand planes of one cluster.  With df, ovvv comes from the factors (the
// slabs are formed once for the maximum in the exact-slice modes, once for
// the slices: the same bits both times); else from c->ovvv.
template <int MODE>
static cudaError_t launch_prep_tc(const te_cluster* c, const TcPlan& pl, const TcBuffers& b, const te_df* df,
                                  const DfScratch* dfs, int num_sms, cudaStream_t s, int64_t* launches) {
  const int o = (int)c->nocc, v = (int)c->nvir;
  const int64_t v3 = (int64_t)v * v * v;
  const int* ex = nullptr;
  cudaError_t e = cudaSuccess;
  if (df) {
    e = slice_planes(df->Bov, df->naux * o * v, DF_NS, dfs->mx, dfs->ex, dfs->bov, s, launches);
    if (e == cudaSuccess) e = slice_planes(df->Bvv, df->naux * v * v, DF_NS, dfs->mx + 1, dfs->ex + 1, dfs->bvv, s, launches);
    if (e != cudaSuccess) return e;
  }
  if (is_ozaki(MODE)) {
    cudaMemsetAsync(b.maxbits, 0, 4 * 8, s);
    k_maxabs<<<1024, 256, 0, s>>>(df ? nullptr : c->ovvv, df ? 0 : (int64_t)o * v3, c->t2, (int64_t)o * o * v * v,
                                  c->ooov, (int64_t)o * o * o * v, b.maxbits);
    ++*launches;
    for (int p0 = 0; df && p0 < o; p0 += dfs->nst) {
      const int ne = std::min(dfs->nst, o - p0);
      e = df_form(df, o, v, p0, ne, *dfs, num_sms, s, launches);
      if (e != cudaSuccess) return e;
      k_maxabs<<<1024, 256, 0, s>>>(dfs->stage, (int64_t)ne * v3, nullptr, 0, nullptr, 0, b.maxbits);
      ++*launches;
    }
    k_exponents<<<1, 1, 0, s>>>(b.maxbits, b.exps);
    ++*launches;
    ex = b.exps;
  }
  const Parts A{{b.a[0], b.a[1], b.a[2], b.a[3], b.a[4]}}, B{{b.b[0], b.b[1], b.b[2], b.b[3], b.b[4]}};
  const Parts Lp{{b.l[0], b.l[1], b.l[2], b.l[3], b.l[4]}}, N{{b.n[0], b.n[1], b.n[2], b.n[3], b.n[4]}};
  if (!df) {
    k_split_rows<MODE><<<gridn((int64_t)o * v * v * pl.vp), 256, 0, s>>>(c->ovvv, A, (int64_t)o * v * v, v, pl.vp,
                                                                         (int64_t)v * v, ex, 0);
    ++*launches;
  }
  // one occupied index's slices of ovvv: nparts consecutive [v^2][vp] blocks
  const size_t group = (size_t)pl.nparts * v * v * pl.vp * pl.es;
  for (int p0 = 0; df && p0 < o; p0 += dfs->nst) {
    const int ne = std::min(dfs->nst, o - p0);
    e = df_form(df, o, v, p0, ne, *dfs, num_sms, s, launches);
    if (e != cudaSuccess) return e;
    Parts Ap{};
    for (int k = 0; k < MAX_PARTS; ++k) Ap.p[k] = A.p[k] ? static_cast<char*>(A.p[k]) + (size_t)p0 * group : nullptr;
    k_split_rows<MODE><<<gridn((int64_t)ne * v * v * pl.vp), 256, 0, s>>>(dfs->stage, Ap, (int64_t)ne * v * v, v,
                                                                          pl.vp, (int64_t)v * v, ex, 0);
    ++*launches;
  }
  k_split_rows<MODE><<<gridn((int64_t)o * o * v * pl.vp), 256, 0, s>>>(c->t2, B, (int64_t)o * o * v, v, pl.vp,
                                                                       (int64_t)v, ex, 1);
  k_split_t2L<MODE><<<gridn((int64_t)o * v * v * pl.op), 256, 0, s>>>(c->t2, Lp, o, v, pl.op, ex, 2);
  k_split_noo<MODE><<<gridn((int64_t)o * o * v * pl.op), 256, 0, s>>>(c->ooov, N, o, v, pl.op, ex, 3);
  k_ovs32<<<gridn((int64_t)o * v * o * pl.vq), 256, 0, s>>>(c->ovov, b.ovs32, o, v, pl.vq);
  k_small_copies<<<gridn((int64_t)o * pl.vq), 256, 0, s>>>(c->t1, b.t1_32, o, v, pl.vq);
  *launches += 5;
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_gemm_tc(const TcMapSet& M, const TcParams& P, size_t smem, int grid_cap, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t grid = std::min<int64_t>(P.total_tiles, grid_cap);
  k_gemm_tc<MODE><<<(unsigned)grid, GEMM_THREADS, smem, s>>>(M, P);
  return cudaGetLastError();
}

static cudaError_t launch_gemm_any(int mode, const TcMapSet& M, const TcParams& P, size_t smem, int grid_cap,
                                   cudaStream_t s) {
  if (mode == TC_BF16X3) return launch_gemm_tc<TC_BF16X3>(M, P, smem, grid_cap, s);
  if (mode == TC_TF32X3) return launch_gemm_tc<TC_TF32X3>(M, P, smem, grid_cap, s);
  if (mode == TC_TF32) return launch_gemm_tc<TC_TF32>(M, P, smem, grid_cap, s);
  if (mode == TC_OZAKI) return launch_gemm_tc<TC_OZAKI>(M, P, smem, grid_cap, s);
  return launch_gemm_tc<TC_OZAKI6>(M, P, smem, grid_cap, s);
}

static cudaError_t launch_prep_any(int mode, const te_cluster* c, const TcPlan& pl, const TcBuffers& b,
                                   const te_df* df, const DfScratch* dfs, int num_sms, cudaStream_t s,
                                   int64_t* launches) {
  if (mode == TC_BF16X3) return launch_prep_tc<TC_BF16X3>(c, pl, b, df, dfs, num_sms, s, launches);
  if (mode == TC_TF32X3) return launch_prep_tc<TC_TF32X3>(c, pl, b, df, dfs, num_sms, s, launches);
  if (mode == TC_TF32) return launch_prep_tc<TC_TF32>(c, pl, b, df, dfs, num_sms, s, launches);
  if (mode == TC_OZAKI) return launch_prep_tc<TC_OZAKI>(c, pl, b, df, dfs, num_sms, s, launches);
  return launch_prep_tc<TC_OZAKI6>(c, pl, b, df, dfs, num_sms, s, launches);
}

// One cluster of a run: its plan, buffers, tensor maps and triple range.
struct TcJob {
  const te_cluster* c = nullptr;
  TcPlan pl{};
  TcBuffers b{};
  TcMaps maps{};
  EnergyMapsHost em{};
  int o = 0, v = 0;
  int64_t t_begin = 0, t_end = 0;
  int64_t nbt = 0, slot_floats = 0, tiles_per_triple = 0;
  double* shares = nullptr;  // share of triple t at shares[t - t_begin]
  double* e_out = nullptr;   // sum of the shares (nullable)
};

static void fill_cluster(const TcJob& J, TcCl* C) {
  C->o = J.o;
  C->v = J.v;
  C->TA = J.pl.TA;
  C->TB = J.pl.TB;
  C->NT = J.pl.NT;
  C->n_mx = J.pl.n_mx;
  C->n_my = J.pl.n_my;
  C->n_nt = J.pl.n_nt;
  C->kw_chunks = J.pl.kw_chunks;
  C->ko_chunks = J.pl.ko_chunks;
  C->kw_elems = J.pl.kw_elems;
  C->ko_elems = J.pl.ko_elems;
  C->cbo = J.pl.cbo;
  C->slot_floats = J.slot_floats;
  C->exps = J.b.exps;
}

// Contraction parameters of one launch over the clusters jl[0..ncl) of `jobs`
// and the given pieces; *smem receives the dynamic shared memory.
static te_status gemm_params(const Handle* h, const std::vector<TcJob>& jobs, const int* jl, int ncl,
                             const TcPiece* pcs, int npieces, int64_t tiles, int mode, TcParams* P, TcMapSet* M,
                             size_t* smem) {
  std::memset(P, 0, sizeof(*P));
  std::memset(M, 0, sizeof(*M));
  uint32_t stage_max = 0;
  int nt_max = 0;
  for (int q = 0; q < ncl; ++q) {
    const TcJob& J = jobs[jl[q]];
    fill_cluster(J, &P->cl[q]);
    M->m[q] = J.maps;
    stage_max = std::max(stage_max, J.pl.stage_bytes);
    nt_max = std::max(nt_max, J.pl.NT);
  }
  const TcPlan& p0 = jobs[jl[0]].pl;
  const int nacc = is_ozaki(mode) ? 3 : 1;
  P->ncl = ncl;
  P->npieces = npieces;
  P->cbw = p0.cbw;
  P->a_part_bytes = 128u * (uint32_t)p0.cbw;
  P->stage_bytes = stage_max;
  const size_t avail = h->smem_optin > 2048 ? h->smem_optin - 2048 : 0;
  P->stages = (int)std::min<size_t>(8, avail / stage_max);
  if (P->stages < 2) return fail(TE_EUNSUPPORTED, "not enough shared memory for two pipeline stages");
  P->nbuf = p0.nbuf;
  P->nt_max = nt_max;
  if (is_ozaki(mode) && P->nbuf == 1 && nt_max > EPI_NT_MAX)
    return fail(TE_EUNSUPPORTED, "N tile %d above the epilogue's %d columns", nt_max, EPI_NT_MAX);
  uint32_t cols = 32;
  while (cols < (uint32_t)(nacc * P->nbuf * nt_max)) cols <<= 1;
  P->tmem_cols = cols;
  P->total_tiles = tiles;
  P->triples = h->d_triples;
  P->err = h->d_err;
  P->wait_ns = h->wait_limit_ns;
  for (int q = 0; q < npieces; ++q) P->pc[q] = pcs[q];
  *smem = (size_t)P->stages * stage_max + 1024 + 256;
  return TE_OK;
}

// Runs the jobs' triples in rounds: each round fills the G pool with pieces
// (up to TC_MAX_CL clusters, TC_MAX_PIECES pieces, one TMEM buffering), then
// launches the contraction, the energy epilogue and the share reduction once.
// Then each job's total.  Pieces follow the jobs' order.
static te_status run_rounds(Handle* h, std::vector<TcJob>& jobs, int mode, float* pool, const TcPool& pq,
                            double* partials, cudaStream_t s) {
  const double nprod = (mode == TC_TF32) ? 1.0 : (mode == TC_OZAKI ? 10.0 : (mode == TC_OZAKI6 ? 15.0 : 3.0));
  const int cw = is_ozaki(mode) ? 2 : 1;
  size_t j = 0;
  int64_t t = jobs.empty() ? 0 : jobs[0].t_begin;
  std::vector<TcPiece> pcs;
  TcMapSet* MS = new TcMapSet;
  TcParams* P = new TcParams;
  EnergyLaunch* EL = new EnergyLaunch;
  te_status st = TE_OK;
  while (st == TE_OK) {
    while (j < jobs.size() && t >= jobs[j].t_end) {
      ++j;
      if (j < jobs.size()) t = jobs[j].t_begin;
    }
    if (j >= jobs.size()) break;
    int jl[TC_MAX_CL];
    int ncl = 0, nbuf = -1, nslots = 0;
    int64_t used = 0, tiles = 0, items = 0;
    double flops = 0.0;
    pcs.clear();
    while (j < jobs.size() && (int)pcs.size() < TC_MAX_PIECES) {
      TcJob& J = jobs[j];
      if (t >= J.t_end) {
        ++j;
        if (j < jobs.size()) t = jobs[j].t_begin;
        continue;
      }
      int cl = -1;
      for (int q = 0; q < ncl; ++q)
        if (jl[q] == (int)j) cl = q;
      if (cl < 0) {
        if (ncl == TC_MAX_CL || (nbuf >= 0 && J.pl.nbuf != nbuf)) break;
        cl = ncl;
      }
      const int64_t fit = std::min((pq.pool_floats - used) / J.slot_floats, pq.max_slots - nslots);
      if (fit <= 0) break;
      if (cl == ncl) {
        jl[ncl++] = (int)j;
        nbuf = J.pl.nbuf;  // one TMEM buffering per launch
      }
      const int ns = (int)std::min<int64_t>(fit, J.t_end - t);
      TcPiece pc{};
      pc.cl = cl;
      pc.ns = ns;
      pc.slot0 = nslots;
      pc.t0 = t;
      pc.tile0 = tiles;
      pc.item0 = items;
      pc.nbt = J.nbt;
      pc.gbuf = pool + used;
      pc.shares = J.shares + (t - J.t_begin);
      pcs.push_back(pc);
      used += (int64_t)ns * J.slot_floats;
      nslots += ns;
      tiles += (int64_t)ns * J.tiles_per_triple;
      items += (int64_t)ns * J.nbt;
      t += ns;
      const double kpad = 2.0 * J.pl.kw_chunks * J.pl.kw_elems + 2.0 * J.pl.ko_chunks * J.pl.ko_elems;
      flops += 2.0 * nprod * (double)ns * J.tiles_per_triple * 128.0 * J.pl.NT * kpad;
    }
    if (pcs.empty()) {
      st = fail(TE_ENOMEM, "G pool smaller than one triple's G blocks");
      break;
    }
    size_t smem = 0;
    st = gemm_params(h, jobs, jl, ncl, pcs.data(), (int)pcs.size(), tiles, mode, P, MS, &smem);
    if (st != TE_OK) break;
    std::memset(EL, 0, sizeof(*EL));
    EL->ncl = ncl;
    EL->npieces = (int)pcs.size();
    EL->cw = cw;
    EL->num_sms = h->num_sms;
    EL->nslots = nslots;
    EL->items = items;
    for (int q = 0; q < ncl; ++q) {
      const TcJob& J = jobs[jl[q]];
      EL->cl[q] = EnergyCl{J.o, J.v, (int)energy_num_blocks(J.v), J.nbt, J.c->eps_o, J.c->eps_v};
      EL->map_ovs[q] = &J.em.ovs;
      EL->map_t1[q] = &J.em.t1;
    }
    for (size_t q = 0; q < pcs.size(); ++q) EL->pc[q] = pcs[q];
    EL->triples = h->d_triples;
    EL->partials = partials;
    EL->err = h->d_err;
    EL->wait_ns = h->wait_limit_ns;
    if (h->log)
      std::fprintf(stderr, "[tenergy] round: %d clusters, %zu pieces, %d triples, %lld tiles, %lld energy items\n",
                   ncl, pcs.size(), nslots, (long long)tiles, (long long)items);
    size_t pm = prof_begin(h, 0, s);
    cudaError_t e = launch_gemm_any(mode, *MS, *P, smem, h->num_sms, s);
    prof_end(h, pm, s);
    h->gemm_flops += flops;
    if (e == cudaSuccess) {
      pm = prof_begin(h, 1, s);
      e = launch_energy_tc(*EL, s);
      prof_end(h, pm, s);
    }
    if (e == cudaSuccess)
      e = launch_reduce_pieces(partials, (int)(energy_tc_grid(h->num_sms, items) * ENERGY_TC_WARPS), h->d_triples,
                               pcs.data(), (int)pcs.size(), nslots, s);
    h->n_launches += 3;
    if (e != cudaSuccess) st = fail(TE_ECUDA, "tensor-core path launch: %s", cudaGetErrorString(e));
  }
  delete MS;
  delete P;
  delete EL;
  if (st != TE_OK) return st;
  for (const TcJob& J : jobs) {
    if (!J.e_out) continue;
    ++h->n_launches;
    cudaError_t e = J.t_end > J.t_begin ? launch_reduce_total(J.shares, J.t_end - J.t_begin, J.e_out, s)
                                        : cudaMemsetAsync(J.e_out, 0, sizeof(double), s);
    if (e != cudaSuccess) return fail(TE_ECUDA, "reduction launch: %s", cudaGetErrorString(e));
  }
  return TE_OK;
}

// Plan, buffers (carved from base), operand preparation and maps of one job.
static te_status setup_job(Handle* h, TcState* st, const te_cluster* c, int mode, int64_t t_begin, int64_t t_end,
                           const TcPlan& pl, char* base, TcJob* J, cudaStream_t s, const te_df* df = nullptr,
                           const DfScratch* dfs = nullptr) {
  J->c = c;
  J->pl = pl;
  J->o = (int)c->nocc;
  J->v = (int)c->nvir;
  J->t_begin = t_begin;
  J->t_end = t_end;
  J->nbt = energy_num_block_triples(J->v);
  J->slot_floats = g_slot_floats(J->v, pl.cw);
  J->tiles_per_triple = 3LL * pl.n_mx * pl.n_my * pl.n_nt;
  tc_carve_cluster(base, pl, J->o, J->v, num_unique_triples(J->o), &J->b);
  J->shares = J->b.etri;
  const cudaError_t e = launch_prep_any(mode, c, pl, J->b, df, dfs, h->num_sms, s, &h->n_launches);
  if (e != cudaSuccess) return fail(TE_ECUDA, "operand split launch: %s", cudaGetErrorString(e));
  te_status rs = build_maps(st, pl, J->o, J->v, J->b, &J->maps);
  if (rs != TE_OK) return rs;
  return build_energy_maps(st, pl, J->o, J->v, J->b, &J->em);
}

static te_status check_k(int mode, int o, int v) {
  // exact level-0/1 sums: K = 2 (v + o) products of at most 2^(2 beta) units stay below 2^24
  if (mode == TC_OZAKI6 && 2 * (v + o) > OZ_K_MAX6)
    return fail(TE_EUNSUPPORTED, "OZAKI mode needs 2 (nvir + nocc) <= %d for exact accumulation", OZ_K_MAX6);
  if (mode == TC_OZAKI && 2 * (v + o) > OZ_K_MAX7)
    return fail(TE_EUNSUPPORTED, "7-bit OZAKI slices need 2 (nvir + nocc) <= %d (use 6-bit slices)", OZ_K_MAX7);
  return TE_OK;
}

static TcPool single_pool(const TcPlan& pl, int v) {
  TcPool q;
  q.pool_floats = (int64_t)pl.nslots * g_slot_floats(v, pl.cw);
  q.max_slots = pl.nslots;
  return q;
}

size_t tc_slices_bytes(int o, int v, int ns) {
  const size_t vp = (size_t)round_up(v, 16), op = (size_t)round_up(o, 16), NS = (size_t)ns, es = 2;
  const size_t na = (size_t)o * v * v * vp, nb = (size_t)o * o * v * vp;
  const size_t nl = (size_t)o * v * v * op, nn = (size_t)o * o * v * op;
  auto al = [](size_t b) { return (b + 1023) & ~size_t(1023); };
  const size_t ng = 2 * (size_t)o + 2 * (size_t)o * o;  // row groups of the four arrays
  return al(NS * na * es) + al(NS * nb * es) + al(NS * nl * es) + al(NS * nn * es) + al(ng * 8) + al(ng * 4) + 1024;
}

template <int MODE>
static void launch_slice_set(const te_cluster* c, int vp, int op, const Parts& pa, const Parts& pb, const Parts& pL,
                             const Parts& pN, const int* e_ovvv, const int* e_t2, const int* e_t2L,
                             const int* e_nooT, cudaStream_t s) {
  const int o = (int)c->nocc, v = (int)c->nvir;
  const int64_t v2 = (int64_t)v * v;
  k_split_rows<MODE><<<gridn((int64_t)o * v * v * vp), 256, 0, s>>>(c->ovvv, pa, (int64_t)o * v * v, v, vp, v2,
                                                                    nullptr, 0, e_ovvv);
  k_split_rows<MODE><<<gridn((int64_t)o * o * v * vp), 256, 0, s>>>(c->t2, pb, (int64_t)o * o * v, v, vp,
                                                                    (int64_t)v, nullptr, 1, e_t2);
  k_split_t2L<MODE><<<gridn((int64_t)o * v * v * op), 256, 0, s>>>(c->t2, pL, o, v, op, nullptr, 2, e_t2L);
  k_split_noo<MODE><<<gridn((int64_t)o * o * v * op), 256, 0, s>>>(c->ooov, pN, o, v, op, nullptr, 3, e_nooT);
}

te_status tc_prepare_slices(const te_cluster* c, void* base_v, SliceSet* out, int num_sms, cudaStream_t s,
                            int ns) {
  const int o = (int)c->nocc, v = (int)c->nvir;
  const int vp = round_up(v, 16), op = round_up(o, 16);
  if (ns != 4 && ns != 5) return fail(TE_EINVAL, "slice count %d (4 or 5)", ns);
  const int NS = ns;
  const size_t es = 2;
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(base_v) + 1023) & ~uintptr_t(1023));
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 1023) & ~size_t(1023);
    char* p = base + off;
    off += bytes;
    return p;
  };
  const size_t na = (size_t)o * v * v * vp, nb = (size_t)o * o * v * vp;
  const size_t nl = (size_t)o * v * v * op, nn = (size_t)o * o * v * op;
  char* A = take(NS * na * es);
  char* B = take(NS * nb * es);
  char* L = take(NS * nl * es);
  char* N = take(NS * nn * es);
  const int64_t oo = (int64_t)o * o, ng = 2 * (int64_t)o + 2 * oo;
  auto* maxbits = reinterpret_cast<unsigned long long*>(take((size_t)ng * 8));
  int* exps = reinterpret_cast<int*>(take((size_t)ng * 4));
  int* e_ovvv = exps;           // [o]
  int* e_t2 = e_ovvv + o;       // [o o]
  int* e_t2L = e_t2 + oo;       // [o]
  int* e_nooT = e_t2L + o;      // [o o]
  Parts pa{}, pb{}, pL{}, pN{};
  for (int k = 0; k < NS; ++k) {
    pa.p[k] = A + (size_t)k * v * v * vp * es;
    pb.p[k] = B + (size_t)k * v * vp * es;
    pL.p[k] = L + (size_t)k * v * v * op * es;
    pN.p[k] = N + (size_t)k * v * op * es;
  }
  // one scale per row group (each strided GEMM reads one group of each
  // operand), so a block far below the array's largest keeps its 28 bits
  cudaMemsetAsync(maxbits, 0, (size_t)ng * 8, s);
  const int64_t v2 = (int64_t)v * v, chunk = 65536;
  const int gm = 4 * std::max(1, num_sms);
  k_group_maxabs<<<gm, 256, 0, s>>>(c->ovvv, 0, o, v, v2 * v, o, chunk, maxbits);
  k_group_maxabs<<<gm, 256, 0, s>>>(c->t2, 1, o, v, v2, oo, chunk, maxbits + o);
  k_group_maxabs<<<gm, 256, 0, s>>>(c->t2, 2, o, v, (int64_t)o * v2, o, chunk, maxbits + o + oo);
  k_group_maxabs<<<gm, 256, 0, s>>>(c->ooov, 3, o, v, (int64_t)o * v, oo, chunk, maxbits + 2 * o + oo);
  k_group_exps<<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(maxbits, ng, exps);
  if (NS == 5) launch_slice_set<TC_SLICE5>(c, vp, op, pa, pb, pL, pN, e_ovvv, e_t2, e_t2L, e_nooT, s);
  else launch_slice_set<TC_SLICE4>(c, vp, op, pa, pb, pL, pN, e_ovvv, e_t2, e_t2L, e_nooT, s);
  if (cudaGetLastError() != cudaSuccess) return fail(TE_ECUDA, "slice preparation launch failed");
  out->ovvv = A;
  out->t2 = B;
  out->t2L = L;
  out->nooT = N;
  out->ovvv_plane = (int64_t)v * v * vp;
  out->t2_plane = (int64_t)v * vp;
  out->t2L_plane = (int64_t)v * v * op;
  out->nooT_plane = (int64_t)v * op;
  out->ovvv_p = NS * (int64_t)v * v * vp;
  out->t2_rq = NS * (int64_t)v * vp;
  out->t2L_q = NS * (int64_t)v * v * op;
  out->nooT_pr = NS * (int64_t)v * op;
  out->vp = vp;
  out->op = op;
  out->ns = NS;
  out->e_ovvv = e_ovvv;
  out->e_t2 = e_t2;
  out->e_t2L = e_t2L;
  out->e_nooT = e_nooT;
  return TE_OK;
}

te_status tc_workspace_bytes(Handle* h, const te_cluster* c, te_precision p, size_t* bytes, const te_df* df) {
  const int o = (int)c->nocc, v = (int)c->nvir;
  const TcPlan pl = make_plan(h, o, v, tc_mode_of(p, o, v, h->ozaki_bits), num_unique_triples(c->nocc));
  TcBuffers b;
  DfScratch d;
  const size_t region = std::max(tc_shared_bytes(single_pool(pl, v), h->num_sms),
                                 df ? df_carve(nullptr, o, v, df->naux, h->num_sms, &d) : size_t(0));
  *bytes = tc_carve_cluster(nullptr, pl, o, v, num_unique_triples(o), &b) + region;
  return TE_OK;
}

te_status ensure_workspace_public(Handle* h, size_t bytes);
te_status ensure_triples_public(Handle* h, int nocc);

te_status tc_autotune(Handle* h, const te_cluster* c, te_precision p, cudaStream_t s) {
  const int o = (int)c->nocc, v = (int)c->nvir, mode = tc_mode_of(p, o, v, h->ozaki_bits);
  const auto key = std::make_tuple(o, v, mode);
  if (h->tuned.count(key)) return TE_OK;
  if (check_k(mode, o, v) != TE_OK) return TE_OK;  // run_tc reports it
  const int64_t nt = num_unique_triples(o);
  if (nt == 0) return TE_OK;
  // candidate M tiles: padding within 15% of the least; candidate N splits: the fewest and one more
  std::vector<std::pair<int, int>> cand;
  int64_t best_rows = -1;
  for (int TB = 128; TB >= 16; TB /= 2) {
    const int TA = 128 / TB;
    const int64_t rows = (int64_t)round_up(v, TA) * round_up(v, TB);
    if (best_rows < 0 || rows < best_rows) best_rows = rows;
  }
  const TcPlan base = make_plan(h, o, v, mode, nt, 128, 0);
  for (int TB = 128; TB >= 16; TB /= 2) {
    const int TA = 128 / TB;
    const int64_t rows = (int64_t)round_up(v, TA) * round_up(v, TB);
    if (rows * 100 > best_rows * 115) continue;
    cand.emplace_back(TB, base.n_nt);
    // one more N split (smaller N tiles re-read the A operand more often), and
    // in the exact-slice modes the fewer splits of 160-column tiles, which do
    // not rotate their TMEM blocks
    if (round_up((v + base.n_nt) / (base.n_nt + 1), 16) >= 32) cand.emplace_back(TB, base.n_nt + 1);
    const int n160 = (v + 159) / 160;
    if (is_ozaki(mode) && n160 < base.n_nt) cand.emplace_back(TB, n160);
  }
  if (cand.size() <= 1) {
    if (!cand.empty()) h->tuned[key] = cand[0];
    return TE_OK;
  }
  const auto cached = h->tune_file.find(key);  // a cache file's pick, if it is one of these
  if (cached != h->tune_file.end() && std::find(cand.begin(), cand.end(), cached->second) != cand.end()) {
    h->tuned[key] = cached->second;
    return TE_OK;
  }
  TcState* st = tc_state(h);
  te_status rs = get_encoder(st);
  if (rs != TE_OK) return rs;
  rs = ensure_triples_public(h, o);
  if (rs != TE_OK) return rs;
  size_t need = 0;
  for (const auto& cd : cand) {
    const TcPlan pl = make_plan(h, o, v, mode, nt, cd.first, cd.second);
    TcBuffers b;
    need = std::max(need, tc_carve_cluster(nullptr, pl, o, v, nt, &b) + tc_shared_bytes(single_pool(pl, v), h->num_sms));
  }
  rs = ensure_workspace_public(h, need);
  if (rs != TE_OK) return rs;
  char* wbase = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(h->ws) + 1023) & ~uintptr_t(1023));
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(TE_ECUDA, "event creation failed");
  float best_ms = 1e30f;
  std::pair<int, int> best = cand[0];
  bool prepped = false;
  std::vector<TcJob> jobs(1);
  TcMapSet* MS = new TcMapSet;
  TcParams* P = new TcParams;
  for (const auto& cd : cand) {
    const TcPlan pl = make_plan(h, o, v, mode, nt, cd.first, cd.second);
    if (pl.stages < 2) continue;
    TcJob& J = jobs[0];
    J = TcJob{};
    J.c = c;
    J.pl = pl;
    J.o = o;
    J.v = v;
    J.nbt = energy_num_block_triples(v);
    J.slot_floats = g_slot_floats(v, pl.cw);
    J.tiles_per_triple = 3LL * pl.n_mx * pl.n_my * pl.n_nt;
    const size_t cbytes = tc_carve_cluster(wbase, pl, o, v, nt, &J.b);
    cudaError_t e = cudaSuccess;
    if (!prepped) {  // the operand planes sit first in the workspace for every candidate
      e = launch_prep_any(mode, c, pl, J.b, nullptr, nullptr, h->num_sms, s, &h->n_launches);
      prepped = true;
    }
    if (e != cudaSuccess || build_maps(st, pl, o, v, J.b, &J.maps) != TE_OK) continue;
    const int ns = (int)std::min<int64_t>(pl.nslots, nt);
    TcPiece pc{};
    pc.cl = 0;
    pc.ns = ns;
    pc.nbt = J.nbt;
    pc.gbuf = reinterpret_cast<float*>(wbase + cbytes);
    const int jl[1] = {0};
    size_t smem = 0;
    if (gemm_params(h, jobs, jl, 1, &pc, 1, (int64_t)ns * J.tiles_per_triple, mode, P, MS, &smem) != TE_OK) continue;
    float ms = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0, s);
      e = launch_gemm_any(mode, *MS, *P, smem, h->num_sms, s);
      cudaEventRecord(e1, s);
      h->n_launches += 1;
      if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) break;
      float tms = 0.f;
      cudaEventElapsedTime(&tms, e0, e1);
      ms = std::min(ms, tms / (float)ns);  // per triple
    }
    if (h->log)
      std::fprintf(stderr, "[tenergy] autotune nocc=%d nvir=%d mode=%d: TB=%d n_nt=%d %.4f ms per triple\n", o, v,
                   mode, cd.first, cd.second, (double)ms);
    if (ms < best_ms) {
      best_ms = ms;
      best = cd;
    }
  }
  delete MS;
  delete P;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess) return fail(TE_ECUDA, "autotune launch failed");
  h->tuned[key] = best;
  if (h->log)
    std::fprintf(stderr, "[tenergy] autotune nocc=%d nvir=%d mode=%d: picked TB=%d n_nt=%d\n", o, v, mode,
                 best.first, best.second);
  tune_save(h);
  return TE_OK;
}

te_status run_tc(Handle* h, const te_cluster* c, te_precision p, int64_t t_begin, int64_t t_end,
                 double* e_tri_out, double* e_total_out, cudaStream_t s, const te_df* df) {
  if (h->cc_major != 10 && h->cc_major != 11)
    return fail(TE_EUNSUPPORTED, "tensor-core modes need an sm_100-family GPU (found sm_%d%d)", h->cc_major,
                h->cc_minor);
  TcState* st = tc_state(h);
  te_status rs = get_encoder(st);
  if (rs != TE_OK) return rs;
  const int o = (int)c->nocc, v = (int)c->nvir;
  const int mode = tc_mode_of(p, o, v, h->ozaki_bits);
  const int64_t ntri = num_unique_triples(o);
  const TcPlan pl = make_plan(h, o, v, mode, t_end - t_begin);
  if (pl.stages < 2) return fail(TE_EUNSUPPORTED, "not enough shared memory for two pipeline stages");
  rs = check_k(mode, o, v);
  if (rs != TE_OK) return rs;
  TcBuffers b;
  const TcPool pq = single_pool(pl, v);
  const size_t cbytes = tc_carve_cluster(nullptr, pl, o, v, ntri, &b);
  DfScratch dfs;
  const size_t bytes = cbytes + std::max(tc_shared_bytes(pq, h->num_sms),
                                         df ? df_carve(nullptr, o, v, df->naux, h->num_sms, &dfs) : size_t(0));
  if (h->log)
    std::fprintf(stderr,
                 "[tenergy] plan nocc=%d nvir=%d mode=%d: M tile %d x %d, N tile %d (%d per row block), %d stages "
                 "of %u bytes, %d triples per launch, %u TMEM columns (%d accumulator sets), workspace %zu bytes\n",
                 o, v, mode, pl.TA, pl.TB, pl.NT, pl.n_nt, pl.stages, pl.stage_bytes, pl.nslots, pl.tmem_cols,
                 pl.nbuf, bytes);
  rs = ensure_workspace_public(h, bytes);
  if (rs != TE_OK) return rs;
  rs = ensure_triples_public(h, o);
  if (rs != TE_OK) return rs;
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(h->ws) + 1023) & ~uintptr_t(1023));
  std::vector<TcJob> jobs(1);
  if (df) df_carve(base + cbytes, o, v, df->naux, h->num_sms, &dfs);  // over the G pool, before its first use
  rs = setup_job(h, st, c, mode, t_begin, t_end, pl, base, &jobs[0], s, df, df ? &dfs : nullptr);
  if (rs != TE_OK) return rs;
  if (e_tri_out) jobs[0].shares = e_tri_out;  // shares[t - t_begin]
  else jobs[0].shares = jobs[0].b.etri;
  jobs[0].e_out = e_total_out;
  float* pool = reinterpret_cast<float*>(base + cbytes);
  double* partials = reinterpret_cast<double*>(base + cbytes + (((size_t)pq.pool_floats * 4 + 1023) & ~size_t(1023)));
  return run_rounds(h, jobs, mode, pool, pq, partials, s);
}

// Batches: every member's operands prepared up front, then rounds that mix
// members (largest first), so the whole batch takes a few launches per round
// instead of three per member per slot group.
static constexpr int64_t BATCH_POOL_BYTES = int64_t(16) << 30;

static TcPool batch_pool(Handle* h, const te_cluster* cs, int64_t n, int mode_p) {
  int64_t need = 0, biggest = 0;
  int cw = 1;
  for (int64_t x = 0; x < n; ++x) {
    const int o = (int)cs[x].nocc, v = (int)cs[x].nvir;
    const int mode = tc_mode_of((te_precision)mode_p, o, v, h->ozaki_bits);
    cw = is_ozaki(mode) ? 2 : 1;
    const int64_t sf = g_slot_floats(v, cw);
    need += num_unique_triples(o) * sf;
    biggest = std::max(biggest, sf);
  }
  TcPool q;
  q.pool_floats = std::max(biggest, std::min<int64_t>(need, BATCH_POOL_BYTES / 4));
  q.max_slots = 2048;
  return q;
}

te_status tc_batched_bytes(Handle* h, const te_cluster* cs, int64_t n, te_precision p, size_t* bytes) {
  size_t b = 0;
  for (int64_t x = 0; x < n; ++x) {
    const int o = (int)cs[x].nocc, v = (int)cs[x].nvir;
    const TcPlan pl = make_plan(h, o, v, tc_mode_of(p, o, v, h->ozaki_bits), num_unique_triples(o));
    TcBuffers bb;
    b += tc_carve_cluster(nullptr, pl, o, v, num_unique_triples(o), &bb);
  }
  *bytes = b + tc_shared_bytes(batch_pool(h, cs, n, (int)p), h->num_sms) + 1024;
  return TE_OK;
}

te_status run_tc_batched(Handle* h, const te_cluster* cs, int64_t n, te_precision p, double* e_out, cudaStream_t s) {
  if (h->cc_major != 10 && h->cc_major != 11)
    return fail(TE_EUNSUPPORTED, "tensor-core modes need an sm_100-family GPU (found sm_%d%d)", h->cc_major,
                h->cc_minor);
  TcState* st = tc_state(h);
  te_status rs = get_encoder(st);
  if (rs != TE_OK) return rs;
  size_t bytes = 0;
  tc_batched_bytes(h, cs, n, p, &bytes);
  rs = ensure_workspace_public(h, bytes);
  if (rs != TE_OK) return rs;
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(h->ws) + 1023) & ~uintptr_t(1023));
  // longest first: the rounds' last pieces are the small members
  std::vector<int64_t> order(n);
  for (int64_t x = 0; x < n; ++x) order[x] = x;
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    const double fa = (double)num_unique_triples(cs[a].nocc) * cs[a].nvir * cs[a].nvir * cs[a].nvir * (cs[a].nvir + cs[a].nocc);
    const double fb = (double)num_unique_triples(cs[b].nocc) * cs[b].nvir * cs[b].nvir * cs[b].nvir * (cs[b].nvir + cs[b].nocc);
    return fa > fb;
  });
  std::vector<TcJob> jobs;
  std::vector<int> modes;
  jobs.reserve(n);
  size_t off = 0;
  for (int64_t x : order) {
    const int o = (int)cs[x].nocc, v = (int)cs[x].nvir;
    const int mode = tc_mode_of(p, o, v, h->ozaki_bits);
    rs = check_k(mode, o, v);
    if (rs != TE_OK) return rs;
    const int64_t nt = num_unique_triples(o);
    if (nt == 0) {
      if (cudaMemsetAsync(e_out + x, 0, sizeof(double), s) != cudaSuccess) return fail(TE_ECUDA, "memset failed");
      ++h->n_launches;
      continue;
    }
    const TcPlan pl = make_plan(h, o, v, mode, nt);
    TcJob J;
    rs = setup_job(h, st, cs + x, mode, 0, nt, pl, base + off, &J, s);
    if (rs != TE_OK) return rs;
    TcBuffers bb;
    off += tc_carve_cluster(nullptr, pl, o, v, nt, &bb);
    J.e_out = e_out + x;
    jobs.push_back(J);
    modes.push_back(mode);
  }
  const TcPool pq = batch_pool(h, cs, n, (int)p);
  float* pool = reinterpret_cast<float*>(base + off);
  double* partials = reinterpret_cast<double*>(base + off + (((size_t)pq.pool_floats * 4 + 1023) & ~size_t(1023)));
  // one kernel per mode: the members of each slice width run in their own rounds
  for (int mode : {TC_TF32, TC_BF16X3, TC_TF32X3, TC_OZAKI, TC_OZAKI6}) {
    std::vector<TcJob> group;
    for (size_t q = 0; q < jobs.size(); ++q)
      if (modes[q] == mode) group.push_back(jobs[q]);
    if (group.empty()) continue;
    rs = run_rounds(h, group, mode, pool, pq, partials, s);
    if (rs != TE_OK) return rs;
  }
  return TE_OK;
}

}  // namespace te
