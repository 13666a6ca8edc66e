// Exact-slice contractions on tcgen05 over tensor-map views (see view_tc.h).
//
// Warp roles of the persistent kernel: warp 0 issues the TMA copies (one
// five-dimensional box per operand slice and stage), one thread of warp 1
// issues tcgen05.mma into three FP32 accumulators in tensor memory, warps 2..9
// (two per TMEM lane quarter, half of the N tile each) drain every
// accumulation block into a double-float (FP32 pair) sum held in registers and
// release the accumulators at once, so the next block's MMAs overlap the rest
// of the epilogue.  A unit's sum goes to float64 once, at its end: GB300's
// float64 rate is a small fraction of its FP32 rate, and a float64 update per
// block and element cost more than the MMAs at short K.
// Shared memory per stage: the A slices (128 rows of 64 bytes each, 64-byte
// swizzle, K-major) then the B slices (NT rows each).  Every wait is bounded;
// on expiry the kernel records the error word and unwinds.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "ptx_sm100.cuh"
#include "tc_path.h"
#include "view_tc.h"

namespace te {

namespace {

constexpr int VT_EPI_WARPS = 8;
constexpr int VT_WARPS = 2 + VT_EPI_WARPS;
constexpr int VT_THREADS = VT_WARPS * 32;
constexpr int VT_HALF = VT_NT_MAX / 2;  // columns one epilogue thread holds
constexpr uint32_t VT_ROW_BYTES = VT_KC * 2;         // 64
constexpr uint32_t VT_A_SLICE = 128u * VT_ROW_BYTES;  // 8 KB

struct VtUnit {
  int job, split, m1_0, m2_0, n0;
  int64_t b_begin, b_end;
};

__device__ __forceinline__ VtUnit vt_decode(const VtParams& P, int64_t u) {
  VtUnit U;
  int j = 0;
  while (j + 1 < P.njobs && P.job[j + 1].unit0 <= u) ++j;
  const VtJob& J = P.job[j];
  int64_t l = u - J.unit0;
  U.job = j;
  U.split = (int)(l % J.nsplit);
  l /= J.nsplit;
  const int nt = (int)(l % J.nn);
  l /= J.nn;
  const int m2t = (int)(l % J.nm2);
  const int m1t = (int)(l / J.nm2);
  U.m1_0 = m1t * J.TA;
  U.m2_0 = m2t * J.TB;
  U.n0 = nt * J.NT;
  U.b_begin = J.nblocks * U.split / J.nsplit;
  U.b_end = J.nblocks * (U.split + 1) / J.nsplit;
  return U;
}

// segment and chunk range [c0, c1) of the job's accumulation block b
__device__ __forceinline__ int vt_block(const VtJob& J, int64_t b, int* c0, int* c1) {
  int s = 0;
  while (s + 1 < J.nseg && b >= J.seg[s].nblk) {
    b -= J.seg[s].nblk;
    ++s;
  }
  *c0 = (int)b * J.seg[s].bchunks;
  *c1 = min(*c0 + J.seg[s].bchunks, J.seg[s].nchunks);
  return s;
}

__device__ __forceinline__ void vt_load(void* dst, const CUtensorMap* map, const VtRoles& R, const int* fix, int kc,
                                        int r2, int r1, int k1, int sl, uint64_t* bar) {
  int c[5];
#pragma unroll
  for (int d = 0; d < 5; ++d) {
    int x = fix[d];
    if (d == R.k2) x = kc;
    if (d == R.r2) x = r2;
    if (d == R.r1) x = r1;
    if (d == R.k1) x = k1;
    if (d == R.s) x = sl;
    c[d] = x;
  }
  ptx::tma_load_5d(dst, map, bar, c[0], c[1], c[2], c[3], c[4]);
}

__device__ __forceinline__ void vt_abort(const VtParams& P, volatile int* abort_flag, unsigned site) {
  *abort_flag = 1;
  if (atomicOr(P.err, ERR_WAIT_TIMEOUT) == 0) {
    P.err[1] = site;
    P.err[2] = blockIdx.x;
  }
}

template <int NS>
__global__ void __launch_bounds__(VT_THREADS, 1)
    k_view_tc(const __grid_constant__ VtMaps maps, const __grid_constant__ VtParams P) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)P.stages * P.stage_bytes);
  uint64_t* empty = full + P.stages;
  uint64_t* tfull = empty + P.stages;
  uint64_t* tempty = tfull + 1;
  uint64_t* drain = tempty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < P.stages; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    ptx::mbar_init(tfull, 1);
    ptx::mbar_init(tempty, VT_EPI_WARPS);
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_barrier_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, P.tmem_cols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      uint32_t stage = 0, phase = 0;
      int pending[8];
      for (int s = 0; s < 8; ++s) pending[s] = -1;
      bool ok = true;
      for (int64_t u = blockIdx.x; ok && u < P.total_units; u += gridDim.x) {
        const VtUnit U = vt_decode(P, u);
        const VtJob& J = P.job[U.job];
        const uint32_t bytes = (uint32_t)NS * (VT_A_SLICE + (uint32_t)J.NT * VT_ROW_BYTES);
        for (int64_t b = U.b_begin; ok && b < U.b_end; ++b) {
          int c0, c1;
          const VtSeg& S = J.seg[vt_block(J, b, &c0, &c1)];
          const VtRoles& RA = P.roles[S.amap];
          const VtRoles& RB = P.roles[S.bmap];
          for (int c = c0; c < c1; ++c) {
            if (*abort_flag || !ptx::mbar_wait(&empty[stage], phase ^ 1u, P.wait_ns)) {
              if (!*abort_flag) vt_abort(P, abort_flag, 21);
              ok = false;
              break;
            }
            ptx::mbar_arrive_expect_tx(&full[stage], bytes);
            pending[stage] = (int)phase;
            unsigned char* sa = smem + (size_t)stage * P.stage_bytes;
            unsigned char* sb = sa + NS * VT_A_SLICE;
            const int k1 = c / S.nk2c;
            const int kc = (c - k1 * S.nk2c) * VT_KC;
#pragma unroll
            for (int sl = 0; sl < NS; ++sl) {
              vt_load(sa + sl * VT_A_SLICE, &maps.m[S.amap], RA, S.afix, kc, U.m2_0, U.m1_0, k1, sl, &full[stage]);
              vt_load(sb + sl * (uint32_t)J.NT * VT_ROW_BYTES, &maps.m[S.bmap], RB, S.bfix, kc, U.n0, 0, k1, sl,
                      &full[stage]);
            }
            if (++stage == (uint32_t)P.stages) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
      }
      // copies still in flight land before the CTA exits
      for (int s = 0; s < P.stages; ++s)
        if (pending[s] >= 0) ptx::mbar_wait(&full[s], (uint32_t)pending[s], P.wait_ns);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      uint32_t stage = 0, phase = 0, acc_phase = 0;
      bool ok = true, issued = false;
      const uint32_t sbo = 8u * VT_ROW_BYTES;  // 8 rows of the 64-byte swizzle
      for (int64_t u = blockIdx.x; ok && u < P.total_units; u += gridDim.x) {
        const VtUnit U = vt_decode(P, u);
        const VtJob& J = P.job[U.job];
        // kind::f16, BF16 A and B (K-major), FP32 accumulation, M = 128, N = NT
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(J.NT >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
        const uint32_t d0 = tmem_base, d1 = tmem_base + (uint32_t)J.NT, dr = tmem_base + 2u * (uint32_t)J.NT;
        for (int64_t b = U.b_begin; ok && b < U.b_end; ++b) {
          int c0, c1;
          vt_block(J, b, &c0, &c1);
          if (*abort_flag || !ptx::mbar_wait(tempty, acc_phase ^ 1u, P.wait_ns)) {
            if (!*abort_flag) vt_abort(P, abort_flag, 22);
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          uint32_t first = 1;
          for (int c = c0; c < c1; ++c) {
            if (*abort_flag || !ptx::mbar_wait(&full[stage], phase, P.wait_ns)) {
              if (!*abort_flag) vt_abort(P, abort_flag, 23);
              ok = false;
              break;
            }
            ptx::tc_fence_after();
            unsigned char* sa = smem + (size_t)stage * P.stage_bytes;
            const uint32_t a0 = ptx::smem_u32(sa);
            const uint32_t b0 = ptx::smem_u32(sa + NS * VT_A_SLICE);
#pragma unroll
            for (int ks = 0; ks < VT_KC / 16; ++ks) {
              uint64_t ad[NS], bd[NS];
#pragma unroll
              for (int k = 0; k < NS; ++k) {
                ad[k] = ptx::smem_desc(a0 + k * VT_A_SLICE + ks * 32, sbo, 4u);
                bd[k] = ptx::smem_desc(b0 + k * (uint32_t)J.NT * VT_ROW_BYTES + ks * 32, sbo, 4u);
              }
              // slice products a_i b_j, i + j <= NS - 1: level 0 and level 1 in
              // their own (exact) accumulators, the higher levels in a third
              const uint32_t acc_in = first ? 0u : 1u;
              ptx::mma<false>(d0, ad[0], bd[0], idesc, acc_in);
              ptx::mma<false>(d1, ad[0], bd[1], idesc, acc_in);
              ptx::mma<false>(d1, ad[1], bd[0], idesc, 1);
              uint32_t rin = acc_in;
#pragma unroll
              for (int lev = 2; lev < NS; ++lev)
#pragma unroll
                for (int i = 0; i <= lev; ++i) {
                  ptx::mma<false>(dr, ad[i], bd[lev - i], idesc, rin);
                  rin = 1;
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
          if (!ok) break;
          ptx::mma_commit(tfull);
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
    // ---------------- epilogue: TMEM -> double-float -> float64 ----------------
    const int quad = warp & 3;               // the lane quarter this warp may read
    const int half = (warp - 2) >> 2;        // which half of the N tile
    const int row = quad * 32 + lane;
    const uint32_t tbase = tmem_base + ((uint32_t)(quad * 32) << 16);
    uint32_t acc_phase = 0;
    bool ok = true;
    for (int64_t u = blockIdx.x; ok && u < P.total_units; u += gridDim.x) {
      const VtUnit U = vt_decode(P, u);
      const VtJob& J = P.job[U.job];
      const int m1 = U.m1_0 + row / J.TB, m2 = U.m2_0 + row % J.TB;
      const bool valid = m1 < J.M1 && m2 < J.M2;
      const int ncol = J.NT >> 1, c_lo = half * ncol;
      // the unit's sum is kept relative to 2^eref, the largest scale of the
      // job's segments: every block's weight 2^(e - eref) <= 1 is exact in FP32
      int eref = -100000;
      for (int q = 0; q < J.nseg; ++q) eref = max(eref, *J.seg[q].ea + *J.seg[q].eb);
      float hi[VT_HALF], lo[VT_HALF];
#pragma unroll
      for (int q = 0; q < VT_HALF; ++q) {
        hi[q] = 0.f;
        lo[q] = 0.f;
      }
      for (int64_t b = U.b_begin; b < U.b_end; ++b) {
        int c0, c1;
        const VtSeg& S = J.seg[vt_block(J, b, &c0, &c1)];
        int got = 0;
        if (!*abort_flag) got = ptx::mbar_wait(tfull, acc_phase, P.wait_ns) ? 1 : 0;
        // warp-uniform: tcgen05.ld below is .sync.aligned
        if (!__all_sync(0xffffffffu, got)) {
          if (!*abort_flag && lane == 0) vt_abort(P, abort_flag, 24);
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        const float wk = ldexpf(S.alpha < 0.0 ? -1.f : 1.f, *S.ea + *S.eb - eref);
#pragma unroll
        for (int q = 0; q < VT_HALF / 8; ++q) {
          if (8 * q < ncol) {
            const uint32_t cc = (uint32_t)(c_lo + 8 * q);
            float a0[8], a1[8], a2[8];
            ptx::tmem_ld8x3(tbase + cc, tbase + (uint32_t)J.NT + cc, tbase + 2u * (uint32_t)J.NT + cc, a0, a1, a2);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              // level 0 + level 1 exactly (both exact FP32 sums), the rest rounded
              const float s0 = __fadd_rn(a0[j], a1[j]);
              const float bb = __fsub_rn(s0, a0[j]);
              const float e0 = __fadd_rn(__fsub_rn(a0[j], __fsub_rn(s0, bb)), __fsub_rn(a1[j], bb));
              const float x = __fmul_rn(s0, wk), y = __fmul_rn(__fadd_rn(e0, a2[j]), wk);
              // (hi, lo) += (x, y)
              const float t = __fadd_rn(hi[8 * q + j], x);
              const float tb = __fsub_rn(t, hi[8 * q + j]);
              const float te = __fadd_rn(__fsub_rn(hi[8 * q + j], __fsub_rn(t, tb)), __fsub_rn(x, tb));
              const float l = __fadd_rn(te, __fadd_rn(lo[8 * q + j], y));
              hi[8 * q + j] = __fadd_rn(t, l);
              lo[8 * q + j] = __fsub_rn(l, __fsub_rn(hi[8 * q + j], t));
            }
          }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(tempty);
        acc_phase ^= 1u;
      }
      if (!ok || !valid) continue;
      const double scale = ldexp(J.jalpha, eref);
      double* dst;
      int64_t dn;
      const bool store = J.nsplit > 1 || J.overwrite;
      if (J.nsplit > 1) {
        dst = J.part + ((int64_t)U.split * ((int64_t)J.M1 * J.M2) + (int64_t)m1 * J.M2 + m2) * J.N;
        dn = 1;
      } else {
        dst = J.C + (int64_t)m1 * J.c_m1 + (int64_t)m2 * J.c_m2;
        dn = J.c_n;
      }
#pragma unroll
      for (int q = 0; q < VT_HALF / 8; ++q) {
        if (8 * q < ncol) {
          const int n0 = U.n0 + c_lo + 8 * q;
          double old[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) old[j] = (!store && n0 + j < J.N) ? dst[(int64_t)(n0 + j) * dn] : 0.0;
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (n0 + j < J.N)
              dst[(int64_t)(n0 + j) * dn] = fma(scale, (double)hi[8 * q + j] + (double)lo[8 * q + j], old[j]);
        }
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

// C[(m1, m2), n] += sum_z part[z][(m1, m2)][n], z in order, for every split job
// of a launch (one index space over their outputs)
__global__ void __launch_bounds__(256) k_vt_reduce(const __grid_constant__ VtParams P) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P.total_red;
       e += (int64_t)gridDim.x * blockDim.x) {
    int j = 0;
    while (P.job[j].nsplit <= 1 || e >= P.job[j].red0 + (int64_t)P.job[j].M1 * P.job[j].M2 * P.job[j].N) ++j;
    const VtJob& J = P.job[j];
    const int64_t total = (int64_t)J.M1 * J.M2 * J.N, x = e - J.red0;
    double s = 0.0;
#pragma unroll 8
    for (int z = 0; z < J.nsplit; ++z) s += J.part[z * total + x];
    const int64_t m = x / J.N;
    const int n = (int)(x - m * J.N);
    double* cp = J.C + (m / J.M2) * J.c_m1 + (m % J.M2) * J.c_m2 + (int64_t)n * J.c_n;
    *cp += s;
  }
}

// dst[p][b][c][r] = src[p][b][r][c] through a 64 x 64 shared tile; pairs of
// BF16 elements move as one 32-bit access when every offset is even (`pairs`)
__global__ void __launch_bounds__(256) k_vt_transpose(const unsigned short* __restrict__ src, int64_t src_ps,
                                                       int64_t src_bs, int64_t src_rs, unsigned short* __restrict__ dst,
                                                       int64_t dst_ps, int64_t dst_bs, int64_t dst_cs, int nb, int R,
                                                       int Cc, int pairs) {
  __shared__ unsigned short tile[64][65];
  const int pb = blockIdx.z, p = pb / nb, b = pb - p * nb;
  const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
  const unsigned short* s = src + p * src_ps + b * src_bs;
  unsigned short* d = dst + p * dst_ps + b * dst_bs;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int i = ty; i < 64; i += 8) {
    const int r = r0 + i, c = c0 + 2 * tx;
    if (r >= R) continue;
    const unsigned short* sr = s + r * src_rs;
    if (pairs && c + 1 < Cc) {
      const unsigned int w = *reinterpret_cast<const unsigned int*>(sr + c);
      tile[i][2 * tx] = (unsigned short)(w & 0xffffu);
      tile[i][2 * tx + 1] = (unsigned short)(w >> 16);
    } else {
      if (c < Cc) tile[i][2 * tx] = sr[c];
      if (c + 1 < Cc) tile[i][2 * tx + 1] = sr[c + 1];
    }
  }
  __syncthreads();
  for (int i = ty; i < 64; i += 8) {
    const int c = c0 + i, r = r0 + 2 * tx;
    if (c >= Cc) continue;
    unsigned short* dc = d + c * dst_cs;
    if (pairs && r + 1 < R) {
      *reinterpret_cast<unsigned int*>(dc + r) = (unsigned int)tile[2 * tx][i] | ((unsigned int)tile[2 * tx + 1][i] << 16);
    } else {
      if (r < R) dc[r] = tile[2 * tx][i];
      if (r + 1 < R) dc[r + 1] = tile[2 * tx + 1][i];
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 vt_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (fn) return fn;
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !p) {
    cudaGetLastError();
    return nullptr;
  }
  fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  return fn;
}

}  // namespace

void vt_begin(VtBuild* b, int ns) {
  std::memset(b, 0, sizeof(*b));
  b->P.ns = ns;
  for (int q = 0; q < VT_BANK_MAX; ++q) b->slot[q] = -1;
}

te_status vt_bank_add(VtBank* k, const VtView& v, int rows_r2, int rows_r1, int* idx) {
  if (k->n >= VT_BANK_MAX) return fail(TE_EINVAL, "view GEMM: more than %d tensor maps", VT_BANK_MAX);
  const VtRoles& R = v.roles;
  if (R.k2 != 0 || v.stride[0] != 1 || R.r2 <= 0 || R.s <= 0 || (R.r1 >= 0 && R.r1 < R.r2))
    return fail(TE_EINVAL, "view GEMM: bad view roles");
  if ((reinterpret_cast<uintptr_t>(v.base) & 15) != 0) return fail(TE_EINVAL, "view GEMM: base not 16-byte aligned");
  if (rows_r2 < 1 || rows_r2 > 256 || rows_r1 < 1 || rows_r1 > 256) return fail(TE_EINVAL, "view GEMM: box rows");
  PFN_cuTensorMapEncodeTiled_v12000 enc = vt_encoder();
  if (!enc) return fail(TE_ECUDA, "cuTensorMapEncodeTiled entry point not available");
  cuuint64_t gd[5], gs[4];
  cuuint32_t box[5], e1[5];
  uint64_t smax = 16;
  for (int d = 1; d < 5; ++d)
    if (v.dims[d] > 1) smax = std::max<uint64_t>(smax, v.stride[d] * 2);
  for (int d = 0; d < 5; ++d) {
    gd[d] = std::max<uint64_t>(1, v.dims[d]);
    box[d] = 1;
    e1[d] = 1;
    if (d >= 1) {
      const uint64_t sb = v.dims[d] > 1 ? v.stride[d] * 2 : smax;
      if (sb % 16 != 0 || sb >= (1ull << 40)) return fail(TE_EINVAL, "view GEMM: stride of dimension %d", d);
      gs[d - 1] = sb;
    }
  }
  box[R.k2] = VT_KC;
  box[R.r2] = (cuuint32_t)rows_r2;
  if (R.r1 >= 0) box[R.r1] = (cuuint32_t)rows_r1;
  CUtensorMap* m = &k->m[k->n];
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(v.base), gd, gs, box, e1,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(TE_ECUDA, "view GEMM: tensor map encoding failed (CUresult %d)", (int)r);
  k->r[k->n] = R;
  *idx = k->n++;
  return TE_OK;
}

int vt_use(VtBuild* b, const VtBank& k, int idx) {
  if (idx < 0 || idx >= k.n) return -1;
  if (b->slot[idx] >= 0) return b->slot[idx];
  if (b->nmaps >= VT_MAX_MAPS) return -1;
  b->maps.m[b->nmaps] = k.m[idx];
  b->P.roles[b->nmaps] = k.r[idx];
  b->slot[idx] = (int8_t)b->nmaps;
  return b->nmaps++;
}

int64_t vt_seg_blocks(int K1, int K2, int bchunks) {
  const int64_t nchunks = (int64_t)K1 * ((K2 + VT_KC - 1) / VT_KC);
  return (nchunks + bchunks - 1) / bchunks;
}

VtJob* vt_job(VtBuild* b, int M1, int M2, int N, int TA, int TB, int NT, double* C, int64_t c_m1, int64_t c_m2,
              int64_t c_n, int overwrite) {
  if (b->P.njobs >= VT_MAX_JOBS) return nullptr;
  VtJob* j = &b->P.job[b->P.njobs++];
  std::memset(j, 0, sizeof(*j));
  j->M1 = M1;
  j->M2 = M2;
  j->N = N;
  j->TA = TA;
  j->TB = TB;
  j->NT = NT;
  j->nm1 = (M1 + TA - 1) / TA;
  j->nm2 = (M2 + TB - 1) / TB;
  j->nn = (N + NT - 1) / NT;
  j->nsplit = 1;
  j->C = C;
  j->c_m1 = c_m1;
  j->c_m2 = c_m2;
  j->c_n = c_n;
  j->overwrite = overwrite;
  j->jalpha = 1.0;
  return j;
}

void vt_seg(VtJob* j, int amap, int bmap, int K1, int K2, const int* afix, const int* bfix, const int* ea,
            const int* eb, double alpha) {
  if (j->nseg >= VT_MAX_SEGS) {  // vt_finish reports it
    j->seg[0].amap = -1;
    return;
  }
  VtSeg& s = j->seg[j->nseg++];
  s.amap = (int8_t)amap;
  s.bmap = (int8_t)bmap;
  s.K1 = K1;
  s.K2 = K2;
  s.nk2c = (K2 + VT_KC - 1) / VT_KC;
  s.nchunks = K1 * s.nk2c;
  s.bchunks = VT_BLOCK_CHUNKS;
  s.nblk = (int)vt_seg_blocks(K1, K2);
  for (int d = 0; d < 5; ++d) {
    s.afix[d] = afix ? afix[d] : 0;
    s.bfix[d] = bfix ? bfix[d] : 0;
  }
  s.ea = ea;
  s.eb = eb;
  s.alpha = alpha;
  j->nblocks += s.nblk;
}

int64_t vt_splits(int64_t tiles, int64_t nblocks, int num_sms) {
  // jobs with long K only (the partials cost a reduction pass): enough units
  // for about four waves over the SMs, and at most 64 blocks per unit
  if (nblocks < 8) return 1;
  const int64_t want = std::max<int64_t>((nblocks + 63) / 64, (4LL * num_sms + tiles - 1) / tiles);
  return std::max<int64_t>(1, std::min<int64_t>(nblocks, want));
}

te_status vt_finish(VtBuild* b, int num_sms, double* part_scratch, int64_t scratch_cap, int64_t* used) {
  int64_t units = 0, off = 0, red = 0;
  for (int q = 0; q < b->P.njobs; ++q) {
    VtJob& J = b->P.job[q];
    if (J.nseg == 0) return fail(TE_EINVAL, "view GEMM: job without segments");
    for (int g = 0; g < J.nseg; ++g) {
      if (J.seg[g].amap < 0 || J.seg[g].bmap < 0 || J.seg[g].amap >= b->nmaps || J.seg[g].bmap >= b->nmaps)
        return fail(TE_EINVAL, "view GEMM: segment without a tensor map");
      if (J.seg[g].alpha != 1.0 && J.seg[g].alpha != -1.0)
        return fail(TE_EINVAL, "view GEMM: segment factor other than +-1");
    }
    const int64_t tiles = (int64_t)J.nm1 * J.nm2 * J.nn;
    if (!J.overwrite && part_scratch && tiles < num_sms && J.nblocks * VT_BLOCK_CHUNKS >= 8 * VT_SPLIT_CHUNKS) {
      J.nblocks = 0;
      for (int g = 0; g < J.nseg; ++g) {
        J.seg[g].bchunks = VT_SPLIT_CHUNKS;
        J.seg[g].nblk = (int)vt_seg_blocks(J.seg[g].K1, J.seg[g].K2, VT_SPLIT_CHUNKS);
        J.nblocks += J.seg[g].nblk;
      }
    }
    int64_t ns = 1;
    if (!J.overwrite && part_scratch) ns = vt_splits(tiles, J.nblocks, num_sms);
    const int64_t mn = (int64_t)J.M1 * J.M2 * J.N;
    while (ns > 1 && off + ns * mn > scratch_cap) ns = std::max<int64_t>(1, ns / 2);
    J.nsplit = (int)ns;
    J.part = nullptr;
    J.red0 = 0;
    if (ns > 1) {
      J.part = part_scratch + off;
      off += ns * mn;
      J.red0 = red;
      red += mn;
    }
    J.unit0 = units;
    units += tiles * ns;
  }
  b->P.total_units = units;
  b->P.total_red = red;
  if (used) *used = off;
  return TE_OK;
}

int64_t vt_split_doubles(int64_t tiles, int64_t nblocks, int64_t mn, int num_sms) {
  const int64_t ns = vt_splits(tiles, nblocks, num_sms);
  return ns > 1 ? ns * mn : 0;
}

template <int NS>
static cudaError_t vt_launch_ns(const VtBuild* b, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_view_tc<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_view_tc<NS><<<(unsigned)grid, VT_THREADS, smem, s>>>(b->maps, b->P);
  return cudaGetLastError();
}

te_status vt_launch(Handle* h, VtBuild* b, cudaStream_t s) {
  VtParams& P = b->P;
  if (P.total_units == 0) return TE_OK;
  int nt_max = 16;
  for (int q = 0; q < P.njobs; ++q) {
    const VtJob& J = P.job[q];
    if (J.NT % 16 != 0 || J.NT < 16 || J.NT > VT_NT_MAX || J.TA * J.TB != 128)
      return fail(TE_EINVAL, "view GEMM: tile %d x %d x %d", J.TA, J.TB, J.NT);
    nt_max = std::max(nt_max, J.NT);
  }
  P.nt_max = nt_max;
  P.stage_bytes = (uint32_t)P.ns * (VT_A_SLICE + (uint32_t)nt_max * VT_ROW_BYTES);
  const size_t avail = h->smem_optin > 2048 ? h->smem_optin - 2048 : 0;
  P.stages = (int)std::min<size_t>(4, avail / P.stage_bytes);
  if (P.stages < 2) return fail(TE_EUNSUPPORTED, "view GEMM: not enough shared memory for two stages");
  uint32_t cols = 32;
  while (cols < 3u * (uint32_t)nt_max) cols <<= 1;
  P.tmem_cols = cols;
  P.err = h->d_err;
  P.wait_ns = h->wait_limit_ns;
  const size_t smem = (size_t)P.stages * P.stage_bytes + 1024 + 256;
  const int grid = (int)std::min<int64_t>(P.total_units, std::max(1, h->num_sms));
  cudaError_t e = P.ns == 5 ? vt_launch_ns<5>(b, grid, smem, s) : vt_launch_ns<4>(b, grid, smem, s);
  if (e != cudaSuccess) return fail(TE_ECUDA, "view GEMM launch: %s", cudaGetErrorString(e));
  ++h->n_launches;
  if (P.total_red > 0) {
    k_vt_reduce<<<(unsigned)std::min<int64_t>((P.total_red + 255) / 256, 4 * std::max(1, h->num_sms)), 256, 0, s>>>(P);
    ++h->n_launches;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(TE_ECUDA, "view GEMM reduce: %s", cudaGetErrorString(e));
  return TE_OK;
}

int vt_ntile(int64_t n) {
  const int64_t t = (n + VT_NT_MAX - 1) / VT_NT_MAX;
  return (int)(((n + t - 1) / t + 15) / 16 * 16);
}

te_status vt_slice_maps(VtBank* k, const SliceSet& S, int o, int v, int nt, int* idx) {
  const uint64_t V = (uint64_t)v, O = (uint64_t)o, NS = (uint64_t)S.ns, vp = (uint64_t)S.vp, op = (uint64_t)S.op;
  const VtRoles XY{0, 1, 2, -1, 3}, ROW{0, 1, -1, -1, 2};
  struct Spec {
    const void* base;
    uint64_t dims[5], str[5];
    VtRoles r;
    int rows2, rows1;
  } sp[6] = {
      {S.ovvv, {V, V, V, NS, O}, {1, vp, V * vp, (uint64_t)S.ovvv_plane, (uint64_t)S.ovvv_p}, XY, 16, 8},
      {S.ovvv, {V, V, V, NS, O}, {1, V * vp, vp, (uint64_t)S.ovvv_plane, (uint64_t)S.ovvv_p}, XY, 16, 8},
      {S.t2L, {O, V, V, NS, O}, {1, op, V * op, (uint64_t)S.t2L_plane, (uint64_t)S.t2L_q}, XY, 16, 8},
      {S.t2L, {O, V, V, NS, O}, {1, V * op, op, (uint64_t)S.t2L_plane, (uint64_t)S.t2L_q}, XY, 16, 8},
      {S.t2, {V, V, NS, O, O}, {1, vp, (uint64_t)S.t2_plane, (uint64_t)S.t2_rq, O * (uint64_t)S.t2_rq}, ROW, nt, 1},
      {S.nooT, {O, V, NS, O, O}, {1, op, (uint64_t)S.nooT_plane, (uint64_t)S.nooT_pr, O * (uint64_t)S.nooT_pr}, ROW,
       nt, 1},
  };
  for (int q = 0; q < 6; ++q) {
    VtView w;
    w.base = sp[q].base;
    for (int d = 0; d < 5; ++d) {
      w.dims[d] = sp[q].dims[d];
      w.stride[d] = sp[q].str[d];
    }
    w.roles = sp[q].r;
    const te_status st = vt_bank_add(k, w, sp[q].rows2, sp[q].rows1, &idx[q]);
    if (st != TE_OK) return st;
  }
  return TE_OK;
}

cudaError_t vt_transpose(const void* src, int64_t src_ps, int64_t src_bs, int64_t src_rs, void* dst, int64_t dst_ps,
                         int64_t dst_bs, int64_t dst_cs, int np, int nb, int R, int Cc, cudaStream_t s) {
  if (np <= 0 || nb <= 0 || R <= 0 || Cc <= 0 || (R + 63) / 64 > 65535) return cudaErrorInvalidValue;
  const int pairs = (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 3) == 0 &&
                     ((src_ps | src_bs | src_rs | dst_ps | dst_bs | dst_cs) & 1) == 0)
                        ? 1
                        : 0;
  const unsigned short* s16 = static_cast<const unsigned short*>(src);
  unsigned short* d16 = static_cast<unsigned short*>(dst);
  // the grid's z extent covers (plane, batch) pairs: planes in groups when
  // all batches fit, else one plane at a time in batch chunks
  if (nb <= 65535) {
    const int per = std::max(1, std::min(np, 65535 / nb));
    for (int p0 = 0; p0 < np; p0 += per) {
      const int n = std::min(per, np - p0);
      dim3 grid((unsigned)((Cc + 63) / 64), (unsigned)((R + 63) / 64), (unsigned)(n * nb));
      k_vt_transpose<<<grid, dim3(32, 8), 0, s>>>(s16 + p0 * src_ps, src_ps, src_bs, src_rs, d16 + p0 * dst_ps, dst_ps,
                                                   dst_bs, dst_cs, nb, R, Cc, pairs);
    }
  } else {
    for (int p0 = 0; p0 < np; ++p0)
      for (int b0 = 0; b0 < nb; b0 += 65535) {
        const int n = std::min(65535, nb - b0);
        dim3 grid((unsigned)((Cc + 63) / 64), (unsigned)((R + 63) / 64), (unsigned)n);
        k_vt_transpose<<<grid, dim3(32, 8), 0, s>>>(s16 + p0 * src_ps + b0 * src_bs, src_ps, src_bs, src_rs,
                                                     d16 + p0 * dst_ps + b0 * dst_bs, dst_ps, dst_bs, dst_cs, n, R, Cc,
                                                     pairs);
      }
  }
  return cudaGetLastError();
}

}  // namespace te
