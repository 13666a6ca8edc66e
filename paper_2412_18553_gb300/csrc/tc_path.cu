// Tensor-core path (TF32, BF16x3, TF32x3) for the W~ contractions.
//
// The same three G blocks as the float64 path (see gemm_fp64.cu):
//   W~_{ijk}[a,b,c] = G(i,j,k)[a,b,c] + G(j,k,i)[b,c,a] + G(k,i,j)[c,a,b]
// each one GEMM  D[(x,y), z] = sum_K A[(x,y), K] B[z, K]  with four K segments
//   S1 ovvv[p,x,y,:] . t2[r,q,z,:]     S2 ovvv[q,y,x,:] . t2[r,p,z,:]
//   S3 t2L[p,y,x,:] . nooT[q,r,z,:]    S4 t2L[q,x,y,:] . nooT[p,r,z,:]
// run on tcgen05: TMA brings 128-row A tiles (TA values of x times TB of y)
// and NT-row B tiles into swizzled shared memory; one elected thread issues
// tcgen05.mma into a double-buffered FP32 accumulator in tensor memory; four
// epilogue warps drain TMEM into the FP32 G buffer.  Operands are split once
// per call: x = hi + lo with hi, lo the nearest 8-bit (BF16) or 11-bit (TF32)
// significands, found by Veltkamp splitting; BF16x3/TF32x3 accumulate
// hi*hi + hi*lo + lo*hi, TF32 uses hi only.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "ptx_sm100.cuh"
#include "tc_path.h"

namespace te {

enum TcMode { TC_TF32 = 0, TC_BF16X3 = 1, TC_TF32X3 = 2 };

static int tc_mode_of(te_precision p) {
  return p == TE_TF32 ? TC_TF32 : (p == TE_BF16X3 ? TC_BF16X3 : TC_TF32X3);
}

// ---------------------------------------------------------------------------
// operand splitting
// ---------------------------------------------------------------------------

// Round x to the nearest value with `bits` significant bits (Veltkamp split).
// __dmul_rn / __dsub_rn keep the compiler from contracting into an FMA.
template <int BITS>
__device__ __forceinline__ double round_sig(double x) {
  const double c = __dmul_rn(x, (double)((1ull << (53 - BITS)) + 1ull));
  return __dsub_rn(c, __dsub_rn(c, x));
}

template <int MODE>
__device__ __forceinline__ void split_store(double x, void* hi, void* lo, int64_t idx) {
  if (MODE == TC_BF16X3) {
    const double h = round_sig<8>(x);
    const double l = round_sig<8>(x - h);
    reinterpret_cast<__nv_bfloat16*>(hi)[idx] = __float2bfloat16_rn((float)h);
    reinterpret_cast<__nv_bfloat16*>(lo)[idx] = __float2bfloat16_rn((float)l);
  } else {
    const double h = round_sig<11>(x);
    reinterpret_cast<float*>(hi)[idx] = (float)h;
    if (MODE == TC_TF32X3) reinterpret_cast<float*>(lo)[idx] = (float)round_sig<11>(x - h);
  }
}

// dst[row][kp] = src[row][k] (k < K) or 0, rows x Kp
template <int MODE>
__global__ void k_split_rows(const double* __restrict__ src, void* hi, void* lo, int64_t rows, int K,
                             int Kp) {
  const int64_t n = rows * Kp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % Kp);
    const int64_t row = idx / Kp;
    const double x = k < K ? src[row * K + k] : 0.0;
    split_store<MODE>(x, hi, lo, idx);
  }
}

// t2L[q][x][y][l] = t2[l][q][x][y], l padded to op
template <int MODE>
__global__ void k_split_t2L(const double* __restrict__ t2, void* hi, void* lo, int o, int v, int op) {
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
    split_store<MODE>(val, hi, lo, idx);
  }
}

// nooT[p][r][z][l] = -ooov[p][l][r][z], l padded to op
template <int MODE>
__global__ void k_split_noo(const double* __restrict__ ooov, void* hi, void* lo, int o, int v, int op) {
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
    split_store<MODE>(val, hi, lo, idx);
  }
}

__global__ void k_ovs32(const double* __restrict__ ovov, float* __restrict__ ovs32, int o, int v) {
  const int64_t n = (int64_t)o * v * o * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(idx % v);
    int64_t rest = idx / v;
    const int j = (int)(rest % o);
    rest /= o;
    const int a = (int)(rest % v);
    const int i = (int)(rest / v);
    ovs32[idx] = (float)(0.5 * (ovov[idx] + ovov[(((int64_t)j * v + b) * o + i) * v + a]));
  }
}

__global__ void k_t1_32(const double* __restrict__ t1, float* __restrict__ out, int64_t n) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x)
    out[idx] = (float)t1[idx];
}

static int gridn(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>(1, (n + 255) / 256), 16384); }

// ---------------------------------------------------------------------------
// the GEMM kernel
// ---------------------------------------------------------------------------

struct TcMaps {
  CUtensorMap a_nat[2];  // ovvv split, dims (Kp, y, x, p): rows (x,y) of ovvv[p]
  CUtensorMap a_tr[2];   // ovvv split, dims (Kp, y, x, q) with strides swapped: ovvv[q,y,x,:]
  CUtensorMap l_nat[2];  // t2L split natural
  CUtensorMap l_tr[2];   // t2L split transposed
  CUtensorMap b_t2[2];   // t2 split, dims (Kp, z, q, r)
  CUtensorMap b_noo[2];  // nooT split, dims (Kp, z, r, p)
};

struct TcParams {
  int o, v;
  int TA, TB, NT;
  int n_mx, n_my, n_nt;
  int kw_chunks, ko_chunks;
  int kw_elems, ko_elems;  // elements per chunk
  int cbw, cbo;            // chunk bytes (v- and o-segments)
  int stages;
  uint32_t stage_bytes, a_part_bytes, b_part_bytes;
  uint32_t tmem_cols;
  int64_t total_tiles;
  int64_t t0;
  const Triple* triples;
  float* gbuf;
  int ldz;
  unsigned int* err;
  unsigned long long wait_ns;
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
  int slot, g, p, q, r, x0, y0, z0;
};

__device__ __forceinline__ TileCoord decode_tile(const TcParams& P, int64_t tt) {
  TileCoord c;
  int64_t rest = tt;
  const int nt = (int)(rest % P.n_nt);
  rest /= P.n_nt;
  const int my = (int)(rest % P.n_my);
  rest /= P.n_my;
  const int mx = (int)(rest % P.n_mx);
  rest /= P.n_mx;
  c.g = (int)(rest % 3);
  c.slot = (int)(rest / 3);
  const Triple T = P.triples[P.t0 + c.slot];
  if (c.g == 0) { c.p = T.i; c.q = T.j; c.r = T.k; }
  else if (c.g == 1) { c.p = T.j; c.q = T.k; c.r = T.i; }
  else { c.p = T.k; c.q = T.i; c.r = T.j; }
  c.x0 = mx * P.TA;
  c.y0 = my * P.TB;
  c.z0 = nt * P.NT;
  return c;
}

template <int MODE>
__global__ void __launch_bounds__(192, 1) k_gemm_tc(const __grid_constant__ TcMaps maps, const TcParams P) {
  constexpr bool TF32 = (MODE != TC_BF16X3);
  constexpr bool X3 = (MODE != TC_TF32);
  constexpr int NPART = X3 ? 2 : 1;
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
      ptx::mbar_init(&tempty[a], 4);
    }
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    for (int k = 0; k < NPART; ++k) {
      ptx::tma_prefetch_desc(&maps.a_nat[k]);
      ptx::tma_prefetch_desc(&maps.a_tr[k]);
      ptx::tma_prefetch_desc(&maps.l_nat[k]);
      ptx::tma_prefetch_desc(&maps.l_tr[k]);
      ptx::tma_prefetch_desc(&maps.b_t2[k]);
      ptx::tma_prefetch_desc(&maps.b_noo[k]);
    }
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
      int pending[16];
      for (int s = 0; s < 16; ++s) pending[s] = -1;
      bool ok = true;
      for (int64_t tt = blockIdx.x; ok && tt < P.total_tiles; tt += gridDim.x) {
        const TileCoord c = decode_tile(P, tt);
        for (int seg = 0; ok && seg < 4; ++seg) {
          const bool wide = seg < 2;
          const int nch = wide ? P.kw_chunks : P.ko_chunks;
          const int cb = wide ? P.cbw : P.cbo;
          const int ce = wide ? P.kw_elems : P.ko_elems;
          const uint32_t bytes = (uint32_t)NPART * (128u * cb + (uint32_t)P.NT * cb);
          for (int ch = 0; ch < nch; ++ch) {
            if (*abort_flag || !ptx::mbar_wait(&empty[stage], phase ^ 1u, P.wait_ns)) {
              if (!*abort_flag) record_abort(P, abort_flag, 1);
              ok = false;
              break;
            }
            ptx::mbar_arrive_expect_tx(&full[stage], bytes);
            pending[stage] = (int)phase;
            unsigned char* sa = smem + (size_t)stage * P.stage_bytes;
            const int kc = ch * ce;
#pragma unroll
            for (int k = 0; k < NPART; ++k) {
              void* da = sa + k * P.a_part_bytes;
              void* db = sa + NPART * P.a_part_bytes + k * P.b_part_bytes;
              if (seg == 0) {
                ptx::tma_load_4d(da, &maps.a_nat[k], &full[stage], kc, c.y0, c.x0, c.p);
                ptx::tma_load_4d(db, &maps.b_t2[k], &full[stage], kc, c.z0, c.q, c.r);
              } else if (seg == 1) {
                ptx::tma_load_4d(da, &maps.a_tr[k], &full[stage], kc, c.y0, c.x0, c.q);
                ptx::tma_load_4d(db, &maps.b_t2[k], &full[stage], kc, c.z0, c.p, c.r);
              } else if (seg == 2) {
                ptx::tma_load_4d(da, &maps.l_tr[k], &full[stage], kc, c.y0, c.x0, c.p);
                ptx::tma_load_4d(db, &maps.b_noo[k], &full[stage], kc, c.z0, c.r, c.q);
              } else {
                ptx::tma_load_4d(da, &maps.l_nat[k], &full[stage], kc, c.y0, c.x0, c.q);
                ptx::tma_load_4d(db, &maps.b_noo[k], &full[stage], kc, c.z0, c.r, c.p);
              }
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
      const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(P.NT >> 3) << 17) |
                             ((uint32_t)(128 >> 4) << 24);
      uint32_t stage = 0, phase = 0, acc = 0, acc_phase = 0;
      bool ok = true;
      bool issued = false;
      for (int64_t tt = blockIdx.x; ok && tt < P.total_tiles; tt += gridDim.x) {
        if (*abort_flag || !ptx::mbar_wait(&tempty[acc], acc_phase ^ 1u, P.wait_ns)) {
          if (!*abort_flag) record_abort(P, abort_flag, 2);
          break;
        }
        ptx::tc_fence_after();
        const uint32_t d_tmem = tmem_base + acc * (uint32_t)P.NT;
        uint32_t accum = 0;
        for (int seg = 0; ok && seg < 4; ++seg) {
          const bool wide = seg < 2;
          const int nch = wide ? P.kw_chunks : P.ko_chunks;
          const int cb = wide ? P.cbw : P.cbo;
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
              const uint64_t ah = ptx::smem_desc(a0 + ks * 32, sbo, lay);
              const uint64_t bh = ptx::smem_desc(b0 + ks * 32, sbo, lay);
              ptx::mma<TF32>(d_tmem, ah, bh, idesc, accum);
              accum = 1;
              if (X3) {
                const uint64_t al = ptx::smem_desc(a0 + P.a_part_bytes + ks * 32, sbo, lay);
                const uint64_t bl = ptx::smem_desc(b0 + P.b_part_bytes + ks * 32, sbo, lay);
                ptx::mma<TF32>(d_tmem, ah, bl, idesc, 1);
                ptx::mma<TF32>(d_tmem, al, bh, idesc, 1);
              }
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
        acc ^= 1u;
        if (acc == 0) acc_phase ^= 1u;
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
    const int row = quad * 32 + lane;
    const int64_t v2 = (int64_t)P.v * P.v;
    uint32_t acc = 0, acc_phase = 0;
    for (int64_t tt = blockIdx.x; tt < P.total_tiles; tt += gridDim.x) {
      const TileCoord c = decode_tile(P, tt);
      int got = 0;
      if (!*abort_flag) got = ptx::mbar_wait(&tfull[acc], acc_phase, P.wait_ns) ? 1 : 0;
      // the decision is warp-uniform: tcgen05.ld below is a .sync.aligned instruction
      if (!__all_sync(0xffffffffu, got)) {
        if (!*abort_flag && lane == 0) record_abort(P, abort_flag, 4);
        break;
      }
      ptx::tc_fence_after();
      const int x = c.x0 + row / P.TB;
      const int y = c.y0 + row % P.TB;
      const bool valid = x < P.v && y < P.v;
      float* out = P.gbuf + ((int64_t)(c.slot * 3 + c.g) * v2 + (int64_t)x * P.v + y) * P.ldz;
      const uint32_t tbase = tmem_base + ((uint32_t)(quad * 32) << 16) + acc * (uint32_t)P.NT;
      for (int c0 = 0; c0 < P.NT; c0 += 16) {
        float vals[16];
        ptx::tmem_ld16(tbase + c0, vals);
        const int z = c.z0 + c0;
        if (valid) {
          if (z + 16 <= P.ldz) {
            float4* o4 = reinterpret_cast<float4*>(out + z);
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4)
              o4[q4] = make_float4(vals[4 * q4], vals[4 * q4 + 1], vals[4 * q4 + 2], vals[4 * q4 + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (z + j < P.v) out[z + j] = vals[j];
          }
        }
      }
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&tempty[acc]);
      acc ^= 1u;
      if (acc == 0) acc_phase ^= 1u;
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
  bool attr_done[3] = {false, false, false};
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
  int mode, es;
  int vp, op;
  int TA, TB, NT, n_mx, n_my, n_nt;
  int kw_chunks, ko_chunks, kw_elems, ko_elems, cbw, cbo;
  int stages;
  uint32_t stage_bytes, a_part_bytes, b_part_bytes, tmem_cols;
  int nslots;
  int ldz;
  size_t smem;
};

static int round_up(int x, int m) { return (x + m - 1) / m * m; }

static TcPlan make_plan(const Handle* h, int o, int v, int mode, int64_t ntri) {
  TcPlan pl{};
  pl.mode = mode;
  pl.es = (mode == TC_BF16X3) ? 2 : 4;
  pl.vp = round_up(v, 16);
  pl.op = round_up(o, 16);
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
  pl.TB = bestTB;
  pl.TA = 128 / bestTB;
  pl.n_mx = (v + pl.TA - 1) / pl.TA;
  pl.n_my = (v + pl.TB - 1) / pl.TB;
  pl.n_nt = (v + 255) / 256;
  pl.NT = round_up((v + pl.n_nt - 1) / pl.n_nt, 16);
  pl.cbw = 128;
  pl.kw_elems = 128 / pl.es;
  pl.kw_chunks = (pl.vp + pl.kw_elems - 1) / pl.kw_elems;
  const int obytes = pl.op * pl.es;
  pl.cbo = obytes <= 32 ? 32 : (obytes <= 64 ? 64 : 128);
  pl.ko_elems = pl.cbo / pl.es;
  pl.ko_chunks = (pl.op + pl.ko_elems - 1) / pl.ko_elems;
  const int npart = (mode == TC_TF32) ? 1 : 2;
  pl.a_part_bytes = 128u * 128u;
  pl.b_part_bytes = (uint32_t)pl.NT * 128u;
  pl.stage_bytes = (uint32_t)npart * (pl.a_part_bytes + pl.b_part_bytes);
  const size_t avail = h->smem_optin > 2048 ? h->smem_optin - 2048 : 0;
  pl.stages = (int)std::min<size_t>(8, avail / pl.stage_bytes);
  pl.smem = (size_t)pl.stages * pl.stage_bytes + 1024 + 256;
  uint32_t cols = 32;
  while (cols < 2u * (uint32_t)pl.NT) cols <<= 1;
  pl.tmem_cols = cols;
  pl.ldz = round_up(v, 4);
  const int64_t tiles = 3LL * pl.n_mx * pl.n_my * pl.n_nt;
  int64_t want = (4LL * std::max(1, h->num_sms) + tiles - 1) / tiles;
  const int64_t per_slot = 3LL * v * v * pl.ldz * 4;
  const int64_t mem_cap = std::max<int64_t>(1, (int64_t)(3LL << 30) / per_slot);
  want = std::min<int64_t>({want, mem_cap, 1024, std::max<int64_t>(1, ntri)});
  pl.nslots = (int)std::max<int64_t>(1, want);
  return pl;
}

struct TcBuffers {
  void *a_hi, *a_lo, *b_hi, *b_lo, *l_hi, *l_lo, *n_hi, *n_lo;
  float *ovs32, *t1_32, *gbuf;
  double *partials, *etri;
};

static size_t tc_carve(char* base, const TcPlan& pl, int64_t o, int64_t v, int64_t nbt, int64_t ntri,
                       TcBuffers* b) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> void* {
    off = (off + 1023) & ~size_t(1023);
    void* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  };
  const bool x3 = pl.mode != TC_TF32;
  const size_t es = (size_t)pl.es;
  const size_t na = (size_t)o * v * v * pl.vp, nb = (size_t)o * o * v * pl.vp;
  const size_t nl = (size_t)o * v * v * pl.op, nn = (size_t)o * o * v * pl.op;
  b->a_hi = take(na * es);
  b->a_lo = x3 ? take(na * es) : nullptr;
  b->b_hi = take(nb * es);
  b->b_lo = x3 ? take(nb * es) : nullptr;
  b->l_hi = take(nl * es);
  b->l_lo = x3 ? take(nl * es) : nullptr;
  b->n_hi = take(nn * es);
  b->n_lo = x3 ? take(nn * es) : nullptr;
  b->ovs32 = static_cast<float*>(take((size_t)o * v * o * v * 4));
  b->t1_32 = static_cast<float*>(take((size_t)o * v * 4));
  b->gbuf = static_cast<float*>(take((size_t)pl.nslots * 3 * v * v * pl.ldz * 4));
  b->partials = static_cast<double*>(take((size_t)pl.nslots * nbt * 8));
  b->etri = static_cast<double*>(take((size_t)std::max<int64_t>(1, ntri) * 8));
  return off + 1024;
}

static te_status encode_4d(TcState* st, CUtensorMap* m, const void* base, CUtensorMapDataType dt, int es,
                           const uint64_t dims[4], const uint64_t strides_bytes[3], const uint32_t box[4],
                           CUtensorMapSwizzle swz, const char* what) {
  cuuint64_t gd[4] = {dims[0], dims[1], dims[2], dims[3]};
  cuuint64_t gs[3] = {strides_bytes[0], strides_bytes[1], strides_bytes[2]};
  cuuint32_t bd[4] = {box[0], box[1], box[2], box[3]};
  cuuint32_t es1[4] = {1, 1, 1, 1};
  (void)es;
  CUresult r = st->encode(m, dt, 4, const_cast<void*>(base), gd, gs, bd, es1, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(TE_ECUDA, "tensor map encoding failed for %s (CUresult %d)", what, (int)r);
  return TE_OK;
}

static CUtensorMapSwizzle swz_of(int cb) {
  return cb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : (cb == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
}

static te_status build_maps(TcState* st, const TcPlan& pl, int o, int v, const TcBuffers& b, TcMaps* M) {
  std::memset(M, 0, sizeof(*M));
  const CUtensorMapDataType dt =
      pl.mode == TC_BF16X3 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const uint64_t es = (uint64_t)pl.es;
  const uint64_t vp = pl.vp, op = pl.op, V = v, O = o;
  const int npart = pl.mode == TC_TF32 ? 1 : 2;
  for (int k = 0; k < npart; ++k) {
    const void* A = k ? b.a_lo : b.a_hi;
    const void* B = k ? b.b_lo : b.b_hi;
    const void* L = k ? b.l_lo : b.l_hi;
    const void* N = k ? b.n_lo : b.n_hi;
    te_status s;
    {  // ovvv[p][x][y][d]: dims (d, y, x, p)
      const uint64_t d[4] = {vp, V, V, O};
      const uint64_t sn[3] = {vp * es, V * vp * es, V * V * vp * es};
      const uint32_t box[4] = {(uint32_t)pl.kw_elems, (uint32_t)pl.TB, (uint32_t)pl.TA, 1};
      if ((s = encode_4d(st, &M->a_nat[k], A, dt, pl.es, d, sn, box, swz_of(pl.cbw), "ovvv")) != TE_OK) return s;
      // transposed rows: element (d, y, x, q) at ovvv[q][y][x][d]
      const uint64_t stt[3] = {V * vp * es, vp * es, V * V * vp * es};
      if ((s = encode_4d(st, &M->a_tr[k], A, dt, pl.es, d, stt, box, swz_of(pl.cbw), "ovvv^T")) != TE_OK) return s;
    }
    {  // t2L[q][x][y][l]: dims (l, y, x, q)
      const uint64_t d[4] = {op, V, V, O};
      const uint64_t sn[3] = {op * es, V * op * es, V * V * op * es};
      const uint32_t box[4] = {(uint32_t)pl.ko_elems, (uint32_t)pl.TB, (uint32_t)pl.TA, 1};
      if ((s = encode_4d(st, &M->l_nat[k], L, dt, pl.es, d, sn, box, swz_of(pl.cbo), "t2L")) != TE_OK) return s;
      const uint64_t stt[3] = {V * op * es, op * es, V * V * op * es};
      if ((s = encode_4d(st, &M->l_tr[k], L, dt, pl.es, d, stt, box, swz_of(pl.cbo), "t2L^T")) != TE_OK) return s;
    }
    {  // t2[r][q][z][d]: dims (d, z, q, r)
      const uint64_t d[4] = {vp, V, O, O};
      const uint64_t sn[3] = {vp * es, V * vp * es, O * V * vp * es};
      const uint32_t box[4] = {(uint32_t)pl.kw_elems, (uint32_t)pl.NT, 1, 1};
      if ((s = encode_4d(st, &M->b_t2[k], B, dt, pl.es, d, sn, box, swz_of(pl.cbw), "t2")) != TE_OK) return s;
    }
    {  // nooT[p][r][z][l]: dims (l, z, r, p)
      const uint64_t d[4] = {op, V, O, O};
      const uint64_t sn[3] = {op * es, V * op * es, O * V * op * es};
      const uint32_t box[4] = {(uint32_t)pl.ko_elems, (uint32_t)pl.NT, 1, 1};
      if ((s = encode_4d(st, &M->b_noo[k], N, dt, pl.es, d, sn, box, swz_of(pl.cbo), "nooT")) != TE_OK) return s;
    }
  }
  return TE_OK;
}

template <int MODE>
static cudaError_t launch_prep_tc(const te_cluster* c, const TcPlan& pl, const TcBuffers& b, cudaStream_t s) {
  const int o = (int)c->nocc, v = (int)c->nvir;
  k_split_rows<MODE><<<gridn((int64_t)o * v * v * pl.vp), 256, 0, s>>>(c->ovvv, b.a_hi, b.a_lo,
                                                                       (int64_t)o * v * v, v, pl.vp);
  k_split_rows<MODE><<<gridn((int64_t)o * o * v * pl.vp), 256, 0, s>>>(c->t2, b.b_hi, b.b_lo,
                                                                       (int64_t)o * o * v, v, pl.vp);
  k_split_t2L<MODE><<<gridn((int64_t)o * v * v * pl.op), 256, 0, s>>>(c->t2, b.l_hi, b.l_lo, o, v, pl.op);
  k_split_noo<MODE><<<gridn((int64_t)o * o * v * pl.op), 256, 0, s>>>(c->ooov, b.n_hi, b.n_lo, o, v, pl.op);
  k_ovs32<<<gridn((int64_t)o * v * o * v), 256, 0, s>>>(c->ovov, b.ovs32, o, v);
  k_t1_32<<<gridn((int64_t)o * v), 256, 0, s>>>(c->t1, b.t1_32, (int64_t)o * v);
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_gemm_tc(TcState* st, const Handle* h, const TcMaps& M, const TcParams& P,
                                  size_t smem, cudaStream_t s) {
  if (!st->attr_done[MODE]) {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    st->attr_done[MODE] = true;
  } else {
    cudaFuncSetAttribute(k_gemm_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  const int64_t grid = std::min<int64_t>(P.total_tiles, h->num_sms);
  k_gemm_tc<MODE><<<(unsigned)grid, 192, smem, s>>>(M, P);
  return cudaGetLastError();
}

te_status tc_workspace_bytes(Handle* h, const te_cluster* c, te_precision p, size_t* bytes) {
  const TcPlan pl = make_plan(h, (int)c->nocc, (int)c->nvir, tc_mode_of(p), num_unique_triples(c->nocc));
  TcBuffers b;
  *bytes = tc_carve(nullptr, pl, c->nocc, c->nvir, energy_num_block_triples(c->nvir),
                    num_unique_triples(c->nocc), &b);
  return TE_OK;
}

te_status ensure_workspace_public(Handle* h, size_t bytes);
te_status ensure_triples_public(Handle* h, int nocc);

te_status run_tc(Handle* h, const te_cluster* c, te_precision p, int64_t t_begin, int64_t t_end,
                 double* e_tri_out, double* e_total_out, cudaStream_t s) {
  if (h->cc_major != 10 && h->cc_major != 11)
    return fail(TE_EUNSUPPORTED, "tensor-core modes need an sm_100-family GPU (found sm_%d%d)", h->cc_major,
                h->cc_minor);
  TcState* st = tc_state(h);
  te_status rs = get_encoder(st);
  if (rs != TE_OK) return rs;
  const int o = (int)c->nocc, v = (int)c->nvir;
  const int mode = tc_mode_of(p);
  const int64_t ntri = num_unique_triples(o);
  const int64_t nt = t_end - t_begin;
  const TcPlan pl = make_plan(h, o, v, mode, nt);
  if (pl.stages < 2) return fail(TE_EUNSUPPORTED, "not enough shared memory for two pipeline stages");
  const int64_t nbt = energy_num_block_triples(v);
  TcBuffers b;
  const size_t bytes = tc_carve(nullptr, pl, o, v, nbt, ntri, &b);
  rs = ensure_workspace_public(h, bytes);
  if (rs != TE_OK) return rs;
  rs = ensure_triples_public(h, o);
  if (rs != TE_OK) return rs;
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(h->ws) + 1023) & ~uintptr_t(1023));
  tc_carve(base, pl, o, v, nbt, ntri, &b);

  cudaError_t e;
  if (mode == TC_BF16X3) e = launch_prep_tc<TC_BF16X3>(c, pl, b, s);
  else if (mode == TC_TF32X3) e = launch_prep_tc<TC_TF32X3>(c, pl, b, s);
  else e = launch_prep_tc<TC_TF32>(c, pl, b, s);
  if (e != cudaSuccess) return fail(TE_ECUDA, "operand split launch: %s", cudaGetErrorString(e));

  TcMaps M;
  rs = build_maps(st, pl, o, v, b, &M);
  if (rs != TE_OK) return rs;

  TcParams P{};
  P.o = o;
  P.v = v;
  P.TA = pl.TA;
  P.TB = pl.TB;
  P.NT = pl.NT;
  P.n_mx = pl.n_mx;
  P.n_my = pl.n_my;
  P.n_nt = pl.n_nt;
  P.kw_chunks = pl.kw_chunks;
  P.ko_chunks = pl.ko_chunks;
  P.kw_elems = pl.kw_elems;
  P.ko_elems = pl.ko_elems;
  P.cbw = pl.cbw;
  P.cbo = pl.cbo;
  P.stages = pl.stages;
  P.stage_bytes = pl.stage_bytes;
  P.a_part_bytes = pl.a_part_bytes;
  P.b_part_bytes = pl.b_part_bytes;
  P.tmem_cols = pl.tmem_cols;
  P.triples = h->d_triples;
  P.gbuf = b.gbuf;
  P.ldz = pl.ldz;
  P.err = h->d_err;
  P.wait_ns = h->wait_limit_ns;

  Prepared Pr{};
  Pr.o = o;
  Pr.v = v;
  Pr.eps_o = c->eps_o;
  Pr.eps_v = c->eps_v;
  Pr.ovs32 = b.ovs32;
  Pr.t1_32 = b.t1_32;
  h->n_launches += 6;
  double* out = e_tri_out ? e_tri_out : b.etri;
  const double nprod = (mode == TC_TF32) ? 1.0 : 3.0;
  const double kpad = 2.0 * pl.kw_chunks * pl.kw_elems + 2.0 * pl.ko_chunks * pl.ko_elems;
  for (int64_t t0 = t_begin; t0 < t_end; t0 += pl.nslots) {
    const int ns = (int)std::min<int64_t>(pl.nslots, t_end - t0);
    P.t0 = t0;
    P.total_tiles = 3LL * ns * pl.n_mx * pl.n_my * pl.n_nt;
    size_t pm = prof_begin(h, 0, s);
    if (mode == TC_BF16X3) e = launch_gemm_tc<TC_BF16X3>(st, h, M, P, pl.smem, s);
    else if (mode == TC_TF32X3) e = launch_gemm_tc<TC_TF32X3>(st, h, M, P, pl.smem, s);
    else e = launch_gemm_tc<TC_TF32>(st, h, M, P, pl.smem, s);
    prof_end(h, pm, s);
    h->gemm_flops += 2.0 * nprod * (double)P.total_tiles * 128.0 * pl.NT * kpad;
    if (e == cudaSuccess) {
      pm = prof_begin(h, 1, s);
      e = launch_energy_f32(&Pr, h->d_triples, t0, ns, b.gbuf, pl.ldz, b.partials, nbt, s);
      prof_end(h, pm, s);
    }
    if (e == cudaSuccess)
      e = launch_reduce_triples(b.partials, nbt, h->d_triples, t0, ns, out + (t0 - t_begin), s);
    h->n_launches += 3;
    if (e != cudaSuccess) return fail(TE_ECUDA, "tensor-core path launch: %s", cudaGetErrorString(e));
  }
  if (e_total_out) {
    ++h->n_launches;
    e = launch_reduce_total(out, nt, e_total_out, s);
    if (e != cudaSuccess) return fail(TE_ECUDA, "reduction launch: %s", cudaGetErrorString(e));
  }
  return TE_OK;
}

}  // namespace te
