// Energy epilogue of the tensor-core modes: a persistent kernel fed by TMA.
//
// Work item = (triple slot, block triple X >= Y >= Z of 8-wide virtual
// blocks).  The contraction kernel stores G orbit-major (energy_tc.h): the
// item's 18 G cubes (3 G blocks x 6 block orders) are contiguous and arrive
// by one bulk copy; the 18 8x8 blocks of the symmetrised ovov the item uses
// and 9 t1 rows come by TMA (few, large copies: the copy engine's per-copy
// cost, not HBM, limited a layout that needed 54 copies per item).  A
// producer warp issues the loads into a double buffer; one thread per
// orbit candidate (a,b,c) of the 8^3 block triple.  G is either FP32 (BF16X3/TF32/TF32X3) or an FP32 pair
// hi + lo (OZAKI), CW = 1 or 2 floats per element.
//
// Orbit sum without cancellation: the 6x6 coefficient matrix C of R between
// the six orbit positions (T = sum_nm W_n C_nm V_m) has zero row and column
// sums, so T is unchanged when W_0 and V_0 are subtracted from every
// position.  The deviations w_n = W_n - W_0 are formed G block by G block
// (differences of close FP32 numbers are nearly exact), so the symmetric
// part of W~, which R annihilates, never enters a rounded product.
//   T = 3 sum_n w_n v_n + Ae Se + Ao So - 2 (Ae So + Ao Se)
// D, its reciprocal (FP32 seed + one Newton step in FP64: error ~1e-14),
// A T / D and the sums are FP64.
#include <cstring>

#include "energy_tc.h"
#include "ptx_sm100.cuh"

namespace te {

namespace {

constexpr int TB = 8;
constexpr int WARPS = 16;                 // compute warps: one orbit candidate (a,b,c) of 8^3 per thread
constexpr int THREADS = (WARPS + 1) * 32;  // + one producer warp

template <int N>
struct Pos {
  static constexpr int s0 = (N <= 1) ? 0 : (N <= 3) ? 1 : 2;
  static constexpr int s1 = (N == 0) ? 1 : (N == 1) ? 2 : (N == 2) ? 0 : (N == 3) ? 2 : (N == 4) ? 0 : 1;
  static constexpr int s2 = 3 - s0 - s1;
  static constexpr int r1 = (N == 0) ? 3 : (N == 1) ? 5 : (N == 2) ? 1 : (N == 3) ? 4 : (N == 4) ? 0 : 2;
  static constexpr int r2 = (N == 0) ? 4 : (N == 1) ? 2 : (N == 2) ? 5 : (N == 3) ? 0 : (N == 4) ? 3 : 1;
};

template <int CW>
struct Layout {
  static constexpr uint32_t cube_bytes = TB * TB * TB * 4 * CW;
  static constexpr uint32_t cubes = 18 * cube_bytes;
  static constexpr uint32_t ovs = 27 * TB * TB * 4;
  static constexpr uint32_t t1 = 9 * 128;
  static constexpr uint32_t eps = 640;  // dAB[64] = e_ijk - e_a - e_b, epsC[8] (FP64, written by the producer)
  static constexpr uint32_t buf = cubes + ovs + t1 + eps;
  // W~ (CW planes) and Y (one plane) of the item's 6 block orders, assembled once per item
  static constexpr uint32_t asm_bytes = 6 * 512 * 4 * (CW + 1);
  static constexpr uint32_t tx = 18 * cube_bytes + 18 * TB * TB * 4 + 9 * TB * 4;
};

__device__ __forceinline__ void decode_bt(int64_t bt, int* blk) {
  // bt = X(X+1)(X+2)/6 + Y(Y+1)/2 + Z, X >= Y >= Z >= 0 (FP32 estimate, exact integer fix-up)
  int x = (int)cbrtf(6.0f * (float)bt);
  while (x > 0 && (int64_t)x * (x + 1) * (x + 2) / 6 > bt) --x;
  while ((int64_t)(x + 1) * (x + 2) * (x + 3) / 6 <= bt) ++x;
  const int64_t rem = bt - (int64_t)x * (x + 1) * (x + 2) / 6;
  int y = (int)sqrtf(2.0f * (float)rem);
  while (y > 0 && (int64_t)y * (y + 1) / 2 > rem) --y;
  while ((int64_t)(y + 1) * (y + 2) / 2 <= rem) ++y;
  blk[0] = x;
  blk[1] = y;
  blk[2] = (int)(rem - (int64_t)y * (y + 1) / 2);
}

// ---- double-float (pair of FP32) arithmetic: error-free transformations ----
// Knuth two-sum, FMA two-product; the rn intrinsics forbid contraction.
struct df {
  float h, l;
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ df df_norm(float h, float l) {
  const float s = __fadd_rn(h, l);
  return {s, __fsub_rn(l, __fsub_rn(s, h))};
}

__device__ __forceinline__ df df_add(df a, df b) {
  const df s = df_two_sum(a.h, b.h);
  return df_norm(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.h, b.h);
  const float e = fmaf(a.h, b.h, -p);
  return df_norm(p, __fadd_rn(e, __fadd_rn(__fmul_rn(a.h, b.l), __fmul_rn(a.l, b.h))));
}

__device__ __forceinline__ df df_scale(df a, float k) {  // k a small integer
  const float p = __fmul_rn(a.h, k);
  const float e = fmaf(a.h, k, -p);
  return df_norm(p, __fadd_rn(e, __fmul_rn(a.l, k)));
}

// G value of block g at cube `pid`, local (x, y, z): hi and lo parts.
template <int CW>
__device__ __forceinline__ void gval(const float* cube, int g, int pid, int x, int y, int z, float& hi,
                                     float& lo) {
  const float* p = cube + (g * 6 + pid) * (TB * TB * TB * CW) + cube_off(x, y, z);
  hi = p[0];
  lo = (CW == 2) ? p[TB * TB * TB] : 0.f;
}

template <int S>
__device__ __forceinline__ int pick(int la, int lb, int lc) {
  return S == 0 ? la : (S == 1 ? lb : lc);
}

// deviation of W~ at position N from position 0, and Y at position N
template <int CW, int N>
__device__ __forceinline__ float w_dev(const float* cube, int la, int lb, int lc) {
  constexpr int s0 = Pos<N>::s0, s1 = Pos<N>::s1, s2 = Pos<N>::s2;
  const int x = pick<s0>(la, lb, lc), y = pick<s1>(la, lb, lc), z = pick<s2>(la, lb, lc);
  float h0, l0, hn, ln, d = 0.f, dl = 0.f;
  // G0[x][y][z] at cube N, minus G0[a][b][c] at cube 0
  gval<CW>(cube, 0, N, x, y, z, hn, ln);
  gval<CW>(cube, 0, 0, la, lb, lc, h0, l0);
  d += hn - h0;
  dl += ln - l0;
  // G1[y][z][x] at cube r1(N), minus G1[b][c][a] at cube 3
  gval<CW>(cube, 1, Pos<N>::r1, y, z, x, hn, ln);
  gval<CW>(cube, 1, 3, lb, lc, la, h0, l0);
  d += hn - h0;
  dl += ln - l0;
  // G2[z][x][y] at cube r2(N), minus G2[c][a][b] at cube 4
  gval<CW>(cube, 2, Pos<N>::r2, z, x, y, hn, ln);
  gval<CW>(cube, 2, 4, lc, la, lb, h0, l0);
  d += hn - h0;
  dl += ln - l0;
  return d + dl;
}

// double-float deviation of W~ at position N from position 0 (CW = 2)
template <int N>
__device__ __forceinline__ df w_dev_df(const float* cube, int la, int lb, int lc) {
  constexpr int s0 = Pos<N>::s0, s1 = Pos<N>::s1, s2 = Pos<N>::s2;
  const int x = pick<s0>(la, lb, lc), y = pick<s1>(la, lb, lc), z = pick<s2>(la, lb, lc);
  float h0, l0, hn, ln;
  gval<2>(cube, 0, N, x, y, z, hn, ln);
  gval<2>(cube, 0, 0, la, lb, lc, h0, l0);
  df acc = df_two_sum(hn, -h0);
  float lsum = __fsub_rn(ln, l0);
  gval<2>(cube, 1, Pos<N>::r1, y, z, x, hn, ln);
  gval<2>(cube, 1, 3, lb, lc, la, h0, l0);
  acc = df_add(acc, df_two_sum(hn, -h0));
  lsum = __fadd_rn(lsum, __fsub_rn(ln, l0));
  gval<2>(cube, 2, Pos<N>::r2, z, x, y, hn, ln);
  gval<2>(cube, 2, 4, lc, la, lb, h0, l0);
  acc = df_add(acc, df_two_sum(hn, -h0));
  lsum = __fadd_rn(lsum, __fsub_rn(ln, l0));
  return df_add(acc, df{lsum, 0.f});
}

template <int N>
__device__ __forceinline__ float y_at(const float* ovsS, const float* t1S, int la, int lb, int lc) {
  constexpr int s0 = Pos<N>::s0, s1 = Pos<N>::s1, s2 = Pos<N>::s2;
  const int x = pick<s0>(la, lb, lc), y = pick<s1>(la, lb, lc), z = pick<s2>(la, lb, lc);
  return ovsS[((0 * 3 + s0) * 3 + s1) * 64 + x * 8 + y] * t1S[(2 * 3 + s2) * 32 + z] +
         ovsS[((1 * 3 + s1) * 3 + s2) * 64 + y * 8 + z] * t1S[(0 * 3 + s0) * 32 + x] +
         ovsS[((2 * 3 + s0) * 3 + s2) * 64 + x * 8 + z] * t1S[(1 * 3 + s1) * 32 + y];
}

struct EnergyMaps {
  CUtensorMap ovs[TC_MAX_CL];  // per cluster: ovs32 [o][v][o][vq], 4D (b, j, a, i)
  CUtensorMap t1[TC_MAX_CL];   // per cluster: t1 [o][vq], 2D (a, i)
};

struct EnergyParams {
  int ncl, npieces;
  int64_t items;
  EnergyCl cl[TC_MAX_CL];
  TcPiece pc[TC_MAX_PIECES];  // G: orbit-major [slot][bt][g][pid][CW planes][512, swizzled] from pc.gbuf
  const Triple* triples;
  double* partials;  // [global slot][grid][WARPS]: the warps' sums of a triple's items
  unsigned int* err;
  unsigned long long wait_ns;
};

struct PieceTable {
  int n;
  TcPiece pc[TC_MAX_PIECES];
};

// A block's items: for each piece, for each of its triples, the block
// triples bt = blockIdx.x, blockIdx.x + gridDim.x, ... (< nbt), in order.
// Which items of a triple a block takes, and in which order, depends on the
// triple's nbt and the grid size alone (the grid is always one block per SM),
// not on the launch's other pieces: a triple's float64 sums have the same bits
// in a single-cluster call and in a batch.
struct ItemCursor {
  int q, ls;   // piece, triple slot within the piece
  int64_t bt;  // block triple
};

__device__ __forceinline__ void cursor_settle(const EnergyParams& P, ItemCursor& c) {
  while (c.q < P.npieces) {
    const TcPiece& pc = P.pc[c.q];
    if (c.bt < pc.nbt) return;
    c.bt = blockIdx.x;  // no (more) items of this triple for this block
    if (++c.ls >= pc.ns) {
      c.ls = 0;
      ++c.q;
    }
  }
}

template <int CW>
__global__ void __launch_bounds__(THREADS, 1)
    k_energy_tc(const __grid_constant__ EnergyMaps M, const __grid_constant__ EnergyParams P) {
  using L = Layout<CW>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) &
                                                         ~uintptr_t(127));
  float* asmW = reinterpret_cast<float*>(smem + 2 * L::buf);           // [CW planes][6][512] then Y [6][512]
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + 2 * L::buf + L::asm_bytes);  // [2]
  uint64_t* empty = full + 2;                                         // [2], one arrival per compute warp
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + 2);
  int* meta = const_cast<int*>(reinterpret_cast<volatile int*>(abort_flag) + 1);  // [2][8]: X, Y, Z, slot, v, item

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int q = 0; q < 2; ++q) {
      ptx::mbar_init(&full[q], 2);  // the copies' arrive.expect_tx and the denominator table's arrive
      ptx::mbar_init(&empty[q], WARPS);
    }
    *abort_flag = 0;
    ptx::fence_barrier_init();
  }
  __syncthreads();

  if (warp == WARPS) {
    // ---------------- producer warp ----------------
    uint32_t ephase = 0u, pending = 0u, fphase = 0u;  // one bit per buffer
    int b = 0;
    bool ok = true;
    ItemCursor cur{0, 0, (int64_t)blockIdx.x};
    cursor_settle(P, cur);
    for (; ok && cur.q < P.npieces; cur.bt += gridDim.x, cursor_settle(P, cur), b ^= 1) {
      // buffer b free: all compute warps done with the item it held
      int good = 1;
      if (lane == 0) good = ptx::mbar_wait(&empty[b], ((ephase >> b) & 1u) ^ 1u, P.wait_ns) ? 1 : 0;
      good = __shfl_sync(0xffffffffu, good, 0);
      if (!good || *abort_flag) {
        if (lane == 0 && !*abort_flag) {
          *abort_flag = 1;
          if (atomicOr(P.err, ERR_WAIT_TIMEOUT) == 0) {
            P.err[1] = 11;
            P.err[2] = blockIdx.x;
          }
        }
        ok = false;
        break;
      }
      ephase ^= 1u << b;
      const TcPiece& pc = P.pc[cur.q];
      const EnergyCl& C = P.cl[pc.cl];
      const int slot = cur.ls;
      const int64_t bt = cur.bt;
      const int64_t local = (int64_t)slot * C.nbt + bt;
      int blk[3];
      decode_bt(bt, blk);
      const Triple tr = P.triples[pc.t0 + slot];
      unsigned char* base = smem + (size_t)b * L::buf;
      if (lane == 0) {
        meta[b * 8 + 0] = blk[0];
        meta[b * 8 + 1] = blk[1];
        meta[b * 8 + 2] = blk[2];
        meta[b * 8 + 3] = pc.slot0 + slot;
        meta[b * 8 + 4] = C.v;
        ptx::mbar_arrive_expect_tx(&full[b], L::tx);  // first of the two arrivals
        pending |= 1u << b;
      }
      __syncwarp();
      const CUtensorMap* map_ovs = &M.ovs[pc.cl];
      const CUtensorMap* map_t1 = &M.t1[pc.cl];
      for (int q = lane; q < 28; q += 32) {
        if (q == 0) {  // the item's 18 cubes, contiguous ([g][pid] as in shared memory)
          ptx::bulk_load(base, pc.gbuf + local * (18 * TB * TB * TB * CW), 18 * L::cube_bytes, &full[b]);
        } else if (q < 19) {
          // ovs block (pair, sx, sy) with sx != sy: the only ones a permutation's Y reads
          const int rr = q - 1, pair = rr / 6, od = rr % 6;
          const int sx = od >> 1, sy = (od == 0) ? 1 : (od == 1) ? 2 : (od == 2) ? 0 : (od == 3) ? 2 : (od == 4) ? 0 : 1;
          const int r = pair * 9 + sx * 3 + sy;
          const int P1 = (pair == 1) ? tr.j : tr.i;
          const int P2 = (pair == 0) ? tr.j : tr.k;
          ptx::tma_load_4d(base + L::cubes + r * 256, map_ovs, &full[b], blk[sy] * TB, P2, blk[sx] * TB, P1);
        } else {
          const int r = q - 19, which = r / 3, s2 = r % 3;
          const int occ = which == 0 ? tr.i : (which == 1 ? tr.j : tr.k);
          ptx::tma_load_2d(base + L::cubes + L::ovs + r * 128, map_t1, &full[b], blk[s2] * TB, occ);
        }
      }
      {  // FP64 denominator pieces while the copies fly: dAB[la][lb] = e_i+e_j+e_k - e_a - e_b, epsC[lc] = e_c
        // the 24 virtual energies of the three blocks, one load per lane, shared by shuffles
        double* dAB = reinterpret_cast<double*>(base + L::cubes + L::ovs + L::t1);
        const int lq = lane < 24 ? blk[lane >> 3] * TB + (lane & 7) : 0;
        const double ev = (lane < 24 && lq < C.v) ? C.eps_v[lq] : 0.0;
        const double eo = C.eps_o[tr.i] + C.eps_o[tr.j] + C.eps_o[tr.k];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const int q = lane + 32 * r;  // every lane shuffles; lanes with q >= 72 store nothing
          const double ea = __shfl_sync(0xffffffffu, ev, q < 64 ? (q >> 3) : 16 + (q & 7));
          const double eb = __shfl_sync(0xffffffffu, ev, 8 + (q & 7));
          if (q < 64) {
            const int qa = blk[0] * TB + (q >> 3), qb = blk[1] * TB + (q & 7);
            dAB[q] = (qa < C.v && qb < C.v) ? (eo - ea) - eb : 0.0;
          } else if (q < 72) {
            const int qc = blk[2] * TB + (q - 64);
            dAB[q] = qc < C.v ? ea : 0.0;
          }
        }
      }
      __syncwarp();  // every lane's dAB stores are ordered before lane 0's release
      if (lane == 0) ptx::mbar_arrive(&full[b]);  // second arrival
      fphase ^= 1u << b;
    }
    // partials of the last items once their warps are done; copies in flight land
    if (lane == 0)
      for (int q = 0; q < 2; ++q)
        if (((pending >> q) & 1u) && !ok) ptx::mbar_wait(&full[q], ((fphase >> q) & 1u) ^ 1u, P.wait_ns);
  } else {
    // ---------------- compute warps ----------------
    // Each item in two phases.  A: every thread forms, at its own local point
    // (la, lb, lc) of each of the 6 block orders P, W~ = G0 + G1 + G2 (as an FP32
    // pair for CW = 2) and Y, into the assembled area; the G buffer is then
    // released to the producer.  B: every thread takes the orbit (a,b,c) =
    // its local point in block order 0 and reads W~ and Y at its 6 positions.
    uint32_t phase = 0u;  // one bit per buffer
    int b = 0;
    const int la = (tid >> 6), lb = (tid >> 3) & 7, lc = tid & 7;
    const int o_own = cube_off(la, lb, lc), o_g1 = cube_off(lb, lc, la), o_g2 = cube_off(lc, la, lb);
    int pos_off[6];
#pragma unroll
    for (int n = 0; n < 6; ++n) {
      const int u = n <= 1 ? la : (n <= 3 ? lb : lc);
      const int w = (n == 0 || n == 5) ? lb : ((n == 1 || n == 3) ? lc : la);
      const int z = 3 * 0 + ((n == 0 || n == 2) ? lc : ((n == 1 || n == 4) ? lb : la));
      pos_off[n] = n * 512 + cube_off(u, w, z);
    }
    float* asmY = asmW + CW * 6 * 512;
    // this thread's float64 sum over its items of the current triple slot; the
    // warp's sum (fixed shuffle order) goes to the partials when the slot
    // changes (a block takes a triple's items one after another)
    double acc = 0.0;
    int cur_slot = -1;
    auto flush = [&]() {
      double a = acc;
      for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
      if (lane == 0) P.partials[((int64_t)cur_slot * gridDim.x + blockIdx.x) * WARPS + warp] = a;
      acc = 0.0;
    };
    ItemCursor cur{0, 0, (int64_t)blockIdx.x};
    cursor_settle(P, cur);
    for (; cur.q < P.npieces; cur.bt += gridDim.x, cursor_settle(P, cur), b ^= 1) {
      int got = 0;
      if (!*abort_flag) got = ptx::mbar_wait(&full[b], (phase >> b) & 1u, P.wait_ns) ? 1 : 0;
      if (!__all_sync(0xffffffffu, got)) {
        if (lane == 0 && !*abort_flag) {
          *abort_flag = 1;
          if (atomicOr(P.err, ERR_WAIT_TIMEOUT) == 0) {
            P.err[1] = 10;
            P.err[2] = blockIdx.x;
          }
        }
        break;
      }
      phase ^= 1u << b;
      const int bx = meta[b * 8 + 0], by = meta[b * 8 + 1], bz = meta[b * 8 + 2], slot = meta[b * 8 + 3];
      const int vcl = meta[b * 8 + 4];
      if (slot != cur_slot) {
        if (cur_slot >= 0) flush();
        cur_slot = slot;
      }
      const unsigned char* base = smem + (size_t)b * L::buf;
      const float* cube = reinterpret_cast<const float*>(base);
      const float* ovsS = reinterpret_cast<const float*>(base + L::cubes);
      const float* t1S = reinterpret_cast<const float*>(base + L::cubes + L::ovs);
      const double* dAB = reinterpret_cast<const double*>(base + L::cubes + L::ovs + L::t1);
      const double D = dAB[la * 8 + lb] - dAB[64 + lc];

      // ---- phase A ----
#pragma unroll
      for (int Pn = 0; Pn < 6; ++Pn) {
        const int r1 = Pn == 0 ? 3 : Pn == 1 ? 5 : Pn == 2 ? 1 : Pn == 3 ? 4 : Pn == 4 ? 0 : 2;
        const int r2 = Pn == 0 ? 4 : Pn == 1 ? 2 : Pn == 2 ? 5 : Pn == 3 ? 0 : Pn == 4 ? 3 : 1;
        const int s0 = Pn <= 1 ? 0 : (Pn <= 3 ? 1 : 2);
        const int s1 = Pn == 0 ? 1 : Pn == 1 ? 2 : Pn == 2 ? 0 : Pn == 3 ? 2 : Pn == 4 ? 0 : 1;
        const int s2 = 3 - s0 - s1;
        const float* g0 = cube + (0 * 6 + Pn) * 512 * CW;
        const float* g1 = cube + (1 * 6 + r1) * 512 * CW;
        const float* g2 = cube + (2 * 6 + r2) * 512 * CW;
        const int wo = Pn * 512 + o_own;
        if constexpr (CW == 2) {
          df wv = df_two_sum(g0[o_own], g1[o_g1]);
          wv = df_add(wv, df{g2[o_g2], 0.f});
          wv = df_norm(wv.h, __fadd_rn(wv.l, __fadd_rn(__fadd_rn(g0[512 + o_own], g1[512 + o_g1]), g2[512 + o_g2])));
          asmW[wo] = wv.h;
          asmW[6 * 512 + wo] = wv.l;
        } else {
          asmW[wo] = (g0[o_own] + g1[o_g1]) + g2[o_g2];
        }
        // Y at (x, y, z) = (la, lb, lc) of blocks (s0, s1, s2):
        //   ovs(i,x,j,y) t1(k,z) + ovs(j,y,k,z) t1(i,x) + ovs(i,x,k,z) t1(j,y)
        asmY[wo] = ovsS[((0 * 3 + s0) * 3 + s1) * 64 + la * 8 + lb] * t1S[(2 * 3 + s2) * 32 + lc] +
                   ovsS[((1 * 3 + s1) * 3 + s2) * 64 + lb * 8 + lc] * t1S[(0 * 3 + s0) * 32 + la] +
                   ovsS[((2 * 3 + s0) * 3 + s2) * 64 + la * 8 + lc] * t1S[(1 * 3 + s1) * 32 + lb];
      }
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&empty[b]);  // this warp no longer reads buffer b
      asm volatile("bar.sync 1, %0;" ::"n"(WARPS * 32) : "memory");

      // ---- phase B ----
      const int a = bx * TB + la, bb = by * TB + lb, c = bz * TB + lc;
      const bool valid = a < vcl && bb < vcl && c < vcl && !(bx == by && la < lb) && !(by == bz && lb < lc);
      if (valid) {
        // orbit weight A (Eq. E_corr_CCSD_T): 1, 1/2 or 1/6
        const bool all3 = (a == bb && bb == c), two = (a == bb || bb == c);
        const double r0 = (double)__frcp_rn((float)D);
        const double r1 = fma(r0, fma(-D, r0, 1.0), r0);  // 1/D to ~1e-14 (one Newton step)
        const float y0 = asmY[pos_off[0]];
        if constexpr (CW == 2) {
          const float h0 = asmW[pos_off[0]], l0 = asmW[6 * 512 + pos_off[0]];
          df wd[5], vd[5];
#pragma unroll
          for (int n = 1; n < 6; ++n) {
            df d = df_two_sum(asmW[pos_off[n]], -h0);
            d = df_norm(d.h, __fadd_rn(d.l, __fsub_rn(asmW[6 * 512 + pos_off[n]], l0)));
            wd[n - 1] = d;
            vd[n - 1] = df_add(d, df{__fsub_rn(asmY[pos_off[n]], y0), 0.f});
          }
          const df w1 = wd[0], w2 = wd[1], w3 = wd[2], w4 = wd[3], w5 = wd[4];
          const df v1 = vd[0], v2 = vd[1], v3 = vd[2], v4 = vd[3], v5 = vd[4];
          const df Ae = df_add(w3, w4), Ao = df_add(df_add(w1, w2), w5);
          const df Se = df_add(v3, v4), So = df_add(df_add(v1, v2), v5);
          df dot = df_mul(w1, v1);
          dot = df_add(dot, df_mul(w2, v2));
          dot = df_add(dot, df_mul(w3, v3));
          dot = df_add(dot, df_mul(w4, v4));
          dot = df_add(dot, df_mul(w5, v5));
          df T = df_add(df_scale(dot, 3.f), df_add(df_mul(Ae, Se), df_mul(Ao, So)));
          T = df_add(T, df_scale(df_add(df_mul(Ae, So), df_mul(Ao, Se)), -2.f));
          if (all3) T = df_mul(T, df{0.16666667f, -4.967054e-09f});  // 1/6 as a float pair
          else if (two) T = df{T.h * 0.5f, T.l * 0.5f};
          acc = fma((double)T.h, r1, acc);
          acc = fma((double)T.l, r1, acc);
        } else {
          const float W0 = asmW[pos_off[0]];
          float w[5], vv[5];
#pragma unroll
          for (int n = 1; n < 6; ++n) {
            w[n - 1] = asmW[pos_off[n]] - W0;
            vv[n - 1] = w[n - 1] + (asmY[pos_off[n]] - y0);
          }
          const float Ae = w[2] + w[3], Ao = w[0] + w[1] + w[4];
          const float Se = vv[2] + vv[3], So = vv[0] + vv[1] + vv[4];
          const float dot = w[0] * vv[0] + w[1] * vv[1] + w[2] * vv[2] + w[3] * vv[3] + w[4] * vv[4];
          const float T = 3.f * dot + Ae * Se + Ao * So - 2.f * (Ae * So + Ao * Se);
          const double Tw = all3 ? (double)T * (1.0 / 6.0) : (double)(two ? 0.5f * T : T);
          acc = fma(Tw, r1, acc);
        }
      }
      asm volatile("bar.sync 1, %0;" ::"n"(WARPS * 32) : "memory");  // assembled area free
    }
    if (cur_slot >= 0) flush();
  }
  __syncthreads();
}

}  // namespace

int64_t energy_tc_grid(int num_sms, int64_t items) {
  (void)items;  // one block per SM whatever the launch holds: the item-to-block map is fixed per triple
  return std::max(1, num_sms);
}

size_t energy_tc_smem(int cw) {
  const size_t buf = cw == 2 ? Layout<2>::buf + Layout<2>::asm_bytes / 2 : Layout<1>::buf + Layout<1>::asm_bytes / 2;
  return 2 * buf + 128 + 512;
}

cudaError_t launch_energy_tc(const EnergyLaunch& e, cudaStream_t s) {
  EnergyMaps M;
  std::memset(&M, 0, sizeof(M));
  for (int c = 0; c < e.ncl; ++c) {
    M.ovs[c] = *e.map_ovs[c];
    M.t1[c] = *e.map_t1[c];
  }
  EnergyParams P;
  std::memset(&P, 0, sizeof(P));
  P.ncl = e.ncl;
  P.npieces = e.npieces;
  P.items = e.items;
  for (int c = 0; c < e.ncl; ++c) P.cl[c] = e.cl[c];
  for (int q = 0; q < e.npieces; ++q) P.pc[q] = e.pc[q];
  P.triples = e.triples;
  P.partials = e.partials;
  P.err = e.err;
  P.wait_ns = e.wait_ns;
  const size_t smem = energy_tc_smem(e.cw);
  const int64_t grid = energy_tc_grid(e.num_sms, P.items);
  // a block writes a slot's partials only if it took one of its items
  cudaError_t err = cudaMemsetAsync(P.partials, 0, (size_t)e.nslots * grid * WARPS * sizeof(double), s);
  if (err != cudaSuccess) return err;
  if (e.cw == 2) {
    err = cudaFuncSetAttribute(k_energy_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_energy_tc<2><<<(unsigned)grid, THREADS, smem, s>>>(M, P);
  } else {
    err = cudaFuncSetAttribute(k_energy_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_energy_tc<1><<<(unsigned)grid, THREADS, smem, s>>>(M, P);
  }
  return cudaGetLastError();
}

// One block per G slot of the launch: the slot's grid x WARPS partials summed
// in a fixed order (thread t takes t, t + 256, ..., then a fixed tree, with
// Neumaier compensation), times m/3, into its piece's shares.
__device__ __forceinline__ void neumaier(double& s, double& c, double x) {
  const double t = s + x;
  if (fabs(s) >= fabs(x)) c += (s - t) + x;
  else c += (x - t) + s;
  s = t;
}

__global__ void __launch_bounds__(256) k_reduce_pieces(const double* __restrict__ partials, int nper,
                                                       const Triple* __restrict__ triples,
                                                       const __grid_constant__ PieceTable T) {
  const int gslot = blockIdx.x;
  int q = 0;
  while (q + 1 < T.n && T.pc[q + 1].slot0 <= gslot) ++q;
  const TcPiece& pc = T.pc[q];
  const int local = gslot - pc.slot0;
  const double* x = partials + (int64_t)gslot * nper;
  __shared__ double ss[256], cc[256];
  double sum = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < nper; i += blockDim.x) neumaier(sum, c, x[i]);
  ss[threadIdx.x] = sum;
  cc[threadIdx.x] = c;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      double s1 = ss[threadIdx.x], c1 = cc[threadIdx.x] + cc[threadIdx.x + w];
      neumaier(s1, c1, ss[threadIdx.x + w]);
      ss[threadIdx.x] = s1;
      cc[threadIdx.x] = c1;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) pc.shares[local] = (ss[0] + cc[0]) * ((double)triples[pc.t0 + local].m / 3.0);
}

cudaError_t launch_reduce_pieces(const double* partials, int nper, const Triple* triples,
                                 const TcPiece* pieces, int npieces, int nslots, cudaStream_t s) {
  PieceTable T;
  std::memset(&T, 0, sizeof(T));
  T.n = npieces;
  for (int q = 0; q < npieces; ++q) T.pc[q] = pieces[q];
  k_reduce_pieces<<<(unsigned)nslots, 256, 0, s>>>(partials, nper, triples, T);
  return cudaGetLastError();
}

}  // namespace te
