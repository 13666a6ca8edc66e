// Energy epilogue and deterministic reductions.
//
// For one unique occupied triple (i,j,k) the share of E(T) is
//   (m/3) sum_{abc} W~^{abc} R[V]^{abc} / D^{abc},   V = W~ + Y,
// with R acting on the occupied indices (Eq. R_opt_in_CCSD(T)).  Because W~,
// Y and D are invariant under simultaneous permutation of (i,j,k) and (a,b,c),
// R acting on occupied indices at fixed abc equals the same operator acting on
// the virtual indices at fixed ijk:
//   R[V]^{xyz} = 4V^{xyz} + V^{yzx} + V^{zxy} - 2V^{zyx} - 2V^{xzy} - 2V^{yxz}.
// The sum over abc is taken over orbits a >= b >= c with the weights A of Eq.
// E_corr_CCSD_T (1, 1/2, 1/6) and the six orbit positions P0..P5 = abc, acb,
// bac, bca, cab, cba.  With even positions {P0,P3,P4} and odd {P1,P2,P5}, the
// orbit sum T = sum_n W_n R[V]_n collapses to
//   T = 3 sum_n W_n V_n + Ae Se + Ao So - 2 (Ae So + Ao Se),
// Ae/Ao the sums of W over even/odd positions, Se/So those of V.
// D, 1/D, A T / D and every sum are float64.
#include "te_internal.h"

namespace te {

// block-order permutations: PERM[n] = slots of positions P0..P5
__constant__ int c_perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

template <int N>
struct Rot {  // index of the permutation (s1,s2,s0) and (s2,s0,s1) for position N
  static constexpr int r1 = (N == 0) ? 3 : (N == 1) ? 5 : (N == 2) ? 1 : (N == 3) ? 4 : (N == 4) ? 0 : 2;
  static constexpr int r2 = (N == 0) ? 4 : (N == 1) ? 2 : (N == 2) ? 5 : (N == 3) ? 0 : (N == 4) ? 3 : 1;
  static constexpr int s0 = (N <= 1) ? 0 : (N <= 3) ? 1 : 2;
  static constexpr int s1 = (N == 0) ? 1 : (N == 1) ? 2 : (N == 2) ? 0 : (N == 3) ? 2 : (N == 4) ? 0 : 1;
  static constexpr int s2 = 3 - s0 - s1;
};

__device__ __forceinline__ void decode_block_triple(int64_t bt, int& X, int& Y, int& Z) {
  // bt = X(X+1)(X+2)/6 + Y(Y+1)/2 + Z with X >= Y >= Z >= 0
  int x = (int)cbrt(6.0 * (double)bt);
  while ((int64_t)x * (x + 1) * (x + 2) / 6 > bt) --x;
  while ((int64_t)(x + 1) * (x + 2) * (x + 3) / 6 <= bt) ++x;
  int64_t rem = bt - (int64_t)x * (x + 1) * (x + 2) / 6;
  int y = (int)sqrt(2.0 * (double)rem);
  while ((int64_t)y * (y + 1) / 2 > rem) --y;
  while ((int64_t)(y + 1) * (y + 2) / 2 <= rem) ++y;
  X = x;
  Y = y;
  Z = (int)(rem - (int64_t)y * (y + 1) / 2);
}

template <typename T, int N>
__device__ __forceinline__ void position(const T* cube, const T* ovsS, const T* t1S, const int* l,
                                         T& Wn, T& Vn) {
  constexpr int TB = ENERGY_TB, TB3 = TB * TB * TB;
  constexpr int s0 = Rot<N>::s0, s1 = Rot<N>::s1, s2 = Rot<N>::s2;
  const int x = l[s0], y = l[s1], z = l[s2];
  // W~[x,y,z] = G0[x][y][z] + G1[y][z][x] + G2[z][x][y]
  Wn = cube[(0 * 6 + N) * TB3 + (x * TB + y) * TB + z]
     + cube[(1 * 6 + Rot<N>::r1) * TB3 + (y * TB + z) * TB + x]
     + cube[(2 * 6 + Rot<N>::r2) * TB3 + (z * TB + x) * TB + y];
  // Y[x,y,z] = ovs(i,x,j,y) t1(k,z) + ovs(j,y,k,z) t1(i,x) + ovs(i,x,k,z) t1(j,y)
  const T yv = ovsS[((0 * 3 + s0) * 3 + s1) * TB * TB + x * TB + y] * t1S[(2 * 3 + s2) * TB + z]
             + ovsS[((1 * 3 + s1) * 3 + s2) * TB * TB + y * TB + z] * t1S[(0 * 3 + s0) * TB + x]
             + ovsS[((2 * 3 + s0) * 3 + s2) * TB * TB + x * TB + z] * t1S[(1 * 3 + s1) * TB + y];
  Vn = Wn + yv;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_energy(const T* __restrict__ gbuf, int o, int v, int ldz, const Triple* __restrict__ triples, int64_t t0,
         const double* __restrict__ eps_o, const double* __restrict__ eps_v,
         const T* __restrict__ ovs, const T* __restrict__ t1, double* __restrict__ partials,
         int64_t nbt) {
  constexpr int TB = ENERGY_TB, TB3 = TB * TB * TB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* cube = reinterpret_cast<T*>(smem_raw);  // [3 G][6 block orders][TB^3]
  T* ovsS = cube + 18 * TB3;                 // [3 pairs ij,jk,ik][3][3][TB][TB]
  T* t1S = ovsS + 27 * TB * TB;              // [3 i,j,k][3][TB]
  double* epsS = reinterpret_cast<double*>(t1S + 9 * TB + (sizeof(T) == 4 ? 8 : 0));  // [3][TB]
  __shared__ double red[8];

  const int tid = threadIdx.x;
  const int slot = blockIdx.y;
  const int64_t bt = blockIdx.x;
  int blk[3];
  decode_block_triple(bt, blk[0], blk[1], blk[2]);
  const Triple tr = triples[t0 + slot];
  const int64_t v2 = (int64_t)v * v;
  const int64_t gstride = v2 * ldz;  // one G block: [v][v][ldz]
  const T* G = gbuf + (int64_t)slot * 3 * gstride;

  for (int idx = tid; idx < 18 * TB3; idx += blockDim.x) {
    const int e = idx % TB3, cp = idx / TB3;
    const int g = cp / 6, pid = cp % 6;
    const int u = e / (TB * TB), w = (e / TB) % TB, z = e % TB;
    const int x = blk[c_perm[pid][0]] * TB + u;
    const int y = blk[c_perm[pid][1]] * TB + w;
    const int zz = blk[c_perm[pid][2]] * TB + z;
    T val = T(0);
    if (x < v && y < v && zz < v) val = G[g * gstride + ((int64_t)x * v + y) * ldz + zz];
    cube[idx] = val;
  }
  for (int idx = tid; idx < 27 * TB * TB; idx += blockDim.x) {
    const int pair = idx / (9 * TB * TB);
    const int rem = idx % (9 * TB * TB);
    const int sx = rem / (3 * TB * TB), sy = (rem / (TB * TB)) % 3;
    const int u = (rem / TB) % TB, w = rem % TB;
    const int P1 = (pair == 1) ? tr.j : tr.i;
    const int P2 = (pair == 0) ? tr.j : tr.k;
    const int x = blk[sx] * TB + u, y = blk[sy] * TB + w;
    T val = T(0);
    if (x < v && y < v) val = ovs[(((int64_t)P1 * v + x) * o + P2) * v + y];
    ovsS[idx] = val;
  }
  if (tid < 9 * TB) {
    const int which = tid / (3 * TB), s = (tid / TB) % 3, u = tid % TB;
    const int occ = (which == 0) ? tr.i : (which == 1) ? tr.j : tr.k;
    const int x = blk[s] * TB + u;
    t1S[tid] = (x < v) ? t1[(int64_t)occ * v + x] : T(0);
  }
  if (tid < 3 * TB) {
    const int s = tid / TB, u = tid % TB;
    const int x = blk[s] * TB + u;
    epsS[tid] = (x < v) ? eps_v[x] : 0.0;
  }
  __syncthreads();

  const double eo = eps_o[tr.i] + eps_o[tr.j] + eps_o[tr.k];
  double acc = 0.0;
  for (int rr = tid; rr < TB3; rr += blockDim.x) {
    const int la = rr / (TB * TB), lb = (rr / TB) % TB, lc = rr % TB;
    const int a = blk[0] * TB + la, b = blk[1] * TB + lb, c = blk[2] * TB + lc;
    if (a >= v || b >= v || c >= v) continue;
    if (blk[0] == blk[1] && la < lb) continue;
    if (blk[1] == blk[2] && lb < lc) continue;
    const int l[3] = {la, lb, lc};
    T W0, W1, W2, W3, W4, W5, V0, V1, V2, V3, V4, V5;
    position<T, 0>(cube, ovsS, t1S, l, W0, V0);
    position<T, 1>(cube, ovsS, t1S, l, W1, V1);
    position<T, 2>(cube, ovsS, t1S, l, W2, V2);
    position<T, 3>(cube, ovsS, t1S, l, W3, V3);
    position<T, 4>(cube, ovsS, t1S, l, W4, V4);
    position<T, 5>(cube, ovsS, t1S, l, W5, V5);
    const T Ae = W0 + W3 + W4, Ao = W1 + W2 + W5;
    const T Se = V0 + V3 + V4, So = V1 + V2 + V5;
    const T dot = W0 * V0 + W1 * V1 + W2 * V2 + W3 * V3 + W4 * V4 + W5 * V5;
    const T Tv = T(3) * dot + Ae * Se + Ao * So - T(2) * (Ae * So + Ao * Se);
    const double wA = (a == b && b == c) ? (1.0 / 6.0) : ((a == b || b == c) ? 0.5 : 1.0);
    const double D = eo - epsS[la] - epsS[TB + lb] - epsS[2 * TB + lc];
    acc = fma(wA * (double)Tv, __drcp_rn(D), acc);
  }
  // fixed-order block reduction
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((tid & 31) == 0) red[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    partials[(int64_t)slot * nbt + bt] = s;
  }
}

template <typename T>
static cudaError_t launch_energy(const Prepared* P, const Triple* d_triples, int64_t t0, int nslots,
                                 const T* gbuf, int ldz, const T* ovs, const T* t1, double* partials,
                                 int64_t nbt, cudaStream_t s) {
  constexpr int TB = ENERGY_TB, TB3 = TB * TB * TB;
  const size_t smem = sizeof(T) * (18 * TB3 + 27 * TB * TB + 9 * TB + (sizeof(T) == 4 ? 8 : 0)) +
                      sizeof(double) * 3 * TB;
  static bool attr_set[2] = {false, false};
  bool& done = attr_set[sizeof(T) == 8];
  if (!done) {
    cudaError_t e = cudaFuncSetAttribute(k_energy<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    done = true;
  }
  dim3 grid((unsigned)nbt, (unsigned)nslots);
  k_energy<T><<<grid, 256, smem, s>>>(gbuf, P->o, P->v, ldz, d_triples, t0, P->eps_o, P->eps_v, ovs, t1,
                                      partials, nbt);
  return cudaGetLastError();
}

cudaError_t launch_energy_f64(const Prepared* P, const Triple* d_triples, int64_t t0, int nslots,
                              const double* gbuf, double* partials, int64_t nbt, cudaStream_t s) {
  return launch_energy<double>(P, d_triples, t0, nslots, gbuf, P->v, P->ovs, P->t1, partials, nbt, s);
}

cudaError_t launch_energy_f32(const Prepared* P, const Triple* d_triples, int64_t t0, int nslots,
                              const float* gbuf, int ldz, double* partials, int64_t nbt, cudaStream_t s) {
  return launch_energy<float>(P, d_triples, t0, nslots, gbuf, ldz, P->ovs32, P->t1_32, partials, nbt, s);
}

// ---------------------------------------------------------------------------
// Deterministic compensated sums
// ---------------------------------------------------------------------------

__device__ __forceinline__ void neumaier_add(double& s, double& c, double x) {
  const double t = s + x;
  if (fabs(s) >= fabs(x)) c += (s - t) + x;
  else c += (x - t) + s;
  s = t;
}

// Sum x[0..n) in a fixed order: thread t takes t, t+256, ...; then a fixed tree.
__device__ double block_sum_fixed(const double* __restrict__ x, int64_t n) {
  __shared__ double ss[256], cc[256];
  double s = 0.0, c = 0.0;
  for (int64_t idx = threadIdx.x; idx < n; idx += blockDim.x) neumaier_add(s, c, x[idx]);
  ss[threadIdx.x] = s;
  cc[threadIdx.x] = c;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      double s1 = ss[threadIdx.x], c1 = cc[threadIdx.x] + cc[threadIdx.x + w];
      neumaier_add(s1, c1, ss[threadIdx.x + w]);
      ss[threadIdx.x] = s1;
      cc[threadIdx.x] = c1;
    }
    __syncthreads();
  }
  const double r = ss[0] + cc[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(256)
k_reduce_triples(const double* __restrict__ partials, int64_t nbt, const Triple* __restrict__ triples,
                 int64_t t0, double* __restrict__ e_out) {
  const int slot = blockIdx.x;
  const double s = block_sum_fixed(partials + (int64_t)slot * nbt, nbt);
  if (threadIdx.x == 0) e_out[slot] = s * ((double)triples[t0 + slot].m / 3.0);
}

__global__ void __launch_bounds__(256)
k_reduce_total(const double* __restrict__ e_triples, int64_t n, double* __restrict__ e_out) {
  const double s = block_sum_fixed(e_triples, n);
  if (threadIdx.x == 0) *e_out = s;
}

cudaError_t launch_reduce_triples(const double* partials, int64_t nbt, const Triple* d_triples,
                                  int64_t t0, int nslots, double* e_out, cudaStream_t s) {
  k_reduce_triples<<<nslots, 256, 0, s>>>(partials, nbt, d_triples, t0, e_out);
  return cudaGetLastError();
}

cudaError_t launch_reduce_total(const double* e_triples, int64_t n, double* e_out, cudaStream_t s) {
  k_reduce_total<<<1, 256, 0, s>>>(e_triples, n, e_out);
  return cudaGetLastError();
}

}  // namespace te
