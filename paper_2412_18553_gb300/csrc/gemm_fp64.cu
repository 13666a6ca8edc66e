// Float64 path: operand preparation and the W~ contractions on the DFMA units.
//
// The connected triples of one occupied triple (i,j,k) (Eq. W times D,
// supplement section on (T)) are assembled from three "G" blocks,
//
//   W~_{ijk}[a,b,c] = G(i,j,k)[a,b,c] + G(j,k,i)[b,c,a] + G(k,i,j)[c,a,b],
//
//   G(p,q,r)[x,y,z] = sum_d ( (px|yd) t_{rq}^{zd} + (qy|xd) t_{rp}^{zd} )
//                   - sum_l ( t_{lp}^{yx} (ql|rz) + t_{lq}^{xy} (pl|rz) )
//
// written as one GEMM per (p,q,r): rows (x,y) flattened (v^2), columns z (v),
// and a K axis made of four segments:
//   S1  A = ovvv[p, x, y, :]        B = t2[r, q, z, :]            K = v
//   S2  A = ovvv[q, y, x, :]        B = t2[r, p, z, :]            K = v
//   S3  A = t2L[p, y, x, :]         B = nooT[q, r, z, :]          K = o
//   S4  A = t2L[q, x, y, :]         B = nooT[p, r, z, :]          K = o
// with t2L[q][x][y][l] = t2[l,q,x,y] and nooT[p][r][z][l] = -ooov[p,l,r,z].
// Each of the six terms of the permutation operator P appears exactly once in
// the three G blocks (S1/S2 carry the sum over d, S3/S4 the sum over l).
#include "te_internal.h"

namespace te {

// ---------------------------------------------------------------------------
// preparation kernels (float64)
// ---------------------------------------------------------------------------

__global__ void k_prep_t2L(const double* __restrict__ t2, double* __restrict__ t2L, int o, int v) {
  const int64_t n = (int64_t)o * v * v * o;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(idx % o);
    int64_t rest = idx / o;
    const int b = (int)(rest % v);
    rest /= v;
    const int a = (int)(rest % v);
    const int q = (int)(rest / v);
    t2L[idx] = t2[(((int64_t)l * o + q) * v + a) * v + b];
  }
}

__global__ void k_prep_nooT(const double* __restrict__ ooov, double* __restrict__ nooT, int o, int v) {
  const int64_t n = (int64_t)o * o * v * o;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(idx % o);
    int64_t rest = idx / o;
    const int z = (int)(rest % v);
    rest /= v;
    const int r = (int)(rest % o);
    const int p = (int)(rest / o);
    nooT[idx] = -ooov[(((int64_t)p * o + l) * o + r) * v + z];
  }
}

__global__ void k_prep_ovs(const double* __restrict__ ovov, double* __restrict__ ovs,
                           float* __restrict__ ovs32, int o, int v) {
  const int64_t n = (int64_t)o * v * o * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(idx % v);
    int64_t rest = idx / v;
    const int j = (int)(rest % o);
    rest /= o;
    const int a = (int)(rest % v);
    const int i = (int)(rest / v);
    const double s = 0.5 * (ovov[idx] + ovov[(((int64_t)j * v + b) * o + i) * v + a]);
    if (ovs) ovs[idx] = s;
    if (ovs32) ovs32[idx] = (float)s;
  }
}

__global__ void k_to_f32(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x)
    y[idx] = (float)x[idx];
}

static int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 8192) g = 8192;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_prep_fp64(const te_cluster* c, Prepared* P, cudaStream_t s) {
  const int o = (int)c->nocc, v = (int)c->nvir;
  // the tensor-core adjoint reads its own slice planes: no float64 t2L / nooT copies
  if (P->t2L) k_prep_t2L<<<grid_for((int64_t)o * v * v * o), 256, 0, s>>>(c->t2, P->t2L, o, v);
  if (P->nooT) k_prep_nooT<<<grid_for((int64_t)o * o * v * o), 256, 0, s>>>(c->ooov, P->nooT, o, v);
  k_prep_ovs<<<grid_for((int64_t)o * v * o * v), 256, 0, s>>>(c->ovov, P->ovs, P->ovs32, o, v);
  if (P->t1_32) k_to_f32<<<grid_for((int64_t)o * v), 256, 0, s>>>(c->t1, P->t1_32, (int64_t)o * v);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// DFMA GEMM: one CTA = 64 rows (x,y) x 64 columns z of one G block
// ---------------------------------------------------------------------------

constexpr int FT = 64;  // tile edge
constexpr int FK = 16;  // K chunk

__global__ void __launch_bounds__(256)
k_gemm_fp64(const double* __restrict__ ovvv, const double* __restrict__ t2,
            const double* __restrict__ t2L, const double* __restrict__ nooT,
            const Triple* __restrict__ triples, int64_t t0, int o, int v,
            double* __restrict__ gbuf) {
  __shared__ double As[FK][FT + 1];
  __shared__ double Bs[FK][FT + 1];
  const int tid = threadIdx.x;
  const int slot = blockIdx.z / 3;
  const int g = blockIdx.z % 3;
  const Triple T = triples[t0 + slot];
  int p, q, r;
  if (g == 0) { p = T.i; q = T.j; r = T.k; }
  else if (g == 1) { p = T.j; q = T.k; r = T.i; }
  else { p = T.k; q = T.i; r = T.j; }
  const int64_t v2 = (int64_t)v * v;
  const int64_t v3 = v2 * v;
  const int64_t row0 = (int64_t)blockIdx.x * FT;
  const int col0 = blockIdx.y * FT;

  // loader coordinates: 64 rows x 16 k, 4 consecutive k per thread
  const int lrow = tid >> 2;
  const int lk = (tid & 3) * 4;
  const int64_t R = row0 + lrow;
  const bool rvalid = R < v2;
  const int rx = rvalid ? (int)(R / v) : 0;
  const int ry = rvalid ? (int)(R % v) : 0;
  const int zc = col0 + lrow;
  const bool cvalid = zc < v;

  const int tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

  for (int seg = 0; seg < 4; ++seg) {
    const double* Arow;
    const double* Brow;
    int K;
    if (seg == 0) {
      Arow = ovvv + (int64_t)p * v3 + ((int64_t)rx * v + ry) * v;
      Brow = t2 + ((int64_t)r * o + q) * v2 + (int64_t)zc * v;
      K = v;
    } else if (seg == 1) {
      Arow = ovvv + (int64_t)q * v3 + ((int64_t)ry * v + rx) * v;
      Brow = t2 + ((int64_t)r * o + p) * v2 + (int64_t)zc * v;
      K = v;
    } else if (seg == 2) {
      Arow = t2L + (int64_t)p * v2 * o + ((int64_t)ry * v + rx) * o;
      Brow = nooT + ((int64_t)q * o + r) * v * o + (int64_t)zc * o;
      K = o;
    } else {
      Arow = t2L + (int64_t)q * v2 * o + ((int64_t)rx * v + ry) * o;
      Brow = nooT + ((int64_t)p * o + r) * v * o + (int64_t)zc * o;
      K = o;
    }
    for (int k0 = 0; k0 < K; k0 += FK) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int kk = k0 + lk + u;
        As[lk + u][lrow] = (rvalid && kk < K) ? Arow[kk] : 0.0;
        Bs[lk + u][lrow] = (cvalid && kk < K) ? Brow[kk] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < FK; ++kk) {
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
  }
  double* out = gbuf + ((int64_t)slot * 3 + g) * v3;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t Ro = row0 + ty * 4 + a;
    if (Ro >= v2) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int z = col0 + tx * 4 + b;
      if (z < v) out[Ro * v + z] = acc[a][b];
    }
  }
}

cudaError_t launch_gemm_fp64(const Prepared* P, const Triple* d_triples, int64_t t0, int nslots,
                             double* gbuf, cudaStream_t s) {
  const int64_t v2 = (int64_t)P->v * P->v;
  dim3 grid((unsigned)((v2 + FT - 1) / FT), (unsigned)((P->v + FT - 1) / FT), (unsigned)(3 * nslots));
  k_gemm_fp64<<<grid, 256, 0, s>>>(P->ovvv, P->t2, P->t2L, P->nooT, d_triples, t0, P->o, P->v, gbuf);
  return cudaGetLastError();
}

}  // namespace te
