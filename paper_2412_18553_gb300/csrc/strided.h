// Strided-view contractions shared by the adjoint (vjp.cu) and the
// fragment-projected energy (frag.cu): a float64 DFMA GEMM and an exact-slice
// BF16 tensor-core GEMM over two-index row and K views, and the per-element
// assembly of W~ and Y from a triple's three natural-layout G blocks.
#pragma once
#include <cuda_bf16.h>

#include "te_internal.h"

namespace te {

// one unique triple's epilogue arguments
struct AdjArgs {
  int o, v;
  int i, j, k;
  double w;  // gE * m / 3
  const double* G;      // [3][v][v][v] for this triple
  const double* ovs;    // [o][v][o][v]
  const double* t1;     // [o][v]
  const double* eps_o;
  const double* eps_v;
  double* dW;           // [v^3]
  double* dY;           // [v^3]
  double* dD;           // [v^3]
  double* epart;        // per-block partial energies (unweighted by gE: m/3 e)
  unsigned long long* dwmax;  // if set: max |dW~| (bit pattern of a non-negative double)
  double* dpart;        // per-block sums of dD (the orbital-energy gradient of the triple's occupied indices)
};

__device__ __forceinline__ double wt_at(const AdjArgs& A, int x, int y, int z) {
  const int64_t v = A.v, v2 = v * v, v3 = v2 * v;
  return A.G[(x * v + y) * v + z] + A.G[v3 + (y * v + z) * v + x] + A.G[2 * v3 + (z * v + x) * v + y];
}

__device__ __forceinline__ double y_at(const AdjArgs& A, int x, int y, int z) {
  const int64_t v = A.v, o = A.o;
  auto ovs = [&](int P1, int a, int P2, int b) { return A.ovs[(((int64_t)P1 * v + a) * o + P2) * v + b]; };
  return ovs(A.i, x, A.j, y) * A.t1[(int64_t)A.k * v + z] + ovs(A.j, y, A.k, z) * A.t1[(int64_t)A.i * v + x] +
         ovs(A.i, x, A.k, z) * A.t1[(int64_t)A.j * v + y];
}

// The orbit of (a, b, c) under permutations, positions in the order abc,
// acb, bac, bca, cab, cba (0, 3, 4 even; 1, 2, 5 odd): their linear indices,
// and which of them are distinct elements (a = b or b = c merge positions).
__device__ __forceinline__ void orbit_index(int64_t v, int a, int b, int c, int64_t* idx) {
  idx[0] = (a * v + b) * v + c;
  idx[1] = (a * v + c) * v + b;
  idx[2] = (b * v + a) * v + c;
  idx[3] = (b * v + c) * v + a;
  idx[4] = (c * v + a) * v + b;
  idx[5] = (c * v + b) * v + a;
}
__device__ __forceinline__ unsigned orbit_distinct(int a, int b, int c) {
  if (a == b && b == c) return 0x01u;
  if (a == b) return 0x13u;  // abc = bac, acb = bca, cab = cba: keep 0, 1, 4
  if (b == c) return 0x0Du;  // abc = acb, bac = cab, bca = cba: keep 0, 2, 3
  return 0x3Fu;
}
// R at every position of the orbit (identity 4, 3-cycles +1, transpositions
// -2): 3 x_p + (sum over p's parity class) - 2 (sum over the other class)
__device__ __forceinline__ void r_orbit(const double* x, double* r) {
  const double se = (x[0] + x[3]) + x[4], so = (x[1] + x[2]) + x[5];
  r[0] = (3.0 * x[0] + se) - 2.0 * so;
  r[3] = (3.0 * x[3] + se) - 2.0 * so;
  r[4] = (3.0 * x[4] + se) - 2.0 * so;
  r[1] = (3.0 * x[1] + so) - 2.0 * se;
  r[2] = (3.0 * x[2] + so) - 2.0 * se;
  r[5] = (3.0 * x[5] + so) - 2.0 * se;
}
// W~ and Y at the six positions of the orbit of (a, b, c)
__device__ __forceinline__ void orbit_values(const AdjArgs& A, int a, int b, int c, double* W, double* Y) {
  const int p[6][3] = {{a, b, c}, {a, c, b}, {b, a, c}, {b, c, a}, {c, a, b}, {c, b, a}};
#pragma unroll
  for (int n = 0; n < 6; ++n) {
    W[n] = wt_at(A, p[n][0], p[n][1], p[n][2]);
    Y[n] = y_at(A, p[n][0], p[n][1], p[n][2]);
  }
}

// Exact slices of x with |x| < 2^e: N = round(x 2^(7 NS - e)) taken from the
// bits of x (no float64 arithmetic: GB300's float64 rate is low), written as
// balanced base-128 digits N = sum_k d_k 128^(NS-1-k), |d_k| <= 128.  Slice k
// is d_k 2^-7(k+1), exact in BF16, and x = 2^e sum_k slice_k to within
// 2^(e - 7 NS - 1).  Zeros and subnormals give N = 0; non-finite x gives
// unspecified digits.
template <int NS>
__device__ __forceinline__ void slice_digits(double x, int e, float* d) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7FFull);
  long long N = 0;
  if (E != 0) {
    // x = M 2^(E - 1075), so x 2^(7 NS - e) = M 2^-sh; |x| < 2^e gives sh >= 18
    const unsigned long long M = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = 1075 - E - 7 * NS + e;
    if (sh > 0 && sh < 64) N = (long long)((M + (1ull << (sh - 1))) >> sh);
    if (bits >> 63) N = -N;
  }
#pragma unroll
  for (int k = NS - 1; k > 0; --k) {
    const int dk = (int)((N + 64) & 127) - 64;
    d[k] = (float)dk;
    N = (N - dk) >> 7;
  }
  d[0] = (float)N;
}

// C[m,n] += alpha sum_k A[m,k] B[k,n], m = (m1, m2) and k = (k1, k2) with a
// stride per index (float64, DFMA; deterministic split-K)
struct GemmView {
  const double* A;
  const double* B;
  double* C;
  int64_t M1, M2, N, K1, K2;
  int64_t a_m1, a_m2, a_k1, a_k2;
  int64_t b_k1, b_k2, b_n;
  int64_t c_m1, c_m2, c_n;
  double alpha;
};

// the same over NS BF16 slice planes per operand (slice s at base + s *
// plane; NS = ns, 4 when 0), C (+)= alpha 2^(ea + eb) sum_k A B (exact-slice
// products on mma.sync)
struct OzView {
  const __nv_bfloat16* A;
  const __nv_bfloat16* B;
  int64_t a_ps, b_ps;  // slice plane strides (elements)
  double* C;
  int64_t M1, M2, N, K1, K2;
  int64_t a_m1, a_m2, a_k1, a_k2;
  int64_t b_k1, b_k2, b_n;
  int64_t c_m1, c_m2, c_n;
  double alpha;
  const int* ea;  // device scale exponents of A's and B's slices
  const int* eb;
  int overwrite;  // store instead of accumulate (single K split only)
  int ns;         // slices per operand: 4 (also when 0) or 5
};

cudaError_t gemm_strided(const GemmView& g, int num_sms, double* scratch, int64_t scratch_cap, cudaStream_t s,
                         int64_t* launches);
cudaError_t gemm_oz(const OzView& g, int num_sms, double* scratch, int64_t scratch_cap, cudaStream_t s,
                    int64_t* launches);
// NS (4 or 5) 7-bit slice planes of x[0..n) with one power-of-two scale:
// *ex = e with 2^e > max |x| (the max's bits go to *mx), slice s at planes +
// s n.  Two launches.
cudaError_t slice_planes(const double* x, int64_t n, int ns, unsigned long long* mx, int* ex,
                         __nv_bfloat16* planes, cudaStream_t s, int64_t* launches);
// doubles of split-K scratch gemm_oz needs for an M x N output over K
int64_t gemm_oz_scratch(int64_t M, int64_t N, int64_t K, int num_sms);
// doubles of split-K scratch the two GEMMs need for a cluster's contractions
int64_t splitk_cap(int64_t o, int64_t v);
int64_t oz_scratch_cap(int64_t o, int64_t v, int num_sms);
// out = scale * (fixed-order sum of part[0..n))
cudaError_t launch_sum_share(const double* part, int64_t n, double scale, double* out, cudaStream_t s);

}  // namespace te
