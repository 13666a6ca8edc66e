// Fragment-projected E(T) (Eq. E_corr_CCSD_T with a general C^f) on the
// strided-view contractions of the adjoint; see the comment below.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "strided.h"
#include "tc_path.h"
#include "view_tc.h"
#include "te_internal.h"

namespace te {

te_status ensure_workspace_public(Handle* h, size_t bytes);
te_status ensure_triples_public(Handle* h, int nocc);

// ---------------------------------------------------------------------------
// Fragment-projected E(T): Eq. E_corr_CCSD_T with a general C^f
// ---------------------------------------------------------------------------
// E_x = (1/3) sum_{ijk} sum_{abc} sum_{i'} C_{ii'} W~_{i'jk} R[Z]_{ijk}: C acts on
// the first occupied index of W~.  Summed over all ordered triples, C on any
// one of the three occupied indices gives the same total, so every unique
// triple takes the average S W~ = 1/3 (C_1 + C_2 + C_3) W~, which keeps the
// joint (ijk, abc) permutation symmetry of W~:
//   share_{ijk} = (m/3) sum_{abc} (S W~)_{ijk} R[V]_{ijk} / D_{ijk},  V = W~ + Y.
// S W~ = P[S X] groups into G-like blocks like W~ = P[X].  C on one occupied
// index of a G segment lands on exactly one of its two factors, and summing
// the three placements gives two products per segment:
//   SG(p,q,r) = 1/3 [ ovvvC[p] t2[r,q] + ovvv[p] t2C[r,q] + ovvvC[q] t2[r,p] + ovvv[q] t2C[r,p]
//                     + t2LC[p] nooT[q][r] + t2L[p] nooTC[q][r] + t2LC[q] nooT[p][r] + t2L[q] nooTC[p][r] ]
// with ovvvC = C on the first index of ovvv; t2C = C on the first plus C on
// the second index of t2; t2LC = the t2L copy of t2 with C on its second
// index; nooTC = the nooT copy of ooov with C on its first plus on its third
// index.

// out[a][p][b] (+)= sum_{p'} C[p][p'] in[a][p'][b]: C on one occupied index,
// `outer` and `inner` the sizes around it; fixed summation order
__global__ void k_occ_transform(const double* __restrict__ in, const double* __restrict__ C, int o, int64_t outer,
                                int64_t inner, double* __restrict__ out, int accumulate) {
  const int64_t n = outer * o * inner;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e / (o * inner), b = e % inner;
    const int p = (int)((e / inner) % o);
    const double* src = in + a * o * inner + b;
    double s = 0.0;
    for (int q = 0; q < o; ++q) s += C[p * o + q] * src[q * inner];
    out[e] = accumulate ? out[e] + s : s;
  }
}

// per-block sums of (S W~) R[V] / D over the abc of one triple, one thread per
// orbit representative a >= b >= c
__global__ void __launch_bounds__(256) k_energy_proj(AdjArgs A, const double* __restrict__ SG) {
  __shared__ double red[8];
  const int64_t v = A.v, v3 = v * v * v;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double contrib = 0.0;
  if (e < v3) {
    const int a = (int)(e / (v * v)), b = (int)((e / v) % v), c = (int)(e % v);
    if (a >= b && b >= c) {
      double W[6], Y[6], V[6], RV[6];
      orbit_values(A, a, b, c, W, Y);
#pragma unroll
      for (int n = 0; n < 6; ++n) V[n] = W[n] + Y[n];
      r_orbit(V, RV);
      AdjArgs S = A;
      S.G = SG;
      const int p[6][3] = {{a, b, c}, {a, c, b}, {b, a, c}, {b, c, a}, {c, a, b}, {c, b, a}};
      const unsigned distinct = orbit_distinct(a, b, c);
      const double D = (A.eps_o[A.i] + A.eps_o[A.j] + A.eps_o[A.k]) - A.eps_v[a] - A.eps_v[b] - A.eps_v[c];
      double t = 0.0;
#pragma unroll
      for (int n = 0; n < 6; ++n)
        if (distinct >> n & 1u) t += wt_at(S, p[n][0], p[n][1], p[n][2]) * RV[n];
      contrib = t / D;
    }
  }
  for (int off = 16; off > 0; off >>= 1) contrib += __shfl_down_sync(0xffffffffu, contrib, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = contrib;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    A.epart[blockIdx.x] = t;
  }
}

struct FragWork {
  double *ovvvC, *t2C, *t2C2, *ooovC;      // C on occupied indices of the inputs
  double *t2L, *nooT, *ovs;                // float64 helper copies of the inputs
  double *t2LC, *nooTC, *ovs_unused;       // the same of t2C2 and ooovC
  double *G, *SG;                          // [3][v][v][v] each
  double *epart, *shares, *scratch;
  int64_t scratch_cap;
  char* slices[3];                         // exact-slice planes (mixed precision only)
};

static size_t frag_layout(int64_t o, int64_t v, bool slices, int num_sms, char* base, FragWork* W);

size_t frag_bytes(int64_t o, int64_t v, te_precision p, int num_sms) {
  FragWork W;
  return frag_layout(o, v, p != TE_FP64, num_sms, nullptr, &W);
}

// carve the workspace (base = nullptr: sizes only)
static size_t frag_layout(int64_t o, int64_t v, bool slices, int num_sms, char* base, FragWork* W) {
  const int64_t v3 = v * v * v, nt = num_unique_triples(o), nblk = (v3 + 255) / 256;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 1023) & ~size_t(1023);
    char* r = base ? base + off : nullptr;
    off += bytes;
    return r;
  };
  auto d = [&](int64_t n) { return reinterpret_cast<double*>(take((size_t)n * 8)); };
  W->ovvvC = d(o * v3);
  W->t2C = d(o * o * v * v);
  W->t2C2 = d(o * o * v * v);
  W->ooovC = d(o * o * o * v);
  W->t2L = d(o * v * v * o);
  W->nooT = d(o * o * v * o);
  W->ovs = d(o * v * o * v);
  W->t2LC = d(o * v * v * o);
  W->nooTC = d(o * o * v * o);
  W->ovs_unused = d(o * v * o * v);
  W->G = d(3 * v3);
  W->SG = d(3 * v3);
  W->epart = d(nblk);
  W->shares = d(std::max<int64_t>(1, nt));
  W->scratch_cap = slices ? oz_scratch_cap(o, v, num_sms) : splitk_cap(o, v);
  W->scratch = d(W->scratch_cap);
  for (int k = 0; k < 3; ++k) W->slices[k] = slices ? take(tc_slices_bytes((int)o, (int)v) + 1024) : nullptr;
  return off + 1024;
}

te_status run_frag(Handle* h, const te_cluster* c, const double* cf, te_precision p, double* e_out,
                   double* e_triples, cudaStream_t s) {
  const int o = (int)c->nocc, v = (int)c->nvir;
  const int64_t v2 = (int64_t)v * v, v3 = v2 * v, nt = num_unique_triples(o), nblk = (v3 + 255) / 256;
  const bool oz = p != TE_FP64;
  te_status st = ensure_workspace_public(h, frag_bytes(o, v, p, h->num_sms));
  if (st != TE_OK) return st;
  st = ensure_triples_public(h, o);
  if (st != TE_OK) return st;
  FragWork W;
  frag_layout(o, v, oz, h->num_sms,
              reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(h->ws) + 1023) & ~uintptr_t(1023)), &W);

  // C on the occupied indices of the inputs
  auto tr = [&](const double* in, int64_t outer, int64_t inner, double* out, int acc) {
    const int64_t n = outer * o * inner;
    k_occ_transform<<<(unsigned)std::min<int64_t>((n + 255) / 256, 8 * 1024), 256, 0, s>>>(in, cf, o, outer,
                                                                                           inner, out, acc);
    ++h->n_launches;
  };
  tr(c->ovvv, 1, v3, W.ovvvC, 0);                           // ovvv[p,a,b,d]: first index
  tr(c->t2, 1, (int64_t)o * v2, W.t2C, 0);                  // t2[r,q,a,b]: first index
  tr(c->t2, o, v2, W.t2C, 1);                               //   plus second index
  tr(c->t2, o, v2, W.t2C2, 0);                              // second index only
  tr(c->ooov, 1, (int64_t)o * o * v, W.ooovC, 0);           // ooov[p,l,r,z]: first index
  tr(c->ooov, (int64_t)o * o, v, W.ooovC, 1);               //   plus third index
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(TE_ECUDA, "transform launch: %s", cudaGetErrorString(e));

  // float64 helper copies: t2L, nooT, ovs of the inputs; t2L of t2C2, nooT of ooovC
  Prepared P{};
  P.o = o; P.v = v; P.eps_o = c->eps_o; P.eps_v = c->eps_v; P.ovvv = c->ovvv; P.t2 = c->t2; P.t1 = c->t1;
  P.t2L = W.t2L; P.nooT = W.nooT; P.ovs = W.ovs;
  e = launch_prep_fp64(c, &P, s);
  te_cluster cx = *c;
  cx.t2 = W.t2C2;
  cx.ooov = W.ooovC;
  Prepared PX{};
  PX.o = o; PX.v = v; PX.t2L = W.t2LC; PX.nooT = W.nooTC; PX.ovs = W.ovs_unused;
  if (e == cudaSuccess) e = launch_prep_fp64(&cx, &PX, s);
  h->n_launches += 6;
  if (e != cudaSuccess) return fail(TE_ECUDA, "prep: %s", cudaGetErrorString(e));

  // exact-slice planes: the inputs; (ovvvC, t2C, ooovC) for ovvv, t2 and nooT;
  // t2C2 for t2L
  SliceSet S0{}, SA{}, SB{};
  if (oz) {
    te_cluster ca = *c, cb = *c;
    ca.ovvv = W.ovvvC;
    ca.t2 = W.t2C;
    ca.ooov = W.ooovC;
    cb.t2 = W.t2C2;
    st = tc_prepare_slices(c, W.slices[0], &S0, h->num_sms, s);
    if (st == TE_OK) st = tc_prepare_slices(&ca, W.slices[1], &SA, h->num_sms, s);
    if (st == TE_OK) st = tc_prepare_slices(&cb, W.slices[2], &SB, h->num_sms, s);
    if (st != TE_OK) return st;
    h->n_launches += 18;
  }
  // exact slices: the tcgen05 view GEMM (view_tc.cu) over the six segment
  // views of each slice set, encoded once
  VtBank bank;
  bank.n = 0;
  int m0[6], mA[6], mB[6];
  const int NT = vt_ntile(v);
  if (oz) {
    if ((st = vt_slice_maps(&bank, S0, o, v, NT, m0)) != TE_OK) return st;
    if ((st = vt_slice_maps(&bank, SA, o, v, NT, mA)) != TE_OK) return st;
    if ((st = vt_slice_maps(&bank, SB, o, v, NT, mB)) != TE_OK) return st;
  }

  std::vector<Triple> trip = unique_triples(o);
  const double third = 1.0 / 3.0;
  for (int64_t t = 0; t < nt && e == cudaSuccess; ++t) {
    const Triple T = trip[t];
    if (oz) {
      // per G block (p, q, r): the block itself (S1..S4 of the input slices)
      // and its projection SG (two products per segment, one operand
      // transformed), 1/3 for the average over the three occupied slots
      VtBuild b;
      vt_begin(&b, S0.ns);
      for (int gi = 0; gi < 3; ++gi) {
        int pp, qq, rr;
        if (gi == 0) { pp = T.i; qq = T.j; rr = T.k; }
        else if (gi == 1) { pp = T.j; qq = T.k; rr = T.i; }
        else { pp = T.k; qq = T.i; rr = T.j; }
        const int f_p[5] = {0, 0, 0, 0, pp}, f_q[5] = {0, 0, 0, 0, qq};
        const int t_qr[5] = {0, 0, 0, qq, rr}, t_pr[5] = {0, 0, 0, pp, rr};
        const int n_rq[5] = {0, 0, 0, rr, qq}, n_rp[5] = {0, 0, 0, rr, pp};
        const int64_t rq = (int64_t)rr * o + qq, rp = (int64_t)rr * o + pp;
        const int64_t nqr = (int64_t)qq * o + rr, npr = (int64_t)pp * o + rr;
        auto u = [&](int m) { return vt_use(&b, bank, m); };
        VtJob* J = vt_job(&b, v, v, v, 8, 16, NT, W.G + gi * v3, v2, v, 1, 1);
        vt_seg(J, u(m0[0]), u(m0[4]), 1, v, f_p, t_qr, S0.e_ovvv + pp, S0.e_t2 + rq, 1.0);
        vt_seg(J, u(m0[1]), u(m0[4]), 1, v, f_q, t_pr, S0.e_ovvv + qq, S0.e_t2 + rp, 1.0);
        vt_seg(J, u(m0[3]), u(m0[5]), 1, o, f_p, n_rq, S0.e_t2L + pp, S0.e_nooT + nqr, 1.0);
        vt_seg(J, u(m0[2]), u(m0[5]), 1, o, f_q, n_rp, S0.e_t2L + qq, S0.e_nooT + npr, 1.0);
        VtJob* JS = vt_job(&b, v, v, v, 8, 16, NT, W.SG + gi * v3, v2, v, 1, 1);
        JS->jalpha = third;
        vt_seg(JS, u(mA[0]), u(m0[4]), 1, v, f_p, t_qr, SA.e_ovvv + pp, S0.e_t2 + rq, 1.0);  // ovvvC[p] t2[r,q]
        vt_seg(JS, u(m0[0]), u(mA[4]), 1, v, f_p, t_qr, S0.e_ovvv + pp, SA.e_t2 + rq, 1.0);  // ovvv[p] t2C[r,q]
        vt_seg(JS, u(mA[1]), u(m0[4]), 1, v, f_q, t_pr, SA.e_ovvv + qq, S0.e_t2 + rp, 1.0);  // ovvvC[q] t2[r,p]
        vt_seg(JS, u(m0[1]), u(mA[4]), 1, v, f_q, t_pr, S0.e_ovvv + qq, SA.e_t2 + rp, 1.0);  // ovvv[q] t2C[r,p]
        vt_seg(JS, u(mB[3]), u(m0[5]), 1, o, f_p, n_rq, SB.e_t2L + pp, S0.e_nooT + nqr, 1.0);  // t2LC[p] nooT[q][r]
        vt_seg(JS, u(m0[3]), u(mA[5]), 1, o, f_p, n_rq, S0.e_t2L + pp, SA.e_nooT + nqr, 1.0);  // t2L[p] nooTC[q][r]
        vt_seg(JS, u(mB[2]), u(m0[5]), 1, o, f_q, n_rp, SB.e_t2L + qq, S0.e_nooT + npr, 1.0);  // t2LC[q] nooT[p][r]
        vt_seg(JS, u(m0[2]), u(mA[5]), 1, o, f_q, n_rp, S0.e_t2L + qq, SA.e_nooT + npr, 1.0);  // t2L[q] nooTC[p][r]
      }
      if ((st = vt_finish(&b, h->num_sms, nullptr, 0, nullptr)) != TE_OK) return st;
      if ((st = vt_launch(h, &b, s)) != TE_OK) return st;
    }
    if (!oz) {
      e = cudaMemsetAsync(W.SG, 0, sizeof(double) * 3 * v3, s);
      if (e != cudaSuccess) break;
      e = launch_gemm_fp64(&P, h->d_triples, t, 1, W.G, s);
      ++h->n_launches;
    }
    for (int gi = 0; gi < 3 && e == cudaSuccess && !oz; ++gi) {
      int pp, qq, rr;
      if (gi == 0) { pp = T.i; qq = T.j; rr = T.k; }
      else if (gi == 1) { pp = T.j; qq = T.k; rr = T.i; }
      else { pp = T.k; qq = T.i; rr = T.j; }
      double* SGg = W.SG + gi * v3;
      // float64: the eight products of SG(p,q,r), rows (x, y), columns z
      auto run = [&](const double* A, int64_t am1, int64_t am2, int64_t K, const double* B, int64_t bn) {
        if (e == cudaSuccess)
          e = gemm_strided(GemmView{A, B, SGg, v, v, v, K, 1, am1, am2, 1, 0, 1, 0, bn, v2, v, 1, third}, h->num_sms,
                           W.scratch, W.scratch_cap, s, &h->n_launches);
      };
      const int64_t orq = ((int64_t)rr * o + qq) * v2, orp = ((int64_t)rr * o + pp) * v2;
      run(W.ovvvC + pp * v3, v2, v, v, c->t2 + orq, v);     // S1: ovvvC[p,x,y,d] t2[r,q,z,d]
      run(c->ovvv + pp * v3, v2, v, v, W.t2C + orq, v);     //     ovvv[p] t2C[r,q]
      run(W.ovvvC + qq * v3, v, v2, v, c->t2 + orp, v);     // S2: ovvvC[q,y,x,d] t2[r,p,z,d]
      run(c->ovvv + qq * v3, v, v2, v, W.t2C + orp, v);     //     ovvv[q] t2C[r,p]
      const int64_t lp = (int64_t)pp * v2 * o, lq = (int64_t)qq * v2 * o;
      const int64_t nqr = ((int64_t)qq * o + rr) * v * o, npr = ((int64_t)pp * o + rr) * v * o;
      run(W.t2LC + lp, o, (int64_t)v * o, o, W.nooT + nqr, o);   // S3: t2LC[p][y][x][l] nooT[q][r][z][l]
      run(W.t2L + lp, o, (int64_t)v * o, o, W.nooTC + nqr, o);   //     t2L[p] nooTC[q][r]
      run(W.t2LC + lq, (int64_t)v * o, o, o, W.nooT + npr, o);   // S4: t2LC[q][x][y][l] nooT[p][r][z][l]
      run(W.t2L + lq, (int64_t)v * o, o, o, W.nooTC + npr, o);   //     t2L[q] nooTC[p][r]
    }
    if (e != cudaSuccess) break;
    AdjArgs A{};
    A.o = o; A.v = v; A.i = T.i; A.j = T.j; A.k = T.k;
    A.G = W.G; A.ovs = W.ovs; A.t1 = c->t1; A.eps_o = c->eps_o; A.eps_v = c->eps_v; A.epart = W.epart;
    k_energy_proj<<<(unsigned)nblk, 256, 0, s>>>(A, W.SG);
    e = launch_sum_share(W.epart, nblk, (double)T.m / 3.0, W.shares + t, s);
    h->n_launches += 2;
  }
  if (e == cudaSuccess && e_triples && nt > 0)
    e = cudaMemcpyAsync(e_triples, W.shares, sizeof(double) * nt, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && e_out) {
    if (nt > 0) {
      e = launch_reduce_total(W.shares, nt, e_out, s);
      ++h->n_launches;
    } else {
      e = cudaMemsetAsync(e_out, 0, sizeof(double), s);
    }
  }
  if (e != cudaSuccess) return fail(TE_ECUDA, "projected energy launch: %s", cudaGetErrorString(e));
  return TE_OK;
}


}  // namespace te
