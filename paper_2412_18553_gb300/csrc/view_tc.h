// Exact-slice contractions on tcgen05 over tensor-map views (view_tc.cu).
//
// One launch runs a list of jobs.  A job is an output C[(m1, m2), n] in
// float64 and a list of K segments, each
//   C[(m1, m2), n] += jalpha alpha 2^(ea + eb) sum_{k1, k2} A[(m1, m2), (k1, k2)] B[n, (k1, k2)]
// (alpha = +-1 per segment, jalpha per job)
// where A and B are BF16 slice planes (value = 2^e sum_s slice_s) read through
// TMA tensor maps whose innermost dimension is the contiguous K index k2.
// Slice products a_i b_j with i + j <= NS - 1 go to three FP32 accumulators in
// tensor memory (level 0, level 1, the rest); K is taken in blocks of at most
// 1024 elements, so the level-0 and level-1 sums are exact.  A unit adds its
// blocks in double-float (FP32 pairs, 2^-48 relative) and its total to C (or
// to a split-K partial) in float64.
//
// Work unit: (job, m tile, n tile, K split).  A unit owns its output tile (or
// its split's partial tile) for the whole launch, so no two units write the
// same element and the result has a fixed summation order.  Jobs of one
// launch must write disjoint outputs.
#pragma once
#include <cuda.h>

#include <cstdint>

#include "te_internal.h"

namespace te {

constexpr int VT_MAX_MAPS = 16;
constexpr int VT_MAX_SEGS = 8;
constexpr int VT_MAX_JOBS = 12;
constexpr int VT_KC = 32;            // K elements per pipeline stage: 64-byte rows, 64-byte swizzle
constexpr int VT_BLOCK_CHUNKS = 32;  // stages per exact accumulation block: K <= 1024
constexpr int VT_NT_MAX = 128;       // N tile: three accumulators; an epilogue thread holds NT/2 column sums

// Which of a tensor map's five dimensions holds each index of the view; -1 when
// the view has no such index (r1 for single-index rows, k1 when K = k2 alone).
// k2 is always dimension 0 (contiguous); rows r2 come before r1.
struct VtRoles {
  int8_t k2, r2, r1, k1, s;
};

struct VtSeg {
  int8_t amap, bmap;
  int K1, K2;
  int nk2c;         // stages along k2: ceil(K2 / VT_KC)
  int nchunks;      // K1 * nk2c
  int bchunks;      // stages per accumulation block (at most VT_BLOCK_CHUNKS)
  int nblk;         // accumulation blocks: ceil(nchunks / bchunks)
  int afix[5], bfix[5];  // coordinates of the dimensions with no role (group indices)
  const int* ea;    // scale exponents (device)
  const int* eb;
  double alpha;     // +1 or -1 (a job's common factor is VtJob::jalpha)
};

struct VtJob {
  int M1, M2, N;
  int TA, TB, NT;   // row tile TA values of m1 x TB values of m2 (TA TB = 128); NT columns
  int nm1, nm2, nn, nsplit, nseg;
  int overwrite;    // the first block of a unit stores (nsplit == 1 only)
  double jalpha;    // factor of the whole job (1 unless set)
  int64_t unit0;    // first unit of the job in the launch
  int64_t nblocks;  // accumulation blocks over all segments
  double* C;        // element (m1, m2, n) at m1 c_m1 + m2 c_m2 + n c_n
  int64_t c_m1, c_m2, c_n;
  double* part;     // nsplit > 1: [nsplit][M1 M2][N], added into C by vt_launch
  int64_t red0;     // first element of the job in the launch's split-reduction index space
  VtSeg seg[VT_MAX_SEGS];
};

struct VtMaps {
  CUtensorMap m[VT_MAX_MAPS];
};

struct VtParams {
  int njobs, ns;
  int stages;
  uint32_t stage_bytes;  // A part (ns x 128 rows x 64 B) then B part (ns x nt_max rows x 64 B)
  uint32_t tmem_cols;
  int nt_max;
  int64_t total_units;
  int64_t total_red;     // outputs of the split jobs
  unsigned int* err;
  unsigned long long wait_ns;
  VtRoles roles[VT_MAX_MAPS];
  VtJob job[VT_MAX_JOBS];
};

// A BF16 slice array seen through a five-dimensional tensor map: dims and
// strides in elements (stride[0] = 1), the roles of the dimensions, and the
// plane stride is the stride of the role-s dimension.
struct VtView {
  const void* base;
  uint64_t dims[5];
  uint64_t stride[5];
  VtRoles roles;
};

// Encoded views shared by the launches of one call.
constexpr int VT_BANK_MAX = 24;
struct VtBank {
  CUtensorMap m[VT_BANK_MAX];
  VtRoles r[VT_BANK_MAX];
  int n;
};
// Encode a view (rows per box: rows_r2 x rows_r1, rows_r1 = 1 for
// single-index rows) as bank entry *idx; fails if a stride or the base breaks
// the tensor-map rules.
te_status vt_bank_add(VtBank* k, const VtView& v, int rows_r2, int rows_r1, int* idx);

// Host-side launch under construction.
struct VtBuild {
  VtMaps maps;
  VtParams P;
  int nmaps;
  int8_t slot[VT_BANK_MAX];  // launch-local map index of each bank entry, -1 if unused
};

void vt_begin(VtBuild* b, int ns);
// launch-local map index of bank entry idx (copied on first use); -1 when the
// launch holds VT_MAX_MAPS maps already
int vt_use(VtBuild* b, const VtBank& k, int idx);
// Append a job; segments are filled by the caller through the returned pointer.
VtJob* vt_job(VtBuild* b, int M1, int M2, int N, int TA, int TB, int NT, double* C, int64_t c_m1, int64_t c_m2,
              int64_t c_n, int overwrite);
void vt_seg(VtJob* j, int amap, int bmap, int K1, int K2, const int* afix, const int* bfix, const int* ea,
            const int* eb, double alpha);
// Choose split counts (jobs that overwrite, or all jobs when part_scratch is
// null, keep one split) and unit offsets; part_scratch holds the partials,
// consecutively per split job.  The doubles of scratch used go to *used.
te_status vt_finish(VtBuild* b, int num_sms, double* part_scratch, int64_t scratch_cap, int64_t* used);
// Split count and partial doubles vt_finish chooses for a job of `tiles`
// output tiles, `nblocks` accumulation blocks and mn outputs.
int64_t vt_splits(int64_t tiles, int64_t nblocks, int num_sms);
int64_t vt_split_doubles(int64_t tiles, int64_t nblocks, int64_t mn, int num_sms);
// Accumulation blocks of one segment over K = K1 x K2 with bchunks stages per
// block.
int64_t vt_seg_blocks(int K1, int K2, int bchunks = VT_BLOCK_CHUNKS);
// Stages per block for a job with few output tiles (more units to split K
// over; each block still ends in exact level-0/1 sums).
constexpr int VT_SPLIT_CHUNKS = 8;
// Launch the units (grid: min(units, SMs)), then add the split partials of
// every job into C in split order.
te_status vt_launch(Handle* h, VtBuild* b, cudaStream_t s);

// N tile for an output of n columns: at most VT_NT_MAX, a multiple of 16.
int vt_ntile(int64_t n);

struct SliceSet;
// The six views of an exact-slice operand set (tc_prepare_slices) that the
// four K segments of a G block read, rows (x, y) in tiles of 8 x 16 and z in
// tiles of nt: idx[0..5] = ovvv rows (x, y), ovvv rows (y, x), t2L rows
// (x, y), t2L rows (y, x), t2 rows z, nooT rows z.  Group coordinates: ovvv
// and t2L take their occupied index at dimension 4; t2[r][q] takes q at 3 and
// r at 4; nooT[p][r] takes r at 3 and p at 4.
te_status vt_slice_maps(VtBank* k, const SliceSet& S, int o, int v, int nt, int* idx);

// Tiled transpose of BF16 slice planes: for every plane p < np and batch b <
// nb, dst[p][b][c][r] = src[p][b][r][c] over r < R, c < Cc (element strides
// given; the innermost index of each side is contiguous).
cudaError_t vt_transpose(const void* src, int64_t src_ps, int64_t src_bs, int64_t src_rs, void* dst,
                         int64_t dst_ps, int64_t dst_bs, int64_t dst_cs, int np, int nb, int R, int Cc,
                         cudaStream_t s);

}  // namespace te
