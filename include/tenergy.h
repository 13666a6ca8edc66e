/*
 * tenergy.h - C ABI of the GB300 library for the closed-shell perturbative
 * triples energy E(T) of an embedded cluster (supplement section "The In-situ
 * Form of Perturbative (T) in SIE", Eqs. E_corr_CCSD_T, W, V, D, P and R, with
 * the fragment projector C^f taken as the identity).
 *
 *   E(T) = (1/3) sum_{ijk} sum_{abc} W~_{ijk}^{abc} R[W~ + Y]_{ijk}^{abc} / D_{ijk}^{abc}
 *
 *   W~ = P[ sum_d (ia|bd) t_kj^cd - sum_l (ia|jl) t_lk^bc ]      (Eq. W times D)
 *   Y  = 1/2 P[ (ia|jb) t_k^c ]                                   (Eq. V times D)
 *   D  = e_i + e_j + e_k - e_a - e_b - e_c                         (Eq. D)
 *
 * which equals the printed restricted sum 2 sum_{a>=b>=c} A R[Z] W~ (Eq.
 * E_corr_CCSD_T) exactly.  Clusters are independent (Eq. C_f: E = sum_x E_x).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * - All array pointers are DEVICE pointers to float64, C-contiguous
 *   (row-major), owned by the caller; the library never frees them:
 *     eps_o [o]          occupied orbital energies (Ha)
 *     eps_v [v]          virtual orbital energies (Ha)
 *     ovvv  [o][v][v][v] ovvv[i,a,b,d] = (ia|bd)
 *     ooov  [o][o][o][v] ooov[j,l,i,a] = (jl|ia)  (= (ia|jl) for real orbitals)
 *     ovov  [o][v][o][v] ovov[i,a,j,b] = (ia|jb)
 *     t1    [o][v]       t1[i,a]       = t_i^a
 *     t2    [o][o][v][v] t2[i,j,a,b]   = t_ij^ab
 *   with o = nocc >= 1, v = nvir >= 1.  No symmetry of any array is assumed.
 * - The orbital energies must satisfy max(eps_o) < min(eps_v) (every D < 0);
 *   they need not be sorted.  Every entry must be finite.
 * - Calls are asynchronous on the given CUDA stream (0 = legacy default
 *   stream): none synchronises the stream or the device once its workspace
 *   exists (te_reserve allocates it up front).  Errors in the descriptor
 *   (null pointers, sizes, mode) are reported before any launch (TE_EINVAL);
 *   the values are checked on the device by the call's first kernel (every
 *   entry finite, max(eps_o) < min(eps_v)), and a violation is reported by
 *   the next te_sync() as TE_EINVAL, naming the array or the ordering and
 *   the cluster; the outputs of that call are then unspecified.  Workspace
 *   allocation failures give TE_ENOMEM, launch failures TE_ECUDA.  A
 *   device-side watchdog never traps: a kernel whose bounded wait expires
 *   records an error word and returns; te_sync() reports it as TE_ETIMEOUT.
 *   The error word is the handle's: it stays set until te_sync reads it.
 * - Results are deterministic: fixed-order reductions, no floating-point
 *   atomics; repeated calls give bitwise identical outputs.
 * - A handle owns its workspace (operand copies for the mixed modes, partial
 *   results); one handle must not be used from two host threads at once, and
 *   calls made on one handle with different streams must be ordered by the
 *   caller.  No exception crosses the ABI.
 *
 * Precision modes (the paper states no precision):
 *   TE_FP64    W~ contractions and everything else in float64 (DFMA);
 *   TE_TF32    W~ contractions on tcgen05 tensor cores, operands rounded to
 *              TF32, FP32 accumulation;
 *   TE_BF16X3  operands split x = hi + lo (hi = bf16(x), lo = bf16(x - hi)),
 *              three products hi*hi + hi*lo + lo*hi on tcgen05 (kind::f16),
 *              FP32 accumulation;
 *   TE_TF32X3  the same split with TF32 parts (kind::tf32).
 *   TE_OZAKI   error-free slicing after Ozaki, Ogita, Oishi and Rump (2012):
 *              every operand array is scaled by one power of two and cut
 *              into four 7-bit BF16 slices; the ten slice products down to
 *              the fifth level run on tcgen05 (kind::f16) into three FP32
 *              accumulators, the first two of which sum exact integers (no
 *              rounding in the tensor-core accumulation), and the G blocks
 *              are kept as FP32 pairs.  Meets 1e-7 Ha where FP32
 *              accumulation does not.
 *   In every mode D, 1/D, the products with 1/D and all sums are float64;
 *   the tensor-core modes form the orbit sum of R from deviations
 *   W_n - W_0 (no cancellation of the part of W~ that R annihilates).
 */
#ifndef TENERGY_H
#define TENERGY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* te_stream_t; /* the same type as cudaStream_t */

typedef enum {
  TE_OK = 0,
  TE_EINVAL = 1,        /* bad argument: null pointer, size, ordering of eps */
  TE_ENOMEM = 2,        /* workspace could not be allocated */
  TE_ECUDA = 3,         /* a CUDA runtime/driver call or launch failed */
  TE_ETIMEOUT = 4,      /* a device-side bounded wait expired (see te_sync) */
  TE_EUNSUPPORTED = 5   /* mode or size not supported on this device */
} te_status;

typedef enum {
  TE_FP64 = 0,
  TE_TF32 = 1,
  TE_BF16X3 = 2,
  TE_TF32X3 = 3,
  TE_OZAKI = 4
} te_precision;

typedef struct {
  int64_t nocc, nvir;
  const double *eps_o, *eps_v, *ovvv, *ooov, *ovov, *t1, *t2;
} te_cluster;

/* Gradient buffers: device float64, same shapes as the te_cluster arrays,
 * caller-allocated, overwritten (not accumulated).  A null member skips that
 * gradient. */
typedef struct {
  double *eps_o, *eps_v, *ovvv, *ooov, *ovov, *t1, *t2;
} te_cluster_grad;

typedef struct te_handle_s* te_handle;

/* Create a handle bound to CUDA device `device`.  Allocates nothing on the
 * device until the first compute call.  *h is set to NULL on failure.
 *
 * autotune_cache_path (nullable): a text file that keeps the tile shapes the
 * autotuner picked (t_energy_batched tunes each new (nocc, nvir, mode) once)
 * across handles and processes.  Read here if it exists: the first line names
 * the format, the SM count and the compute capability, and entries written on
 * another kind of GPU, malformed lines and shapes the tuner would not propose
 * are ignored.  Rewritten (whole, through a temporary file and a rename) after
 * every new tuning; a file that cannot be written is not an error, the tuning
 * then only lasts for the handle.  A tile shape changes the speed, never the
 * result beyond summation order inside a tile. */
te_status te_create(te_handle* h, int device, const char* autotune_cache_path);

/* Free the handle and its workspace (synchronises the device first). */
te_status te_destroy(te_handle h);

/* E(T) of one cluster.  e_out: device pointer to one double, overwritten.
 * The sum over unique occupied triples (i >= j >= k, not all equal) of the
 * per-triple shares (see t_energy_triples), reduced in a fixed order with
 * compensated float64 summation. */
te_status t_energy(te_handle h, const te_cluster* c, te_precision p,
                   double* e_out, te_stream_t s);

/* Per-triple shares of E(T) for the unique occupied triples with canonical
 * index t in [t_begin, t_end).  Canonical order: lexicographic in (i, j, k)
 * over i >= j >= k with i = j = k left out (there R vanishes), i.e. for
 * nocc = 3: (1,0,0) (1,1,0) (2,0,0) (2,1,0) (2,1,1) (2,2,0) (2,2,1).  There are
 * nocc (nocc+1)(nocc+2)/6 - nocc triples.  e_triples: device array of
 * (t_end - t_begin) doubles, overwritten with (m/3) e_ijk where m is the
 * number of distinct orderings of (i,j,k) and
 *   e_ijk = sum_{abc} W~_{ijk}^{abc} R[W~ + Y]_{ijk}^{abc} / D_{ijk}^{abc}.
 * Summed over all triples this is E(T).  Useful to shard a cluster, to
 * resume, or to check sampled triples. */
te_status t_energy_triples(te_handle h, const te_cluster* c, te_precision p,
                           int64_t t_begin, int64_t t_end,
                           double* e_triples, te_stream_t s);

/* E(T) of n independent clusters (Eq. C_f: clusters do not interact).
 * cs: HOST array of n cluster descriptors (their array pointers are device
 * pointers).  e_out: device array of n doubles, e_out[x] = E(T) of cluster x. */
te_status t_energy_batched(te_handle h, const te_cluster* cs, int64_t n,
                           te_precision p, double* e_out, te_stream_t s);

/* Vector-Jacobian product of E(T): g.X = gE * dE/dX for every non-null member
 * of *g, every stored entry of every input treated as an independent variable
 * (no symmetrisation of t2 or of the integrals).  If e_out is non-null it
 * receives E(T) (one device double).  TE_FP64 runs every contraction in
 * float64; the other modes run them on the tcgen05 tensor cores in exact
 * 7-bit BF16 slices (the TE_OZAKI scheme; gradients to ~1e-7 of each tensor's
 * largest entry), with the epilogue and all sums in float64.  Deterministic. */
te_status t_energy_vjp(te_handle h, const te_cluster* c, te_precision p,
                       double gE, double* e_out, te_cluster_grad* g,
                       te_stream_t s);

/* The adjoint restricted to the canonical triples [t_begin, t_end) (order as in
 * t_energy_triples): g.X = gE * d/dX of the sum of those triples' shares, and
 * e_out (nullable) receives that sum.  E(T) is additive over triples, so the
 * adjoints of ranges that partition [0, ntriples) add up to t_energy_vjp's
 * gradient: a caller can shard one cluster's gradient across GPUs, resume
 * it, or time and check a sample of a large cluster.  Same modes, layouts
 * and accuracy as t_energy_vjp; gradients are overwritten, not accumulated. */
te_status t_energy_vjp_triples(te_handle h, const te_cluster* c, te_precision p,
                               int64_t t_begin, int64_t t_end, double gE,
                               double* e_out, te_cluster_grad* g, te_stream_t s);

/* The adjoint of n independent clusters in one call (Eq. C_f: E = sum_x E_x,
 * so dE/dX of cluster x is that cluster's own adjoint).  cs: HOST array of n
 * descriptors; gE: HOST array of n upstream gradients (NULL: all 1);
 * e_out: device array of n doubles (nullable); grads: HOST array of n
 * gradient descriptors (device buffers, overwritten).  Every descriptor is
 * checked before any launch; the handle's workspace is sized once for the
 * largest member.  The clusters run one after another on s. */
te_status t_energy_vjp_batched(te_handle h, const te_cluster* cs, int64_t n,
                               te_precision p, const double* gE, double* e_out,
                               te_cluster_grad* grads, te_stream_t s);

/* Fragment-projected E(T) of one cluster: Eq. E_corr_CCSD_T with a general
 * C^f, i.e. the first occupied index of W~ projected,
 *   E_x = (1/3) sum_{ijk} sum_{abc} sum_{i'} cf[i][i'] W~_{i'jk}^{abc} R[Z]_{ijk}^{abc},
 * summed over all ordered occupied triples (the printed restricted sum over
 * a >= b >= c is this sum when cf is the identity; for other cf it would
 * depend on the labelling of the virtual orbitals).  cf: device float64
 * [nocc][nocc], row-major, caller-owned; a fragment projector is
 * cf[i][i'] = sum_f C[i][f] C[i'][f], symmetric, but any matrix is accepted.
 * With cf = identity the result is t_energy's.  Projectors of fragments that
 * partition the occupied space sum to t_energy (Eq. C_f).
 * p: TE_FP64 (DFMA contractions) or TE_OZAKI (exact BF16 slices on the tensor
 * cores, same accuracy class as t_energy's TE_OZAKI); others give
 * TE_EUNSUPPORTED.  e_out (nullable): device, one double, overwritten.
 * e_triples (nullable, not both null): device [nocc (nocc+1)(nocc+2)/6 -
 * nocc] doubles, the per-triple shares in t_energy_triples' canonical order,
 * (1/3) sum over each triple's distinct orderings.  Costs about three
 * times t_energy's contractions, on the adjoint's GEMMs (DFMA in TE_FP64,
 * tcgen05 in TE_OZAKI); deterministic.  Workspace (what te_reserve with TE_RESERVE_FRAG
 * allocates): about 8 nocc nvir^3 bytes for the transformed ovvv, plus three
 * exact-slice operand sets of the same size each in TE_OZAKI (about 34 GB at
 * nocc=32, nvir=320); TE_ENOMEM before any launch when the device cannot
 * hold it. */
te_status t_energy_frag(te_handle h, const te_cluster* c, const double* cf, te_precision p,
                        double* e_out, double* e_triples, te_stream_t s);

/* ---------------------------------------------------------------------------
 * E(T) with the (ov|vv) block formed on the fly from density-fitting factors
 * (the integrals of the clusters are density-fitted, (pq|rs) = sum_P B[P,p,q]
 * B[P,r,s]; by the supplement's remark on the divisibility of the (T)
 * contraction, the energy never needs a whole six-index tensor, and with
 * these factors it needs no float64 ovvv either)
 *
 *   ovvv[i,a,b,d] = sum_P Bov[P,i,a] Bvv[P,b,d]
 *
 * The slabs ovvv[i] are formed in groups on the tensor cores (Bov and Bvv cut
 * into five 7-bit BF16 slices with one power-of-two scale each, fifteen slice
 * products with exact level-0/1 sums over K blocks of at most 1024, float64
 * across blocks: each entry within naux 2^(ea + eb - 34) of the float64
 * product, where 2^ea > max |Bov| and 2^eb > max |Bvv|) and written straight
 * into the contraction's operand form.  The
 * exact-slice modes need max |ovvv| before slicing, so the slabs are formed
 * twice (once for the maximum, once for the slices); the two passes give the
 * same bits.  No float64 ovvv is allocated or read.
 * ------------------------------------------------------------------------- */
typedef struct {
  int64_t naux;
  const double *Bov;  /* device [naux][nocc][nvir], float64, C-contiguous */
  const double *Bvv;  /* device [naux][nvir][nvir], float64, C-contiguous */
} te_df;

/* E(T) of one cluster whose ovvv comes from df (c->ovvv is not read and may
 * be NULL; the other arrays as for t_energy).  p: a tensor-core mode
 * (TE_OZAKI, TE_BF16X3, TE_TF32X3, TE_TF32); TE_FP64 gives TE_EUNSUPPORTED.
 * The result equals t_energy's with ovvv = the float64 DF product, within the
 * mode's accuracy class.  Input values (including Bov and Bvv) are checked on
 * the device and reported by te_sync.  Workspace: the contraction operands of
 * t_energy (about 8 nocc nvir^3 bytes of ovvv slices in TE_OZAKI) plus the
 * larger of the G pool and the formation's scratch (five slices of Bov and
 * Bvv, 10 naux (nocc nvir + nvir^2) bytes, and a staging block of at most
 * 2 GiB of float64 slabs); te_df_workspace_bytes gives it.  Asynchronous,
 * deterministic. */
te_status t_energy_df(te_handle h, const te_cluster* c, const te_df* df, te_precision p, double* e_out,
                      te_stream_t s);

/* The per-triple shares of [t_begin, t_end) (t_energy_triples' canonical
 * order) with ovvv from df; as t_energy_df otherwise. */
te_status t_energy_df_triples(te_handle h, const te_cluster* c, const te_df* df, te_precision p,
                              int64_t t_begin, int64_t t_end, double* e_triples, te_stream_t s);

/* Device bytes of workspace t_energy_df needs for this cluster, factors and
 * mode (only the sizes are read). */
te_status te_df_workspace_bytes(te_handle h, const te_cluster* c, const te_df* df, te_precision p,
                                size_t* bytes);

/* ---------------------------------------------------------------------------
 * The MP2 step before (T): amplitudes, one-body density, BNO populations
 * (supplement section on bath-natural-orbital construction)
 *
 *   (ia|jb)  = sum_P Bov[P,i,a] Bov[P,j,b]
 *   t_ij^ab  = -(ia|jb) / D_ij^ab,   D_ij^ab = e_a + e_b - e_i - e_j
 *   gamma_ab = 2 sum_ij sum_c t_ij^ac (2 t_ij^bc - t_ij^cb)
 *   gamma_ij = 2 delta_ij - 2 sum_k sum_ab t_ik^ab (2 t_jk^ab - t_jk^ba)
 *
 * and the BNO populations, the eigenvalues of gamma_oo and gamma_vv (the
 * occupied-virtual block of the MP2 1-RDM is zero).  The t2 produced here is
 * the t2 input of t_energy.
 * ------------------------------------------------------------------------- */
typedef struct {
  int64_t nocc, nvir, naux;
  const double *eps_o, *eps_v;  /* device [o], [v]; max(eps_o) < min(eps_v) */
  const double *Bov;            /* device [naux][o][v]: the occupied-virtual block of the DF factor */
} te_mp2_cluster;

/* Outputs (device float64, caller-allocated, overwritten; a null member is
 * not returned, but at least one must be set). */
typedef struct {
  double *t2;        /* [o][o][v][v]  t2[i,j,a,b] = t_ij^ab */
  double *gamma_oo;  /* [o][o] */
  double *gamma_vv;  /* [v][v] */
  double *pop_o;     /* [o]  eigenvalues of gamma_oo, ascending */
  double *pop_v;     /* [v]  eigenvalues of gamma_vv, ascending */
} te_mp2_out;

/* The MP2 step for n clusters (HOST arrays cs and outs of n entries each).
 * p = TE_FP64 (every contraction on the DFMA units) or TE_OZAKI (the three
 * (ia|jb) contraction in exact BF16 slices on the tensor cores, the density
 * contractions in float64; outputs within about 2e-8 of their largest entry,
 * so populations far below the largest are better taken from TE_FP64).  The
 * eigenvalues come from a float64 Jacobi solver in
 * either mode (nvir <= 4094).  Input values are checked on the device
 * (finite, max eps_o < min eps_v; te_sync reports TE_EINVAL naming the
 * array and the cluster).  Workspace: about 8 (4 o^2 v^2) bytes for the
 * largest member in TE_FP64, plus its exact-slice copies and split-K partial
 * tiles in TE_OZAKI.  Deterministic. */
te_status t_mp2_bno_batched(te_handle h, const te_mp2_cluster* cs, const te_mp2_out* outs, int64_t n,
                            te_precision p, te_stream_t s);

/* Wait for the work of handle h on stream s and report a device-side
 * watchdog expiry (TE_ETIMEOUT) or an asynchronous CUDA error (TE_ECUDA). */
te_status te_sync(te_handle h, te_stream_t s);

/* Device bytes the handle's workspace would need for this cluster and mode
 * (before any call), so a caller can check memory up front. */
te_status te_workspace_bytes(te_handle h, const te_cluster* c, te_precision p,
                             size_t* bytes);

/* Allocate the handle's workspace (and its table of occupied triples) for a
 * cluster of c->nocc, c->nvir in mode p now, instead of on the first call, so
 * that later calls of that size or smaller allocate nothing.  Only nocc and
 * nvir are read; the array pointers may be NULL.  what: any non-empty
 * combination of TE_RESERVE_ENERGY (t_energy, t_energy_triples,
 * t_energy_batched), TE_RESERVE_VJP (t_energy_vjp) and TE_RESERVE_FRAG
 * (t_energy_frag).  TE_ENOMEM if the device cannot hold it (the handle keeps
 * what it had); TE_EUNSUPPORTED inside a stream capture.  Synchronises the
 * device when a smaller workspace is replaced. */
#define TE_RESERVE_ENERGY 1
#define TE_RESERVE_VJP 2
#define TE_RESERVE_FRAG 4
te_status te_reserve(te_handle h, const te_cluster* c, te_precision p, int what);

/* Launch accounting of one handle.  Kernel launches are always counted; with
 * profiling on, CUDA events are recorded on the caller's stream around every
 * contraction (GEMM) and energy-epilogue launch, and te_profile_read returns
 * the summed device durations.  Not part of the paper: measurement support. */
typedef struct {
  int64_t launches;         /* kernels launched by the library */
  int64_t gemm_launches;    /* W~ contraction launches */
  double gemm_ms;           /* their summed device time (profiling on) */
  int64_t energy_launches;  /* energy-epilogue launches */
  double energy_ms;         /* their summed device time (profiling on) */
  double gemm_flops;        /* tensor/DFMA flops issued by the timed GEMM launches (incl. padding) */
} te_profile;

te_status te_profile_enable(te_handle h, int on);
/* Synchronises the device, fills *out, and zeroes the counters if reset != 0. */
te_status te_profile_read(te_handle h, te_profile* out, int reset);

/* E(T) in float64 (the TE_FP64 arithmetic) without allocating any device
 * memory.  The paper has no counterpart: this exists for callers that cannot
 * let a library allocate - a host program that hands the whole GPU to its own
 * memory pool and treats any other allocation as a budget violation, or one
 * that cannot afford cudaMalloc's implicit device-wide synchronisation in the
 * middle of its work.  No handle is used; the current CUDA device is.
 *
 * All scratch (prepared operand copies, G blocks, partial sums, the triple
 * table) lives in one 64 MiB array compiled into the library; every GPU that
 * loads the library holds it until the process exits.  A cluster needs about
 * 8 (2 o^2 v^2 + o^3 v + 3 v^3) bytes plus small tables (nocc = 8, nvir = 80
 * fits; nocc = 16, nvir = 120 does not); larger clusters are rejected with
 * TE_EINVAL, and the message names the bytes needed, before any device
 * memory is touched.  The call allocates nothing: no cudaMalloc, cudaFree or
 * other allocating routine.
 *
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress, which allocates nothing), so the address stays
 * right after a device reset reloads the library image.  Unlike t_energy it
 * reads eps_o/eps_v back to the host to check max(eps_o) < min(eps_v) (it
 * has no handle whose error word could carry the result), which
 * synchronises stream s.
 *
 * Every call shares the one array and it keeps the last call's contents;
 * each call writes every scratch byte before reading it.  Calls whose work
 * overlaps on the GPU (other streams, other host threads) race on the array
 * and give wrong results: order them.
 *
 * c: cluster (device float64 arrays as above); e_out: device pointer to one
 * double, overwritten with E(T); s: stream (0 = legacy default stream). */
te_status t_energy_fp64_noalloc(const te_cluster* c, double* e_out, te_stream_t s);

/* Most device bytes of workspace the handle may hold (0 = no limit, the
 * default).  A call or te_reserve that would need more fails with TE_ENOMEM
 * before any launch, as it would if the device had no room: a caller can
 * give the library a memory budget (and test its handling of allocation
 * failures).  TE_EINVAL if the handle already holds more than `bytes`.
 * Not part of the paper. */
te_status te_set_workspace_limit(te_handle h, size_t bytes);

/* Message for the last non-OK status returned on the calling host thread. */
const char* te_last_error(void);

/* Test hook for the device watchdog: limit (ns) for every bounded wait of
 * later launches on this handle; 0 restores the default (4 s). */
te_status te_set_wait_limit_ns(te_handle h, uint64_t ns);

/* Slice width of TE_OZAKI for later calls on this handle.  bits = 0
 * (default): 7-bit slices (four slices, ten slice products) when the K axis
 * K = 2 (nvir + nocc) <= 1024, else 6-bit slices (five slices, fifteen
 * products; K <= 4096).  bits = 7 or 6 forces one width (7 with K > 1024
 * then fails with TE_EUNSUPPORTED).  6-bit slicing carries 30 bits of each
 * operand instead of 28 and keeps one more level of slice products: about
 * ten times more accurate, about 1.5 times the tensor work.  Sums of the
 * level-0 and level-1 products are exact in either width: K products of at
 * most 2^(2 bits) units stay below 2^24. */
te_status te_set_ozaki_bits(te_handle h, int bits);

/* Logging: with the environment variable TE_LOG set (and not "0") when a
 * handle is created, the handle prints its tile plans, workspace sizes and
 * autotune decisions to stderr. */

/* Self-test of the device watchdog.  Launches on s one single-thread kernel
 * whose bounded wait is on a shared-memory mbarrier that nothing ever
 * arrives on; after limit_ns (1 ms .. 10 s, else TE_EINVAL) the wait gives
 * up, the kernel sets the handle's error word (ERR_WAIT_TIMEOUT) and returns,
 * so the context stays usable.  The following te_sync must then return
 * TE_ETIMEOUT (and clear the word).  Exercises the same wait routine and
 * error path as the tensor-core pipelines without faulting or hanging. */
te_status te_watchdog_selftest(te_handle h, uint64_t limit_ns, te_stream_t s);

#ifdef __cplusplus
}
#endif
#endif /* TENERGY_H */
