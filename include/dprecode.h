/*
 * dprecode.h -- C ABI of the GB300 (sm_103a) library for feedforward
 * decentralized precoding in the massive MU-MIMO downlink
 * (Li, Jeon, Cavallaro, Studer, arXiv:1804.10987).
 *
 * Problem (Sec. II-A, Sec. III-A): for every OFDM subcarrier n a base station
 * with B antennas serves U single-antenna users over the U x B channel H_n,
 * constant over K OFDM symbols.  The antennas are split into C clusters of
 * B_c contiguous antennas, H = [H_1, ..., H_C].  Given symbol vectors
 * s[k] in C^U the library computes the precoded vectors x[k] = [x_1; ...; x_C]
 * in C^B:
 *
 *   DP_WF   centralized Wiener filter, computed the partially decentralized way
 *           (PD-WF, Sec. III-B): G_c = H_c H_c^H, G = sum_c G_c,
 *           A = G + kappa I with kappa = U N0 / rho^2 (Thm. 1),
 *           scale = 1/beta = rho / sqrt(Es tr(A^{-1} G A^{-1})) (Thm. 1,
 *           Lemma 1), z[k] = A^{-1} s[k], x_c[k] = scale H_c^H z[k].
 *   DP_ZF   zero forcing: the same with kappa = 0 (needs B >= U).
 *   DP_FDWF fully decentralized WF (Sec. III-D): every cluster runs its own WF
 *           on (H_c, rho_c^2 = rho^2 / C) with kappa_c = tau U N0 / rho_c^2
 *           (Eq. (16)): x_c[k] = scale_c H_c^H (G_c + kappa_c I)^{-1} s[k].
 *
 * Memory layouts (row-major; complex = interleaved float pair re, im, i.e.
 * the paper's single-precision complex type; every array pointer is
 * caller-owned DEVICE memory unless a parameter says "host"):
 *   H     [n_sc][B][U]  complex  the U x B channel stored column-major, user
 *                                index fastest; cluster c is the contiguous
 *                                antenna block [off_c, off_c + B_c)
 *   S     [n_sc][K][U]  complex  symbol vectors
 *   X     [n_sc][K][B]  complex  precoded vectors
 *   G     [n_sc][U][U]  complex  summed Gram (full Hermitian matrix)
 *   Gloc  [C][n_sc][U][U]        per-cluster Grams
 *   Z     WF/ZF [n_sc][K][U], FD [n_sc][C][K][U]   z = A^{-1} s (unscaled)
 *   scale WF/ZF [n_sc],       FD [n_sc][C]         float, scale = 1 / beta
 * All device pointers must be 16-byte aligned (cudaMalloc / torch allocations
 * are).
 *
 * Execution: every compute call is asynchronous on the plan's stream and
 * returns after enqueueing.  Argument errors are detected on the host and
 * returned synchronously (nothing is enqueued).  Numerical failures of one
 * subcarrier (a non-positive pivot, i.e. A not positive definite, or a
 * non-finite input) never trap: the outputs of that subcarrier are zeroed and
 * its entry of the plan's device status array is set; dp_status_get() reads
 * it.  There is no CPU fallback: without a CUDA device every compute call
 * returns DP_ERR_CUDA.
 */
#ifndef DPRECODE_H
#define DPRECODE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DP_OK = 0,
  DP_ERR_INVALID_ARG = 1,  /* NULL pointer, size out of range, bad enum */
  DP_ERR_PARTITION = 2,    /* cluster sizes < 1 or not summing to B */
  DP_ERR_UNSUPPORTED = 3,  /* valid but not implemented (e.g. ZF with B < U) */
  DP_ERR_OOM = 4,          /* device allocation failed */
  DP_ERR_CUDA = 5,         /* a CUDA runtime call failed / no device */
  DP_ERR_NOT_PD = 6,       /* per subcarrier: A not positive definite */
  DP_ERR_NONFINITE = 7,    /* per subcarrier: non-finite H or s */
  DP_ERR_TIMEOUT = 8       /* a bounded on-device wait gave up */
} dp_status;

/* DP_ZF: kappa = 0.  DP_WF: Thm. 1, computed as PD-WF through the summed
 * cluster Grams (Sec. III-B).  DP_FDWF: Sec. III-D, Eq. (16).  DP_MRT:
 * maximum ratio transmission, the fully distributed baseline the paper
 * compares against (Sec. I, Sec. III-E): x = scale H^H s with scale = rho /
 * sqrt(Es tr(G)) -- no inverse; dp_solve returns Z = S. */
typedef enum { DP_ZF = 0, DP_WF = 1, DP_FDWF = 2, DP_MRT = 3 } dp_mode;

/* Arithmetic of the path (Sec. III-B).  DP_FP32: every step in FP32 on the
 * SIMT cores.  DP_BF16 / DP_FP16: the Gram contraction G_c = H_c H_c^H on the
 * tensor cores (tcgen05) with BF16 / FP16 inputs and FP32 accumulation; the
 * solve in FP32; the apply x_c = H_c^H z on the tensor cores as a split-FP16
 * product (H = H_hi + 2^-11 H_lo, z = z_hi + z_lo, three FP16 products with
 * FP32 accumulation, about 22 significant bits).  Any U <= 64. */
typedef enum { DP_FP32 = 0, DP_BF16 = 1, DP_FP16 = 2 } dp_precision;

/* Stream handle; identical to cudaStream_t.  NULL = the legacy default
 * stream. */
typedef struct CUstream_st *dp_stream_t;

typedef struct {
  int U;                     /* users, 1 <= U <= 64 */
  int B;                     /* antennas, U <= B for ZF, B <= 4096 */
  int C;                     /* clusters, 1 <= C <= B */
  const int *cluster_sizes;  /* host array of C sizes B_c >= 1 summing to B
                                (contiguous antenna blocks in order), or NULL
                                for C equal clusters (needs B % C == 0).
                                Copied by dp_plan_create. */
  int n_sc;                  /* subcarriers, >= 0 */
  int K;                     /* OFDM symbols per subcarrier, 0 <= K <= 64 */
  dp_mode mode;
  dp_precision prec;
  float rho2;                /* total transmit power rho^2 > 0 */
  float N0;                  /* noise variance per entry >= 0 (WF, FD) */
  float Es;                  /* symbol energy E|s_u|^2 > 0 (1 for normalized QAM) */
  float tau;                 /* FD-WF tau_c >= 0 (Eq. (16)); ignored otherwise */
  int refine;                /* BF16/FP16 only (ignored for DP_FP32 and MRT): one
                                step of iterative refinement of z against the
                                reduced-precision Gram -- the residual
                                r = s - (H H^H + kappa I) z from the exact FP32 H
                                with FP32 accumulation, z += (G_lp + kappa I)^{-1} r,
                                then the apply again; the precoding factor keeps
                                the low-precision inverse's value.
                                0 (default): automatic -- a system with
                                eps ||G||_F ||A^{-1}||_F / U >= 2e-3, eps the 16-bit
                                type's unit roundoff (2^-8 BF16, 2^-11 FP16), i.e.
                                whose 16-bit Gram could move the output by about
                                5e-4 or more (ZF with few antennas per user,
                                strongly correlated channels), is escalated: its
                                Gram is recomputed in FP32 and solved again, which
                                also corrects the precoding factor (refining z
                                alone leaves the factor's error, which comes from
                                the low-precision inverse);
                                1: the refinement step for every subcarrier;
                                -1: neither */
  const float *cluster_power; /* FD-WF only (NULL otherwise): host array of C
                                 weights w_c > 0 allocating the transmit power
                                 per cluster, rho_c^2 = rho^2 w_c / sum_c' w_c'
                                 (Sec. III-D: sum_c rho_c^2 = rho^2; the paper's
                                 choice rho_c^2 = rho^2 / C is w_c = 1, also what
                                 NULL means).  Each cluster's regularizer follows
                                 Eq. (16), kappa_c = tau U N0 / rho_c^2, and its
                                 factor sqrt(rho_c^2 / (Es t_c)).  Copied by
                                 dp_plan_create; DP_ERR_INVALID_ARG for another
                                 mode or a weight that is not a positive finite
                                 number. */
} dp_plan_desc;

typedef struct dp_plan *dp_plan_t;

/* Validate the description, copy it, and allocate the plan's workspace (the
 * cluster offsets and a device status array [n_sc]) on the current device.
 * stream: where every call of this plan enqueues.  On error *out is NULL. */
dp_status dp_plan_create(const dp_plan_desc *desc, dp_stream_t stream, dp_plan_t *out);
/* Free the plan and its workspace (synchronizes the plan's stream). */
dp_status dp_plan_destroy(dp_plan_t plan);
/* Change the stream later calls enqueue on. */
dp_status dp_plan_set_stream(dp_plan_t plan, dp_stream_t stream);

/* Step a1 (Sec. III-B, local Gram of every cluster):
 * Gloc[c][n] = H_c H_c^H for all clusters c and subcarriers n. */
dp_status dp_gram_local(dp_plan_t plan, const void *H, void *Gloc);

/* Step a2 (Sec. III-B, feedforward adder tree; Fig. 1(a)):
 * G[n] = sum_c Gloc[c][n], summed in cluster order. */
dp_status dp_gram_reduce(dp_plan_t plan, const void *Gloc, void *G);

/* Steps a3-a5 (Thm. 1, Lemma 1, Eq. (14); Sec. III-B whitening node;
 * Sec. III-D for FD-WF): regularize, factor, precoding factor, whitening.
 * WF/ZF: input G [n_sc][U][U]; A = G + kappa I; Z[n][k] = A^{-1} s[k];
 *        scale[n] = rho / sqrt(Es tr(A^{-1} G A^{-1})).
 * FD:    input Gloc [C][n_sc][U][U]; per cluster A_c = G_c + kappa_c I;
 *        Z[n][c][k] = A_c^{-1} s[k]; scale[n][c] = rho_c / sqrt(Es t_c).
 * For FD clusters with B_c < U the U x U system equals the paper's
 * B_c x B_c form by the push-through identity when kappa_c > 0; with
 * kappa_c = 0 such a cluster returns DP_ERR_UNSUPPORTED. */
dp_status dp_solve(dp_plan_t plan, const void *G_or_Gloc, const void *S, void *Z, float *scale);

/* Step a6 (Sec. III-B local precoding, with the normalization fused):
 * X[n][k][b] = scale * sum_u conj(H[n][b][u]) Z[n][k][u] over each cluster's
 * antennas, with the cluster's own Z and scale in FD mode. */
dp_status dp_precode_apply(dp_plan_t plan, const void *H, const void *Z, const float *scale,
                           void *X);

/* Steps a1-a6 fused: X from H and S.  Reads H once from HBM for every size
 * whose per-system antenna block fits in shared memory; the plan's
 * precision selects the Gram arithmetic. */
dp_status dp_precode(dp_plan_t plan, const void *H, const void *S, void *X);

/* dp_precode for arrays in HOST memory (the slot arrives from and leaves to
 * host memory, Sec. IV-B's end-to-end setting).  H [n_sc][B][U], S
 * [n_sc][K][U] and X [n_sc][K][B] are host pointers, with the dp_precode
 * layouts; page-locked memory (cudaHostAlloc / cudaHostRegister) lets the
 * copies overlap, pageable memory works without overlap.  The subcarriers
 * go in chunks of chunk_sc (<= 0: n_sc / 8 rounded up, at least 1): chunk
 * i's upload of H and S, its precoding and its download of X run on three
 * streams through a 3-deep ring of device staging buffers that the plan
 * allocates on first use (3 chunks of H, S and X; freed with the plan), so
 * that uploads, kernels and downloads of consecutive chunks overlap.
 * Results and per-subcarrier status equal those of dp_precode bit for bit.
 * The call returns once everything is enqueued; it is ordered after the
 * work already on the plan's stream and completes on that stream
 * (synchronize it, or call dp_status_get, before reading X).  The host
 * arrays must stay valid until then.  DP_ERR_OOM if the staging buffers
 * cannot be allocated. */
dp_status dp_precode_host(dp_plan_t plan, const void *H, const void *S, void *X, int chunk_sc);

/* Failure injection for tests of the timeout path (Sec. IV-B's pipeline has
 * no counterpart; this checks the library's own bounded waits).  While
 * microseconds > 0, every later dp_precode of this plan that runs the
 * warp-specialized tensor-core kernel (BF16/FP16, users padded to 8 or 16,
 * 1 <= K <= 16, U even) makes that kernel's MMA-issuing thread first wait,
 * for that long, on a flag that nothing sets.  The wait then runs out as any
 * bounded on-device wait does: the kernel's other roles stop, its copies and
 * MMAs in flight land, its TMEM is freed, and every subcarrier of the call
 * ends with DP_ERR_TIMEOUT and zeroed outputs.  0 turns it off; other plans
 * and other kernels ignore it.  DP_ERR_INVALID_ARG outside [0, 1e6]. */
dp_status dp_debug_stall(dp_plan_t plan, int microseconds);

/* Wait for the plan's stream and copy the per-subcarrier status of the last
 * call that wrote it into host_status[n_sc] (host memory; may be NULL).
 * Returns the first non-DP_OK entry (DP_OK if all succeeded). */
dp_status dp_status_get(dp_plan_t plan, int *host_status);

/* ---- Batched uneven precoding ---------------------------------------------
 * The paper aggregates the N_sc subcarriers x K symbols of a slot into one
 * batch to fill the GPU (Sec. IV-B); a batch here goes further and runs n
 * independent instances of uneven size (each its own dp_plan_desc: users,
 * antennas, clusters, subcarriers, mode, precision) in persistent launches.
 * Instances are bucketed by kernel family and padded user count: the
 * tensor-core family (prec BF16/FP16), the FP32 family with the antenna
 * block resident in shared memory, the B_c x B_c family (FD-WF clusters with
 * B_c < U), and a streaming remainder.  Each bucket is one persistent launch whose CTAs pull
 * work items from an atomic queue, largest first; the bucket launches are
 * captured once into a CUDA graph (on a non-NULL stream) and replayed on
 * every call.  Per-instance outputs and status follow the single-plan
 * conventions.
 *
 * dp_batch_create: validate and copy the n descriptions (as dp_plan_create
 *   does, same error codes), build the work lists and allocate the batch's
 *   workspace on the current device.  stream: where the batch enqueues.
 * dp_batch_precode: H[i], S[i], X[i] are host arrays of n device pointers to
 *   instance i's H [n_sc][B][U], S [n_sc][K][U] and X [n_sc][K][B] (layouts
 *   and alignment as above).  Asynchronous; the pointer table is copied
 *   before the call returns.
 * dp_batch_tune: autotuner.  Runs every bucket at each feasible number of
 *   CTAs per SM (trials timed runs each, after one warm-up, each run
 *   starting with a cold L2: a temporary buffer twice the L2 size is written
 *   first) on the given arrays, keeps the largest count within 2 % of the
 *   fastest, and rebuilds the graph.  Synchronous.
 * dp_batch_status_get: waits, then writes the per-subcarrier status of every
 *   instance, instance after instance, into host_status (sum of n_sc entries;
 *   NULL allowed) and returns the first failure.
 * dp_batch_describe: a JSON string (owned by the batch) with the buckets,
 *   their work items, systems, algorithmic bytes (every system's H and X
 *   rows and the symbols it reads, once each), the chosen CTAs per SM and
 *   the kernel launches each bucket makes per call.
 * dp_batch_set_timing: mode 1 records a CUDA event before every bucket launch
 *   and one after the last, inside the graph; mode 2 does the same with
 *   eager launches (no graph); 0 turns it off.  Synchronizes the stream and
 *   rebuilds the graph.
 * dp_batch_bucket_ms: waits for the stream, then writes the device time of
 *   each bucket of the last call (in describe's order, n entries at most)
 *   into ms (host).  DP_ERR_UNSUPPORTED when timing is off. */
typedef struct dp_batch *dp_batch_t;
dp_status dp_batch_create(const dp_plan_desc *descs, int n, dp_stream_t stream, dp_batch_t *out);
dp_status dp_batch_destroy(dp_batch_t b);
dp_status dp_batch_precode(dp_batch_t b, const void *const *H, const void *const *S,
                           void *const *X);
dp_status dp_batch_tune(dp_batch_t b, const void *const *H, const void *const *S, void *const *X,
                        int trials);
dp_status dp_batch_status_get(dp_batch_t b, int *host_status);
const char *dp_batch_describe(dp_batch_t b);
dp_status dp_batch_set_timing(dp_batch_t b, int mode);
dp_status dp_batch_bucket_ms(dp_batch_t b, float *ms, int n);

/* ---- Continuous-batching server -------------------------------------------
 * Serving form of the precoder: a cell is one channel (its dp_plan_desc with
 * n_sc = subcarriers of one slot, and a device-resident H [n_sc][B][U] owned
 * by the caller, which may point the cell at a new estimate at any time);
 * a request precodes one slot of a cell from device symbols S [n_sc][K][U]
 * into an output X [n_sc][K][B] that the server places in its device arena.
 * A worker thread admits pending requests in arrival order whenever fewer
 * than max_inflight are on the GPU and the arena has room for the request's
 * output and status (admission by free device memory), launches them
 * round-robin over the server's streams (requests overlap on the GPU, those
 * of one cell included; cells in the streaming FP32 form, whose workspace is
 * per cell, keep their slots in order on one stream) and retires them when
 * they complete, recording the latency from submission to the observed
 * completion.  Every request runs the same kernels as dp_precode
 * with the cell's precision (or, with cache_solve, the cached-solve kernels),
 * so its result does not depend on the mix.
 * The paper has no serving layer; this packages its per-slot precoder
 * (Sec. IV) for an arrival process of slots. */
typedef struct {
  int device;          /* CUDA device the server runs on */
  int streams;         /* CUDA streams the requests are spread over, 1..64 */
  int max_inflight;    /* requests on the GPU at once, 1..1024 */
  size_t arena_bytes;  /* device memory for request outputs, status and, with
                          cache_solve, each request's z and scale */
  int auto_release;    /* 1: a request's output is freed as soon as it completes;
                          0: kept until dp_server_release (other values: invalid) */
  int cache_solve;     /* 1: per cell, everything that depends on the channel
                          alone -- G, T = (G + kappa I)^{-1} and the scale
                          (Thm. 1, Lemma 1) -- is computed in FP32 on the first
                          request after each dp_server_set_channel and kept;
                          every request then only whitens (z = T s) and applies
                          (FP32).  FD-WF clusters with B_c < U stay per request.
                          0: every request runs the dp_precode kernels (other
                          values: invalid) */
} dp_server_config;

typedef struct {
  long long completed, failed, subcarriers;
  double p50_ms, p99_ms, mean_ms, max_ms;  /* submission -> completion latency */
  double wall_s;                           /* first submission -> last completion */
  int inflight_peak;
  long long arena_high_water;              /* bytes */
} dp_server_stats_t;

typedef struct dp_server *dp_server_t;
/* Create the server (allocates its arena and streams, starts its worker). */
dp_status dp_server_create(const dp_server_config *cfg, dp_server_t *out);
/* Stop the worker after the submitted requests complete; free everything. */
dp_status dp_server_destroy(dp_server_t s);
/* Register a cell (validated like dp_plan_create; K >= 1, n_sc >= 1); H is a
 * 16-byte aligned device array that must stay valid while the cell uses it.
 * DP_ERR_OOM if one request of the cell could never fit the arena. */
dp_status dp_server_add_cell(dp_server_t s, const dp_plan_desc *desc, const void *H, int *cell_id);
/* Point the cell at another device channel array (requests submitted from
 * now on use it). */
dp_status dp_server_set_channel(dp_server_t s, int cell, const void *H);
/* Submit one slot: S is a device array; returns at once with the id. */
dp_status dp_server_submit(dp_server_t s, int cell, const void *S, unsigned long long *req_id);
/* Block until every submitted request has completed. */
dp_status dp_server_drain(dp_server_t s);
/* A completed request's output (device pointer into the arena, valid until
 * released) and its worst per-subcarrier status. */
dp_status dp_server_result(dp_server_t s, unsigned long long req_id, void **X, int *status);
/* Copy a completed request's output to dst (device, or host if to_host). */
dp_status dp_server_copy_result(dp_server_t s, unsigned long long req_id, void *dst, int to_host);
/* Return a completed request's output buffer to the arena. */
dp_status dp_server_release(dp_server_t s, unsigned long long req_id);
/* Open-loop load generator: submit request i for cells[i] with symbols S[i]
 * at arrival_s[i] seconds after the call (busy-waiting on the host clock;
 * if H_switch is non-NULL and H_switch[i] is non-NULL, the cell is pointed at
 * that channel first), then drain. */
dp_status dp_server_replay(dp_server_t s, int n, const int *cells, const void *const *S,
                           const double *arrival_s, const void *const *H_switch);
dp_status dp_server_stats(dp_server_t s, dp_server_stats_t *out);
dp_status dp_server_reset_stats(dp_server_t s);

/* Allocation-free precoding (the paper has no counterpart: this is a
 * deployment variant of dp_precode).  For callers that cannot call
 * cudaMalloc: a baseband runtime whose device memory is carved up once at
 * start-up, a real-time slot loop where an allocation's latency or implicit
 * synchronization would break the slot deadline, or code that runs while
 * the caller's allocator is locked.  It runs the streaming form of
 * dp_precode (Gram with the cluster sum, solve, apply; FP32; FD-WF clusters
 * with B_c < U and B_c <= 32 in the B_c x B_c form of Sec. III-D, as
 * dp_precode does) with all of its workspace in one static device array of
 * DP_NOALLOC_SCRATCH_BYTES that every GPU loading the library reserves until
 * the process exits.  No plan is
 * needed and nothing is allocated: the caller passes the description (as for
 * dp_plan_create; prec must be DP_FP32, refine 0), the stream, and the device
 * arrays H [n_sc][B][U], S [n_sc][K][U], X [n_sc][K][B] in the layouts above
 * (per-cluster power, cluster_power != NULL, returns DP_ERR_UNSUPPORTED).
 * The workspace needs, rounding each part up to 256 bytes,
 *   4 (C + 1) + 4 n_sys + 8 n_sys U^2 + 8 n_sys K U + 4 n_sys  bytes,
 * n_sys = n_sc (WF/ZF) or n_sc C (FD-WF); a larger problem returns
 * DP_ERR_UNSUPPORTED before anything is enqueued.
 * The first call on a device looks up the array's device address with that
 * device current (cudaGetSymbolAddress) and keeps it for the life of the
 * process; make that first call before any stream capture, and do not use
 * the entry point after a cudaDeviceReset of that device (the kept address
 * belongs to the old context).  The cluster offsets reach the device as
 * kernel parameters: the call copies nothing from host memory.  All calls
 * on a device share the array and each call overwrites what it reads, so
 * calls whose work overlaps on the GPU race: serialize them (one stream, or
 * events).  host_status: NULL to return after
 * enqueueing; otherwise the call waits for the stream and writes the
 * per-subcarrier status codes into host_status[n_sc] (host memory) and
 * returns the first failure, as dp_status_get does. */
#define DP_NOALLOC_SCRATCH_BYTES (8u << 20)
dp_status dp_precode_noalloc(const dp_plan_desc *desc, dp_stream_t stream, const void *H,
                             const void *S, void *X, int *host_status);

/* Static description of a status code. */
const char *dp_status_string(dp_status s);

/* Library version string. */
const char *dp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DPRECODE_H */
