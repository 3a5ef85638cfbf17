/*
 * kpp.h -- C ABI of libkpp, GB300 (sm_103a) k-means++ D^2 seeding.
 *
 * The method is k-means++ seeding as parallelised in Heydarpour Shahrezaei &
 * Tavoli, "Parallelization of Kmeans++ using CUDA" (arXiv:1908.02136):
 *   - Algorithm 1 (serial) / Algorithm 2 (parallel): the first seed is a
 *     uniformly random point; every point's nearest squared distance D^2
 *     starts at infinity; after each new seed every point's distance to it is
 *     taken and D^2 keeps the minimum; the next seed is drawn with probability
 *     D^2_i / sum_w D^2_w.
 *   - Section II: chosen seeds are kept as an index array and their
 *     coordinates are read from the point array by index; the sum of D^2 is
 *     taken in double precision (the Thrust reduction).
 * Conventions this library fixes where the paper is silent:
 *   - draws: u_m = Philox4x64-10(key = {seed, stream_id}, counter = {m,0,0,0}),
 *     word 0 mapped to [0,1) as (w0 >> 11) * 2^-53 (Salmon et al., SC'11);
 *   - first seed: i_0 = min(floor(u_0 * N), N - 1);
 *   - seed m >= 1: inverse CDF in index order, t = u_m * T with T = sum D^2 in
 *     FP64; i_m is the first index whose FP64 prefix sum exceeds t (strictly),
 *     so points with D^2 = 0 are never drawn; if rounding leaves none, the
 *     last point with D^2 > 0 is taken.  Prefix sums are hierarchical
 *     (per-CTA FP64 block sums, then a rescan of the winning block only).
 *   - distances are squared Euclidean in the difference form
 *     sum_j (x_ij - c_j)^2, accumulated in FP32; D^2 is stored in FP32.
 *   - K distance passes and K-1 draws; phi = sum_i D^2_i in FP64 after the
 *     last pass.
 *   - if sum D^2 = 0 at a draw (fewer distinct points than K), seeding stops:
 *     the remaining indices are -1 and the device status becomes
 *     KPP_ERR_DEGENERATE.
 *
 * Memory and ownership: every buffer is allocated and owned by the caller.
 * Unless a parameter says "host", pointers are CUDA device pointers on the
 * current device.  Points are row-major [N x d], contiguous, and the base
 * must be 16-byte aligned.  No entry point allocates device memory; scratch
 * lives in the caller's workspace (size from kpp_workspace_size, 256-byte
 * aligned).  A workspace must not be shared by calls in flight at the same
 * time.
 *
 * Debug build: compiled with KPP_DEBUG=1, the kernels check the index of
 * every shared- and global-memory access on their hot paths before making
 * it; an index outside its buffer skips the access and records
 * KPP_ERR_BOUNDS (with a site number) in the device status word, so a
 * faulty index shows up as a status, never as a memory fault.  The release
 * build compiles the checks away.
 *
 * Asynchrony and errors: compute entry points enqueue work on `stream` and
 * return at once.  Argument errors are returned synchronously and nothing is
 * enqueued.  Errors found on the device (degenerate data, a barrier
 * timeout) are written to a status word in the workspace; kpp_read_status
 * synchronises the stream and returns it.  No exception crosses this ABI.
 */
#ifndef KPP_H
#define KPP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define KPP_API __attribute__((visibility("default")))
#else
#define KPP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *kpp_stream_t;

typedef enum {
    KPP_OK = 0,
    KPP_ERR_INVALID_ARG = 1, /* bad size, NULL or misaligned pointer, K > N ... */
    KPP_ERR_CUDA = 2,        /* a CUDA runtime call failed */
    KPP_ERR_LAUNCH = 3,      /* a launch was refused (e.g. co-residency) */
    KPP_ERR_TIMEOUT = 4,     /* a bounded device wait gave up (device status) */
    KPP_ERR_DEGENERATE = 5,  /* sum D^2 = 0 before K seeds (device status) */
    KPP_ERR_WORKSPACE = 6,   /* workspace NULL, misaligned or too small */
    KPP_ERR_UNSUPPORTED = 7, /* option combination not built */
    KPP_ERR_CAPACITY = 8,    /* k-means||: more candidates than the caller's room */
    KPP_ERR_BOUNDS = 9       /* debug build only (KPP_DEBUG): a kernel computed an index
                                outside its buffer; the access was skipped (device status) */
} kpp_status;

/* Storage type of the points; distances are always accumulated in FP32. */
typedef enum {
    KPP_F32 = 0,
    KPP_BF16 = 1,     /* bfloat16 bit patterns */
    KPP_FP8_E4M3 = 2  /* OCP E4M3 codes, value = row_scale[i] * decode(q_ij) */
} kpp_dtype;

typedef enum {
    KPP_FORM_AUTO = 0,
    KPP_FORM_STREAMED = 1,   /* one kernel per seed, captured in a CUDA graph */
    KPP_FORM_PERSISTENT = 2, /* one cooperative launch for all K passes */
    KPP_FORM_RECOMPUTE = 3,  /* for comparison only: the paper's own step (Section II),
                                every pass recomputes each point's distance to all
                                seeds chosen so far (O(N K^2 d) work) in the streamed
                                form's launches; results identical to the streamed form */
    KPP_FORM_SMALL = 4       /* one CTA of 1024 threads holds the points (as FP32, FP8 as
                                its E4M3 values plus the row scales) and D^2 in shared
                                memory for all K passes: 4 N (d + 1) bytes (+ 4 N for
                                FP8) must fit one SM's shared memory; the automatic
                                choice whenever they do */
} kpp_form;

/* Tuning knobs; a zeroed struct (or NULL) means "choose automatically". */
typedef struct {
    int32_t form;             /* kpp_form */
    int32_t lanes_per_row;    /* lanes that share one point row: 1,2,4,8,16,32 */
    int32_t ctas_per_sm;      /* resident CTAs per SM the grid is sized for */
    int32_t use_graph;        /* streamed form: 0/1 = CUDA graph, -1 = plain launches */
    uint32_t timeout_us;      /* persistent form: bound of each grid-barrier wait;
                                 0 = 2,000,000 us */
    int32_t smem_cache;       /* persistent form: -1 = no shared-memory point cache,
                                 0 = as many rows as fit, > 0 = at most this many
                                 rows per CTA */
    int32_t alternate;        /* persistent form: 0/1 = walk rows backwards on odd
                                 passes (L2 reuse), -1 = always forwards */
    int32_t l2_policy;        /* persistent form, streamed rows: 0 = evict-last,
                                 -1 = no hint, 2 = evict-first */
    int32_t min_rows_per_cta; /* persistent form: smallest row block; 0 = 2048 */
    int32_t exact_draws;      /* 1 = decide every "prefix > t" comparison of every draw
                                 in FP64 (t = u * T as the FP64 product of the draw's
                                 uniform and the pair total), the path otherwise taken
                                 only at near ties, where an FP32 estimate of the
                                 prefix lies within 2^-40 t of t; same results, slower
                                 draws; for testing that path.  0 = FP32 estimates
                                 decide away from ties (default) */
    int32_t reserved[2];
} kpp_options;

/* The launch plan kpp_seed would use for a problem (filled by kpp_describe). */
typedef struct {
    int32_t form;                /* kpp_form actually chosen */
    int32_t grid;                /* CTAs per launch */
    int32_t threads;             /* threads per CTA */
    int32_t launches;            /* kernel launches per seeding */
    int32_t lanes_per_row;       /* 0 for the generic (any d) kernel */
    int32_t d2_in_smem;          /* persistent form: D^2 held in shared memory */
    int64_t rows_per_cta;        /* contiguous row block of each CTA */
    int64_t rows_per_segment;    /* rows under one middle-level sum of the draw
                                    (one warp's contiguous share of a block) */
    int64_t cached_rows_per_cta; /* persistent form: rows kept in shared memory */
    int64_t smem_bytes;          /* dynamic shared memory per CTA */
    int64_t workspace_bytes;     /* same as kpp_workspace_size */
} kpp_plan;

/* Human-readable name of a status code (static string, never NULL). */
KPP_API const char *kpp_status_string(kpp_status status);

/* Library version as 10000*major + 100*minor + patch. */
KPP_API int32_t kpp_version(void);

/*
 * Bytes of device workspace kpp_seed needs for this problem on the current
 * device (0 if the arguments are invalid).  The size depends on N, d, dtype,
 * the options and the device's SM count, not on the data.
 */
KPP_API size_t kpp_workspace_size(int64_t N, int32_t d, int32_t K, kpp_dtype dtype,
                          const kpp_options *opts);

/*
 * Fills `plan` with the form, grid and memory layout kpp_seed would use for
 * these arguments on the current device.  Host-side only; nothing is
 * launched.  Returns KPP_OK or the error kpp_seed would return.
 */
KPP_API kpp_status kpp_describe(int64_t N, int32_t d, int32_t K, kpp_dtype dtype,
                                const kpp_options *opts, kpp_plan *plan);

/*
 * k-means++ seeding of one problem (Algorithm 1 / Algorithm 2).
 *   points        [N x d] stored values of `dtype`, 16-byte aligned
 *   row_scales    [N] FP32 per-row scales (KPP_FP8_E4M3 only, else NULL)
 *   N, d, K       1 <= K <= N < 2^31, 1 <= d <= 4096
 *   seed, stream_id  Philox key of the draws
 *   forced_prefix [n_forced] device indices that replace the first n_forced
 *                 draws (replay / teacher forcing), or NULL with n_forced = 0
 *   indices_out   [K] int64: chosen seeds in draw order
 *   d2_out        [N] FP32: nearest squared distance after the last pass
 *   phi_out       [1] FP64: sum of d2_out, or NULL
 *   workspace     >= kpp_workspace_size(...) bytes, 256-byte aligned
 * Returns KPP_OK once the work is enqueued on `stream`; device-side
 * outcomes are read with kpp_read_status.
 */
KPP_API kpp_status kpp_seed(const void *points, const float *row_scales, int64_t N, int32_t d,
                    int32_t K, kpp_dtype dtype, uint64_t seed, uint64_t stream_id,
                    const int64_t *forced_prefix, int32_t n_forced,
                    int64_t *indices_out, float *d2_out, double *phi_out,
                    void *workspace, size_t workspace_bytes, kpp_stream_t stream,
                    const kpp_options *opts);

/*
 * End-to-end seeding from HOST buffers: copies the host points (and scales)
 * into the caller's device buffers, seeds as kpp_seed, copies indices, D^2
 * and phi back to the host, and synchronises `stream`.  Pinned host memory
 * gives asynchronous copies; pageable memory works but is slower.
 *   host_points   [N x d] host stored values; dev_points: device buffer of
 *                 the same size (16-byte aligned)
 *   host_scales / dev_scales   FP8 only, else NULL
 *   host_indices [K] int64, host_d2 [N] FP32, host_phi [1] FP64 (may be NULL)
 *   dev_indices [K], dev_d2 [N], dev_phi [1] device buffers
 * Returns the device status (KPP_OK, KPP_ERR_DEGENERATE, ...) after the sync.
 */
KPP_API kpp_status kpp_seed_host(const void *host_points, const float *host_scales,
                         void *dev_points, float *dev_scales, int64_t N, int32_t d,
                         int32_t K, kpp_dtype dtype, uint64_t seed, uint64_t stream_id,
                         int64_t *host_indices, float *host_d2, double *host_phi,
                         int64_t *dev_indices, float *dev_d2, double *dev_phi,
                         void *workspace, size_t workspace_bytes, kpp_stream_t stream,
                         const kpp_options *opts);

/*
 * Synchronises `stream` and returns the device status word of the last
 * call that used `workspace`: KPP_OK, KPP_ERR_DEGENERATE or KPP_ERR_TIMEOUT
 * (KPP_ERR_CUDA if the copy itself fails).
 */
KPP_API kpp_status kpp_read_status(const void *workspace, kpp_stream_t stream);

/*
 * Precision forms (not in the paper): quantise FP32 points once, before
 * seeding, so each pass reads fewer bytes.
 *   x [N x d] FP32 device input.
 *   to = KPP_BF16: out is [N x d] uint16 BF16, round to nearest even;
 *        row_scales must be NULL.
 *   to = KPP_FP8_E4M3: out is [N x d] uint8 E4M3 codes and row_scales [N]
 *        FP32 with s_i = max_j |x_ij| / 448 (1 for an all-zero row) and
 *        q_ij = round-to-nearest-even, saturating, of the FP32 x_ij / s_i.
 * Asynchronous on `stream`.
 */
KPP_API kpp_status kpp_quantize(const float *x, int64_t N, int32_t d, kpp_dtype to, void *out,
                        float *row_scales, kpp_stream_t stream);

/*
 * Measurement utility (not part of the method; the paper has no
 * counterpart): the rate at which this GPU streams reads from a buffer, the
 * denominator a seeding pass -- a pure read stream over the points -- is
 * compared with.  Reads `bytes` of `buf` once untimed, then `reps` times in
 * one launch of one full wave of resident CTAs (16-byte loads, every thread
 * reading the same addresses in every sweep, so a CTA keeps its SM and its
 * nearby L2 slices across sweeps, as the persistent seeding form does),
 * timed with CUDA events on `stream`; *ms_out (host) receives the mean
 * milliseconds per timed sweep.  A buffer far larger than L2 gives the HBM read bandwidth; a
 * buffer well inside L2, read again and again, the L2 read bandwidth.
 *   buf    device, 16-byte aligned; bytes a multiple of 16 (>= 16)
 *   reps   >= 1
 * Blocks the calling thread (it waits for the last sweep).  Returns KPP_OK,
 * KPP_ERR_INVALID_ARG, KPP_ERR_LAUNCH or KPP_ERR_CUDA.
 */
KPP_API kpp_status kpp_measure_read(const void *buf, size_t bytes, int32_t reps,
                                    kpp_stream_t stream, float *ms_out);

/*
 * Batching form (not in the paper): many independent seedings -- of uneven
 * N, d and K, all stored as `dtype` -- in one cooperative launch.  Each
 * problem is exactly the kpp_seed problem (same draws for the same seed and
 * stream id, same results up to the blocking of the prefix sums).
 * Problems costing more than one SM's share of the batch run on a team of
 * CTAs; the others on one CTA each, longest first, from a work queue.
 * d must be one of 2, 4, 8, 16, 32, 64, 128 (KPP_ERR_UNSUPPORTED otherwise).
 */
typedef struct {
    const void *points;      /* [N x d] device, 16-byte aligned */
    const float *row_scales; /* [N] FP8 only, else NULL */
    int64_t N;
    int32_t d;
    int32_t K;
    uint64_t seed;
    uint64_t stream_id;
    int64_t *indices_out; /* [K] device */
    float *d2_out;        /* [N] device */
    double *phi_out;      /* [1] device, or NULL */
} kpp_problem;

/* Workspace bytes kpp_seed_batched needs for this HOST array of problems
 * on the current device (0 if the problems are invalid). */
KPP_API size_t kpp_batch_workspace_size(const kpp_problem *problems, int32_t n, kpp_dtype dtype,
                                        const kpp_options *opts);

/*
 * Seeds every problem of the HOST array `problems` (read during the call;
 * the device buffers it points to must stay valid until the work is done).
 * Asynchronous on `stream`.  Device outcomes: kpp_read_status(workspace)
 * gives the first non-OK status of any problem (a degenerate problem does
 * not stop the others; its indices end with -1).
 */
KPP_API kpp_status kpp_seed_batched(const kpp_problem *problems, int32_t n, kpp_dtype dtype,
                                    void *workspace, size_t workspace_bytes, kpp_stream_t stream,
                                    const kpp_options *opts);

/*
 * Autotuner (not in the paper, which fixes one kernel shape): chooses the
 * form (persistent or streamed), the lanes that share a point row (how many
 * points a warp covers per iteration), the smallest row block per CTA, the
 * CTAs per SM of the streamed grid, the persistent form's shared-memory
 * point cache, its L2 policy and traversal, by timing the candidates on the
 * caller's own data: each candidate runs min(K, passes) passes (passes = 0:
 * min(K, 32)) once untimed and twice timed with CUDA events on `stream`;
 * candidates are tried defaults first, and a later one replaces the best so
 * far only if it is more than 1 % faster.
 *   points, row_scales, N, d, K, dtype   as for kpp_seed
 *   indices_out [K], d2_out [N]          device scratch for the trial runs
 *                                        (their contents are undefined after)
 *   workspace   >= kpp_tune_workspace_size(N, d, K, dtype) bytes covers every
 *               candidate; a smaller one skips the candidates it cannot hold
 *   best_out    host: the winning options (form never KPP_FORM_AUTO)
 *   best_ms_per_pass  host, may be NULL: the winner's mean time per pass
 * Blocks the calling thread (it synchronises `stream`).  The winner is also
 * recorded per (device, dtype, d, N, K) for the rest of the process: a later
 * kpp_seed / kpp_workspace_size / kpp_describe for that shape whose options
 * leave form, lanes_per_row, ctas_per_sm, smem_cache, alternate, l2_policy
 * and min_rows_per_cta all zero (or opts NULL) uses it (keeping the caller's
 * timeout_us and use_graph) -- so size the workspace after tuning.
 * Returns KPP_OK, KPP_ERR_DEGENERATE (the data has fewer than min(K, passes)
 * distinct points; nothing is recorded), KPP_ERR_UNSUPPORTED (no candidate
 * could run in the given workspace) or kpp_seed's argument errors.
 * If the environment variable KPP_TUNE_CACHE names a file, every winner is
 * also appended to it as one text line keyed by the GPU model (name and SM
 * count), dtype, d, N and K, and a process reads that file's lines for its
 * GPU model once, at its first automatic choice on a device: later
 * processes then use the recorded winners without tuning (a later line wins
 * over an earlier one for the same shape).
 */
KPP_API size_t kpp_tune_workspace_size(int64_t N, int32_t d, int32_t K, kpp_dtype dtype);
KPP_API kpp_status kpp_tune(const void *points, const float *row_scales, int64_t N, int32_t d,
                            int32_t K, kpp_dtype dtype, int64_t *indices_out, float *d2_out,
                            void *workspace, size_t workspace_bytes, kpp_stream_t stream,
                            int32_t passes, kpp_options *best_out, float *best_ms_per_pass);
/* Forgets every shape recorded by kpp_tune in this process, and what was
 * read from a KPP_TUNE_CACHE file (which is not read again in this process;
 * the file itself is left as it is). */
KPP_API void kpp_tune_clear(void);

/*
 * One Lloyd iteration -- the clustering stage the seeds are for (Section II:
 * "the clustering part is implemented the same as the K-means algorithm"):
 * every point is assigned to its nearest centre (squared Euclidean; the
 * smallest index wins a tie), then every centre moves to the mean of its
 * points; a centre no point chose keeps its position.
 *   points      [N x d] FP32 device, d <= 128, 1 <= K <= min(N, 4096)
 *   centres     [K x d] FP32 device (e.g. the seeded points)
 *   labels_out  [N] int32: the assigned centre
 *   d2_out      [N] FP32 or NULL: squared distance to it (FP32 difference
 *               form, the seeding pass's arithmetic)
 *   centres_out [K x d] FP32: the means (may not alias `centres`)
 *   counts_out  [K] int64 or NULL: points per centre
 *   phi_out     [1] FP64 or NULL: sum of d2 (the cost of the assignment)
 *   workspace   >= kpp_lloyd_workspace_size(N, d, K) bytes, 256-byte aligned,
 *               prepared once by kpp_lloyd_prepare for these points
 * The assignment runs on the tensor cores: |c|^2 - 2 x.c with x and c split
 * into two BF16 planes (hi + lo) and x.c = hi.hi + hi.lo + lo.hi accumulated
 * in FP32, so a label can differ from the exact nearest centre only when two
 * centres are within ~2^-15 |x||c| of each other.  kpp_lloyd_prepare writes
 * the split of the points into the workspace; call it again whenever the
 * points change.  Asynchronous on `stream`; a bounded wait that gave up is
 * reported as KPP_ERR_TIMEOUT by kpp_read_status(workspace).
 * The assignment runs on clusters of two CTAs sharing each MMA
 * (tcgen05 cta_group::2) wherever such a cluster can be launched, else on
 * one SM per CTA; the environment variable KPP_LLOYD_PAIR=0 selects the
 * one-SM kernel.  Both give the same labels.
 */
KPP_API size_t kpp_lloyd_workspace_size(int64_t N, int32_t d, int32_t K);
KPP_API kpp_status kpp_lloyd_prepare(const float *points, int64_t N, int32_t d, int32_t K,
                                     void *workspace, size_t workspace_bytes,
                                     kpp_stream_t stream);
/*
 * The assignment half alone: labels_out [N] int32 = nearest of the K
 * centres [K x d] FP32 for the points prepared in `workspace` (same rule and
 * bound as kpp_lloyd_step).
 */
KPP_API kpp_status kpp_lloyd_assign(const float *centres, int64_t N, int32_t d, int32_t K,
                                    int32_t *labels_out, void *workspace,
                                    size_t workspace_bytes, kpp_stream_t stream);
KPP_API kpp_status kpp_lloyd_step(const float *points, int64_t N, int32_t d,
                                  const float *centres, int32_t K, int32_t *labels_out,
                                  float *d2_out, float *centres_out, int64_t *counts_out,
                                  double *phi_out, void *workspace, size_t workspace_bytes,
                                  kpp_stream_t stream);

/*
 * k-means|| -- the oversampling initialisation of Bahmani et al., which the
 * paper cites as the parallel alternative to k-means++ (Section I):
 *   1. c_0 = the first k-means++ seed, min(floor(u_0 N), N - 1) with u_0 the
 *      Philox draw of kpp_seed; D^2 = squared distance to it, phi = sum D^2.
 *   2. For rounds r = 0 .. rounds-1: point i joins the candidates iff
 *      u_{r,i} < ell D^2_i / phi, evaluated in FP64 on the stored FP32 D^2,
 *      with u_{r,i} = Philox4x64-10(key {seed, stream_id}, counter {i, r + 1,
 *      0, 0}) mapped like u_m.  The round's new candidates are appended in
 *      increasing point index; D^2 then takes the minimum over them and phi
 *      is summed again (FP64).
 *   3. Weight of a candidate = the number of points whose nearest candidate
 *      it is (the earliest in list order on a tie).
 *   4. Recluster: weighted k-means++ over the candidates in list order, on
 *      w_c (first centre) and then w_c D^2_c, draws from Philox counter
 *      {m, 0, 1, 0}, inverse CDF as in kpp_seed.
 * Arguments:
 *   points      [N x d] FP32 device, d <= 128, 1 <= K <= N < 2^31
 *   ell         expected candidates per round (> 0; e.g. 2K)
 *   rounds      >= 0 oversampling rounds (e.g. 5)
 *   cand_cap    room of cand_out / weights_out (>= 1)
 *   idx_out     [K] int64 device: the chosen points (-1 after a degenerate
 *               stop)
 *   cand_out    [cand_cap] int64 device: the candidates in list order
 *   n_cand_out  host int64: the number of candidates
 *   weights_out [cand_cap] int64 device or NULL: their weights
 *   labels_out  [N] int32 device or NULL: each point's nearest candidate
 *               (position in cand_out)
 *   d2_out      [N] FP32 device or NULL: D^2 after the rounds
 *   phi_out     [1] FP64 device or NULL: phi after the rounds
 *   workspace   >= kpp_kmeans_par_workspace_size(N, d, cand_cap) bytes,
 *               256-byte aligned
 * Distances are the FP32 difference form.  The nearest new candidate of a
 * point is searched on the tensor cores (the assignment of kpp_lloyd_step,
 * same near-tie bound) and its distance then taken exactly; the recluster
 * runs on one thread-block cluster.  The rounds keep their state on the
 * device; the call synchronises `stream` after the rounds (the number of
 * candidates sizes the recluster) and at the end -- and, only if a round drew
 * more than 4096 candidates, runs the rounds again synchronising once per
 * round -- and returns the device status: KPP_OK, KPP_ERR_DEGENERATE (fewer than K
 * candidates carry weight), KPP_ERR_TIMEOUT, or KPP_ERR_CAPACITY (more than
 * cand_cap candidates; nothing past the last whole round is written).
 */
KPP_API size_t kpp_kmeans_par_workspace_size(int64_t N, int32_t d, int64_t cand_cap);
KPP_API kpp_status kpp_kmeans_par(const float *points, int64_t N, int32_t d, int32_t K,
                                  double ell, int32_t rounds, uint64_t seed, uint64_t stream_id,
                                  int64_t cand_cap, int64_t *idx_out, int64_t *cand_out,
                                  int64_t *n_cand_out, int64_t *weights_out, int32_t *labels_out,
                                  float *d2_out, double *phi_out, void *workspace,
                                  size_t workspace_bytes, kpp_stream_t stream);

/*
 * Point-sharded seeding of one problem over several processes (one GPU
 * each): Algorithm 2's partition of the points into N_1 .. N_l, with each
 * process holding one contiguous range of rows.  Contiguous ranges keep the
 * index order of the inverse-CDF draw, so the result is the single-GPU
 * seeding's (bit-identical on data whose sums are exact).  Per pass the
 * processes exchange two small messages, which the caller carries with its
 * own collectives (e.g. NCCL through torch.distributed):
 *
 *   kpp_shard_first(s, X)                   first seed's row into X (owner) or 0s
 *   sum-all-reduce X over the processes    (int64 words)
 *   for m = 0 .. K-1:
 *     kpp_shard_pass(s, m, X, total)        D^2 update; this shard's total
 *     all-gather `total` into totals        (world x 2 floats, rank order)
 *     if m < K-1:
 *       kpp_shard_pick(s, m, totals, X)     draw of seed m+1: its owner writes
 *       sum-all-reduce X                    its row into X, the others 0s
 *   kpp_shard_phi(totals, world, phi)       phi from the last totals
 *
 * Every call is asynchronous on `stream`; nothing waits on the host between
 * passes.  The draw: every process finds, from the gathered totals, the rank
 * whose running total passes t = u * T (the same FP32-pair arithmetic on the
 * same values everywhere); that rank narrows t to a block, a warp segment and
 * a row of its own D^2 as kpp_seed's streamed form does.  T = 0 before K
 * seeds stops every process alike (indices -1, status KPP_ERR_DEGENERATE);
 * kpp_read_status(s->workspace, stream) reads a process's status.
 */
typedef struct {
    const void *points;       /* [n_local x d] this process's rows, 16-byte aligned */
    const float *row_scales;  /* [n_local] FP8 only, else NULL */
    int64_t row0;             /* global index of the first local row */
    int64_t n_local;          /* >= 1 */
    int64_t n_global;         /* rows over all processes, < 2^31 */
    int32_t d;                /* 1 <= d <= 4096 */
    int32_t K;                /* 1 <= K <= n_global */
    int32_t dtype;            /* kpp_dtype */
    int32_t rank, world;      /* 0 <= rank < world <= 1024; ranges in rank order */
    uint64_t seed, stream_id; /* Philox key of the draws, as kpp_seed */
    int64_t *indices_out;     /* [K] device: the global indices (on every process) */
    float *d2_out;            /* [n_local] device: this process's D^2 */
    void *workspace;          /* >= kpp_shard_workspace_size bytes, 256-byte aligned */
    size_t workspace_bytes;
} kpp_shard;

/* 64-bit words of the exchange buffer X for rows of d values of `dtype`
 * (the centre's global index, its FP8 scale and its stored row). */
KPP_API int64_t kpp_shard_exchange_words(int32_t d, kpp_dtype dtype);
/* Workspace bytes of one process (0 if the descriptor is invalid). */
KPP_API size_t kpp_shard_workspace_size(const kpp_shard *s, const kpp_options *opts);
/* X: [kpp_shard_exchange_words] int64 device, 16-byte aligned.  Also resets
 * the workspace's status. */
KPP_API kpp_status kpp_shard_first(const kpp_shard *s, int64_t *exchange, kpp_stream_t stream);
/* Pass m with the centre in X (after the sum-all-reduce): writes
 * indices_out[m], updates d2_out, and writes this shard's D^2 sum as an FP32
 * pair (hi, lo) to total_out[0..1] (device). */
KPP_API kpp_status kpp_shard_pass(const kpp_shard *s, int32_t m, const int64_t *exchange,
                                  float *total_out, kpp_stream_t stream,
                                  const kpp_options *opts);
/* The draw after pass m < K-1 from all_totals [world x 2] (device, rank
 * order): writes X (the owner's row, zeros elsewhere). */
KPP_API kpp_status kpp_shard_pick(const kpp_shard *s, int32_t m, const float *all_totals,
                                  int64_t *exchange, kpp_stream_t stream,
                                  const kpp_options *opts);
/* phi_out [1] FP64 device: the sum of the last gathered totals. */
KPP_API kpp_status kpp_shard_phi(const float *all_totals, int32_t world, double *phi_out,
                                 kpp_stream_t stream);

/*
 * Seeding for callers that cannot allocate device memory.  (The paper has
 * no counterpart; this is a calling convention of this library.)
 *
 * kpp_seed needs a caller-provided workspace.  Some callers cannot provide
 * one: code running under an allocator or memory pool it does not own and
 * may not grow, plugin code that is handed only its inputs and outputs, and
 * latency-critical paths where cudaMalloc -- which can synchronise the whole
 * device -- is not allowed.  kpp_seed_noalloc runs the persistent form with
 * its scratch in a fixed 16 KiB array inside the library (a static device
 * variable that every GPU loading the library holds until process exit),
 * and calls no cudaMalloc, cudaFree or allocating routine.
 *
 *   Arguments as kpp_seed, without forced prefix and workspace; `opts` may
 *   tune the persistent form (its `form` field is ignored).
 *   device_status  optional HOST pointer: if given, the call synchronises
 *                  `stream` and stores the device status there (KPP_OK,
 *                  KPP_ERR_DEGENERATE, KPP_ERR_TIMEOUT); if NULL the call
 *                  stays asynchronous.
 * Returns KPP_ERR_WORKSPACE if the problem's plan needs more scratch than
 * the fixed array holds (more than 252 CTAs), KPP_ERR_UNSUPPORTED if the
 * persistent form is not built for (dtype, d), or kpp_seed's other errors.
 *
 * The first call on each device looks up the array's device address while
 * that device is current; make that first call before any stream capture.
 * The address is kept with the device's context: after the context is
 * replaced (cudaDeviceReset), the next call looks it up again, and that
 * call too belongs before any capture.  Plans have one CTA per SM (at most
 * 152 on a GB300) unless opts asks for more per SM and they fit; a plan of
 * more than 252 CTAs is rejected as said above.
 * All calls share the one array and it keeps the last call's contents (each
 * call clears what must start at zero), so calls whose work overlaps on the
 * GPU -- on different streams, or from different threads -- race; serialise
 * them on one stream.
 */
KPP_API kpp_status kpp_seed_noalloc(const void *points, const float *row_scales, int64_t N,
                                    int32_t d, int32_t K, kpp_dtype dtype, uint64_t seed,
                                    uint64_t stream_id, int64_t *indices_out, float *d2_out,
                                    double *phi_out, kpp_stream_t stream,
                                    const kpp_options *opts, int32_t *device_status);

#ifdef __cplusplus
}
#endif

#endif /* KPP_H */
