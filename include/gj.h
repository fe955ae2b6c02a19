/*
 * gj.h -- C ABI of the GB300 epsilon-distance similarity self-join.
 *
 * The library finds every ordered pair (a, b) of rows of a point set D whose
 * Euclidean distance is at most eps (Sec. 3.1, problem statement): dist(a,b) =
 * sqrt(sum_j (a_j - b_j)^2) <= eps.  Like the paper's result tuples (Sec. 3.2.1:
 * key/value pairs, one per neighbour of each query point) and its selectivity
 * S_D = (|R| - |D|)/|D| (Sec. 5.2, Eq. 1), the result R holds both orientations
 * (a,b) and (b,a) of every pair and the |D| self-pairs (a,a).
 *
 * Method (Alg. 1): REORDER dimensions by variance (Sec. 4.2); build a grid
 * index of eps-wide cells over the first k reordered dimensions, non-empty
 * cells only, linearised and sorted (Sec. 3.2.1, 4.1); search the 3^k adjacent
 * cells of each query cell (Sec. 3.2.1, Fig. 1), optionally narrowed by a
 * window on one un-indexed dimension (SORTIDU, Sec. 4.3); compute FP64 squared
 * distances that stop once the running sum exceeds eps^2 (SHORTC, Sec. 4.4);
 * emit pairs in result-set batches (Sec. 3.2.2) over a work queue ordered by
 * estimated cell load.  Every stage runs as CUDA kernels on one GPU.
 *
 * Exactness.  A pair is reported iff its FP64 squared distance, summed over
 * the reordered dimensions, is <= fl(eps*eps).  The summation order (reordered
 * dimensions, fused multiply-add) differs from the original-order sum only in
 * the last bits, so the result can differ from an original-order reference
 * only for pairs whose squared distance lies within ~d*2^-53 relative of eps^2.
 *
 * Threading: a handle is used by one host thread at a time.  Status codes are
 * returned by value; gj_index_build returns NULL and leaves its status in a
 * thread-local slot read by gj_last_status().
 */
#ifndef GJ_H
#define GJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define GJ_OK                 0
#define GJ_ERR_INVALID_ARG   -1  /* n < 0, d < 1, eps <= 0 or NaN, k out of range, NULL handle ... */
#define GJ_ERR_NONFINITE     -2  /* a coordinate is NaN or infinite                                  */
#define GJ_ERR_OOM           -3  /* device or pinned host allocation failed                          */
#define GJ_ERR_CUDA          -4  /* a CUDA runtime call or kernel launch failed                      */
#define GJ_ERR_CAPACITY      -5  /* |R| > cap: *count holds |R|; output contents unspecified         */
#define GJ_ERR_TIMEOUT       -6  /* a bounded device-side wait ran out; the context stays usable     */
#define GJ_ERR_UNSUPPORTED   -7  /* no usable device (needs compute capability 10.3, sm_103a), or a
                                 * join whose tiles do not fit shared memory (plain form: d above
                                 * about 290 with the default query block)                        */
#define GJ_ERR_TOO_LARGE     -8  /* n >= 2^32 (pair ids are 32-bit) or d > GJ_MAX_DIMS               */

#define GJ_MAX_DIMS 1024

/* ---- flags (gj_config.flags) -------------------------------------------- */
#define GJ_REORDER    (1u << 0)  /* Sec. 4.2: index the k highest-variance dimensions       */
#define GJ_SORTIDU    (1u << 1)  /* Sec. 4.3: sort cells by one un-indexed dim, window search */
#define GJ_SHORTC     (1u << 2)  /* Sec. 4.4: stop a distance once it exceeds eps^2          */
#define GJ_TC_FILTER  (1u << 3)  /* tensor-core candidate filter + exact FP64 recheck (no paper counterpart);
                                  * the index also holds the fp16 operand rows (2 x 2 x Kp bytes per
                                  * point, Kp = d + 4 rounded up to 16) and a row-major FP64 copy of
                                  * the points for the recheck (8 x (d rounded up to 4) bytes)        */
#define GJ_AUTOTUNE   (1u << 4)  /* build: pick k, query block, tile and b_s by timed trials (gj_autotune) */
#define GJ_TUNE_FORM  (1u << 5)  /* autotune: also try both forms (plain and GJ_TC_FILTER), keep the faster */
#define GJ_HOST_BATCHED (1u << 6) /* host output always through the result batches of Sec. 3.2.2
                                   * (a tensor-core index otherwise fills one device buffer of cap
                                   * pairs and copies it)                                      */
#define GJ_DEFAULT_FLAGS (GJ_REORDER | GJ_SORTIDU | GJ_SHORTC)

/* One result pair: original row indices of the two points. */
typedef struct {
    uint32_t a, b;
} gj_pair;

/* Opaque index handle (library-owned device memory). */
typedef struct gj_index gj_index;

/* Build options.  Zero-initialise, then set what you need; gj_config_init
 * fills the defaults. */
typedef struct {
    int32_t  k;           /* indexed dimensions: 0 = choose automatically; else 1..min(d,8)      */
    uint32_t flags;       /* GJ_* flags; gj_config_init sets GJ_DEFAULT_FLAGS                     */
    void    *stream;      /* cudaStream_t to run on; NULL = a stream the handle creates             */
    uint64_t batch_pairs; /* result batch size b_s in pairs; 0 = the rule of Sec. 3.2.2           */
    int32_t  device;      /* CUDA device ordinal; -1 = the calling thread's current device        */
    int32_t  query_block; /* points per work item (query tile): 0 = default (120 points; the
                           * tensor-core form: pieces of a cell between multiples of 128
                           * sorted positions); 8..128, and at most 120 with GJ_TC_FILTER   */
    int32_t  tile;        /* plain form: candidate points staged per shared-memory tile,
                           * 0 = default (64 for d <= 32, else 32), 32 or 64                    */
    uint32_t reserved[5];
} gj_config;

/* Read-only facts about a built index. */
typedef struct {
    int64_t  n;
    int32_t  d;
    int32_t  k;              /* indexed dimensions actually used                                 */
    double   eps;
    int64_t  nonempty_cells; /* |G| (Sec. 3.2.1)                                                  */
    int64_t  work_items;     /* query blocks in the load-ordered work queue                     */
    uint64_t candidate_pairs;/* unordered candidate pairs i<j in adjacent cells (no SORTIDU)     */
    uint64_t window_pairs;   /* unordered candidate pairs left after the SORTIDU window          */
    uint32_t flags;
    int32_t  sortidu_dim;    /* reordered index of the SORTIDU dimension, -1 if off             */
    int32_t  perm[GJ_MAX_DIMS]; /* REORDER: perm[r] = original index of reordered dimension r   */
} gj_index_info_t;

/* Per-call measurements of the last gj_self_join on a handle. */
typedef struct {
    uint64_t pairs;          /* |R|                                                               */
    uint32_t launches;       /* join kernel launches (result batches + overflow resumes)          */
    uint32_t batches_planned;/* n_b from the sampled estimate (Sec. 3.2.2)                       */
    uint64_t batch_pairs;    /* b_s used                                                         */
    uint64_t estimate;       /* sampled |R| estimate                                             */
    uint64_t tc_survivors;   /* GJ_TC_FILTER: candidates passed to the FP64 recheck             */
    uint64_t evaluated;      /* candidate pairs whose distance was computed (after SORTIDU)       */
    uint64_t dims;           /* FP64 dimensions evaluated, summed over those pairs (SHORTC depth) */
    double   join_ms;        /* device time of the join kernels (CUDA events)                   */
    double   estimate_ms;    /* device time of the sampled estimate                              */
    double   total_ms;       /* host wall time of the call                                       */
    double   busy_ms;        /* join kernels: each SM's occupied span (earliest CTA start to
                              * latest CTA exit), averaged over the SMs of a launch, summed over
                              * launches (the join's work spread evenly over the SMs: its time
                              * without the tail)                                                 */
    uint64_t candidates;     /* gj_join_qe: query x entry pairs in adjacent cells (its evals unit) */
} gj_join_stats;

/* Fill *cfg with defaults (k = 0, GJ_DEFAULT_FLAGS, own stream, paper batch rule). */
void gj_config_init(gj_config *cfg);

/*
 * Build the index of Alg. 1 (REORDER, constructIndex) for n points of d
 * dimensions.
 *   points  row-major n x d FP64, in host memory (pageable or pinned) or in
 *           device memory of the chosen device; detected with
 *           cudaPointerGetAttributes.  It is copied; the caller keeps ownership
 *           and may free or change it after the call returns.
 *   n       number of points, 0 <= n < 2^32.
 *   d       dimensions, 1 <= d <= GJ_MAX_DIMS.  The plain join holds a query
 *           tile and a candidate tile of d FP64 rows in shared memory: up to
 *           about 290 dimensions with the default blocks (64 queries x 32
 *           candidates above 32 dimensions); the tensor-core form up to 124.
 *   eps     search distance, finite and > 0.
 *   k       indexed dimensions: 0 = choose automatically (Sec. 4.1 trade-off),
 *           else 1 <= k <= min(d, 8).  The library may index fewer dimensions
 *           than asked when the linear cell id would not fit in 62 bits; the
 *           pair set never depends on k.
 * Returns a handle, or NULL with the reason in gj_last_status().
 */
gj_index *gj_index_build(const double *points, int64_t n, int32_t d, double eps, int32_t k);
gj_index *gj_index_build_ex(const double *points, int64_t n, int32_t d, double eps,
                            const gj_config *cfg);

/* Choices of the autotuner for one input. */
typedef struct {
    int32_t  k;            /* indexed dimensions                                              */
    uint32_t flags;        /* the input flags with GJ_TC_FILTER set or cleared by the pick     */
    int32_t  query_block;  /* gj_config.query_block of the pick (0 = the default blocks)      */
    int32_t  tile;         /* plain form: candidate tile (0 for the tensor-core form)         */
    uint64_t batch_pairs;  /* result batch size b_s for host output                           */
    uint64_t est_pairs;    /* |R| extrapolated from the trial join of the pick                */
    double   build_ms;     /* device-synchronous host time of the pick's index build          */
    double   join_ms;      /* join kernel time extrapolated from the pick's trial             */
    int32_t  trials;       /* timed trials run                                                */
    int32_t  reserved;
} gj_tune_result;

/*
 * Autotuner (no paper counterpart; the paper fixes k by a comparison of
 * candidate counts against index search cost, Sec. 4.1).  Picks k, the query
 * block and the plain form's candidate tile by timed trials: for each
 * candidate setting it builds the index and times a count-only join over a
 * fixed, load-stratified share of the work items (one part of an entity
 * partition, Sec. 6.2; the part sized so that a trial's join takes about
 * 40 ms), extrapolated to the whole queue; the setting with the least build +
 * join time wins (by at least 2 %, else the earlier setting stays).  k runs
 * over 1..min(d, 8) (1..3 for the tensor-core form), then the query block
 * over {default, 64} and the plain candidate tile over {64, 32}.  With
 * GJ_TUNE_FORM in cfg->flags both forms are tried, else only the form
 * cfg->flags names.  The result batch size b_s is then
 * chosen from the trial's |R| estimate, a timed device-to-host copy and the
 * measured per-launch overhead, so that the drain of each batch hides under
 * the join of the next (at least 3 batches, Sec. 3.2.2).
 *   points, n, d, eps, cfg  as for gj_index_build_ex (cfg->k is ignored).
 *   out     the pick.
 * Returns GJ_OK or an error code.  Every trial runs on cfg's device and
 * stream; nothing persists after the call.
 */
int gj_autotune(const double *points, int64_t n, int32_t d, double eps, const gj_config *cfg,
                gj_tune_result *out);

/*
 * The self-join (Alg. 1, batch loop and SelfJoinKernel): writes R into
 * pairs_out in no particular order.
 *   pairs_out  host memory (pageable or pinned) or device memory of the
 *              handle's device, for cap pairs; NULL with cap == 0 asks for the
 *              count only (returns GJ_OK).
 *   cap        capacity of pairs_out in pairs.
 *   count      out: |R| (always the full size, also on GJ_ERR_CAPACITY).
 * Returns GJ_OK, or GJ_ERR_CAPACITY when |R| > cap (the contents of pairs_out
 * are then unspecified), GJ_ERR_INVALID_ARG when pairs_out is device memory of
 * another device, or another error code.  Pageable host output is
 * copied in result batches (Sec. 3.2.2) on a second stream while the next
 * batch runs.  The kernels write device memory only: host output, pageable
 * or pinned, is always filled by copies.  For an index built with
 * GJ_TC_FILTER (and without GJ_HOST_BATCHED) the join runs in one pass into a
 * device buffer of cap pairs from the stream-ordered pool, copied to
 * pairs_out when the join ends; it falls back to the result batches when that
 * buffer cannot be allocated.  Memory: the first join on a handle allocates
 * its launch state (control block, pinned mirrors, work order, deferred
 * lists, events), which the handle keeps until gj_free; the per-call buffers
 * (staging, result batches, the tensor-core output buffer) come from the
 * device's stream-ordered pool, which keeps freed blocks for reuse.
 */
int gj_self_join(gj_index *h, gj_pair *pairs_out, uint64_t cap, uint64_t *count);

/*
 * Entity partitioning (Sec. 6.2): the part of R computed by query set
 * l = part of N_b = nparts, where the load-ordered query blocks are dealt to
 * the sets round-robin (block r goes to set r mod N_b).  Every unordered pair
 * is computed by exactly one query block, which emits both orientations, so
 * the parts are disjoint and their union is R.  Semantics of
 * pairs_out/cap/count as in gj_self_join.
 */
int gj_self_join_part(gj_index *h, int32_t part, int32_t nparts, gj_pair *pairs_out,
                      uint64_t cap, uint64_t *count);

/*
 * The similarity join Q join_eps E (Sec. 3.1; the self-join is the case
 * Q = E): every pair (q, e) of a query row q and an entry row e with
 * dist(q, e) <= eps, one orientation, q indexing the queries and e the rows
 * the index h was built from (the entries, E).  The queries are keyed into
 * E's grid (its REORDER permutation, cell width and origin), sorted by cell
 * and by E's SORTIDU dimension; each query cell searches all adjacent
 * non-empty entry cells; distances are the FP64 SHORTC sums of the self-join.
 * The join runs in the index's form: the plain FP64 kernel, or, for an index
 * built with GJ_TC_FILTER, the tensor-core filter and its FP64 recheck (the
 * same pair set).  The tensor-core form packs the queries as fp16 A rows under
 * the entries' centre, with one power-of-two scale for both sets: queries
 * farther from that centre than every entry give a smaller scale, for which
 * the entries are re-packed for the call (more device memory, a looser
 * filter, the same result).
 *   h          an index over E (any flags)
 *   queries    row-major nq x d FP64 (d = E's), host or device memory (of
 *              any device); copied, the caller keeps ownership
 *   pairs_out  host memory or device memory of the handle's device for cap
 *              pairs (a = query row, b = entry row); another device's memory
 *              returns GJ_ERR_INVALID_ARG; NULL with cap == 0 counts only
 *   count      out: |Q join_eps E|
 * One kernel launch writes the pairs and counts them: into pairs_out directly
 * when it is device memory, else into a device buffer of cap pairs that is
 * then copied to the host buffer.  Returns GJ_OK;
 * GJ_ERR_CAPACITY when the result exceeds cap (*count holds its size; the
 * buffer holds an unspecified cap of them); GJ_ERR_NONFINITE for a NaN or
 * infinite query coordinate; or another error code.  The eps is the index's.
 */
int gj_join_qe(gj_index *h, const double *queries, int64_t nq, gj_pair *pairs_out, uint64_t cap,
               uint64_t *count);

/*
 * The neighbour table (Alg. 1, constructNeighborTable; Sec. 3.2.2: the
 * result's key/value pairs stored with each key once).  Compressed sparse
 * rows over the original point order: the neighbours of point a are
 * nbr[row_start[a] .. row_start[a+1]), ascending, a itself included.  Built on
 * the device from a join into library-allocated device memory (8 bytes per
 * pair, plus 20 bytes per pair while the pairs are sorted).
 *   row_start  device memory of the handle's device, int64 [n + 1]
 *   nbr        device memory, uint32 [cap]
 *   count      out: |R|
 * Returns GJ_OK; GJ_ERR_CAPACITY when |R| > cap (*count = |R|, nothing
 * written); GJ_ERR_INVALID_ARG when a buffer is not device memory; or another
 * error code.
 */
int gj_neighbor_table(gj_index *h, int64_t *row_start, uint32_t *nbr, uint64_t cap, uint64_t *count);

/*
 * A self-join that allocates nothing (no paper counterpart).  gj_self_join
 * allocates its launch state on a handle's first join and takes its staging
 * and batch buffers from the stream-ordered pool on every call.  Callers whose
 * device memory is reserved up front by a caching allocator, or whose latency
 * budget forbids entering the driver's allocator during a join, cannot accept
 * that; this entry point serves them.  It runs the plain FP64 join (not the tensor-core filter)
 * and writes pairs straight into pairs_out, which must be device memory of the
 * handle's device, else GJ_ERR_INVALID_ARG (NULL with cap == 0: count only; a
 * non-NULL pairs_out with cap == 0 writes nothing and returns GJ_ERR_CAPACITY
 * with *count = |R| when |R| > 0).  Its scratch -- the
 * control block and the dequeue order of the part's work items -- lives in one
 * 4 MiB array in device global memory that the library declares at file scope;
 * every GPU that loads the library holds that array until the process exits.
 *   h, part, nparts  as gj_self_join_part (part = 0, nparts = 1: the whole R).
 *   limit            at most (4 MiB - 256 B) / 4 = 1,048,512 work items in the
 *                    part (about 125 million points in large cells); larger
 *                    parts return GJ_ERR_TOO_LARGE.  Indices built with
 *                    GJ_TC_FILTER return GJ_ERR_INVALID_ARG.
 *   set-up           the first call on a device looks up the array's device
 *                    address (cudaGetSymbolAddress) with that device current,
 *                    and so does the first call after that device's context
 *                    was reset; make that first call before any stream
 *                    capture.  The call is synchronous: it returns once the
 *                    join has finished on the handle's stream.
 *   sharing          all calls share the array and find the last call's
 *                    contents (the call clears what must start at zero).
 *                    Calls that overlap on the GPU race on it: do not run two
 *                    at once, on any handle or stream of the same device.
 * Returns as gj_self_join: GJ_OK, or GJ_ERR_CAPACITY with *count = |R| when
 * |R| > cap (then pairs_out holds cap pairs of R), or another error code.
 * The call itself allocates nothing: no cudaMalloc, no cudaFree, no event or
 * stream creation.
 */
int gj_self_join_noalloc(const gj_index *h, int32_t part, int32_t nparts, gj_pair *pairs_out,
                         uint64_t cap, uint64_t *count);

/* ---- many independent self-joins in one launch (no paper counterpart) ---- */

/* One job of a batched self-join: its own points (host or device, as for
 * gj_index_build), size, dimension, search distance and k (0 = automatic). */
typedef struct {
    const double *points;
    int64_t n;
    int32_t d;
    int32_t k;
    double eps;
} gj_job;

typedef struct gj_batch gj_batch;

/*
 * Build the indices of njobs independent self-joins and combine them into one
 * structure: points back to back (zero-padded to the largest d, which changes
 * no distance), cells, adjacency and work items shifted per job, and one
 * queue of every job's work items in descending estimated load.  All jobs use
 * the tensor-core filter form (largest d at most 124).  cfg: device and
 * stream as for gj_index_build_ex; flags REORDER/SORTIDU/SHORTC apply to
 * every job.  Returns NULL with the reason in gj_last_status().
 */
gj_batch *gj_batch_build(const gj_job *jobs, int32_t njobs, const gj_config *cfg);
/*
 * With GJ_AUTOTUNE in cfg->flags, every job whose k is 0 gets its k from
 * timed trials: the whole batch is built and joined (count only) once with
 * every such job at k = 1, 2 and 3 (capped at its d), the kernel timing each
 * job's work items on the SM clock, and each job keeps the k of its fastest
 * trial.  The picks are remembered per process for the same list of job
 * shapes (n, d, eps), so a later build of that list skips the trials.
 */

/*
 * Join every job in one persistent kernel launch.  The launch (parameter
 * upload, counter reset, kernel, counter download) is captured in a CUDA graph
 * on the first call and replayed on later calls.
 *   outs[j]   device buffer of job j for caps[j] pairs (original row ids of
 *             job j); NULL with caps[j] == 0 counts job j only.  outs and caps
 *             may be NULL: count every job.
 *   counts[j] out: |R_j|.
 * Returns GJ_OK, or GJ_ERR_CAPACITY when some job's |R_j| exceeds caps[j]
 * (that buffer then holds caps[j] pairs of R_j).
 */
int gj_batch_self_join(gj_batch *b, gj_pair *const *outs, const uint64_t *caps, uint64_t *counts);

/* Work items, total points and the summed unordered candidate pairs of the
 * jobs' grids (the unit of the distance-evaluation rate).  Any output may be NULL. */
int gj_batch_get_info(const gj_batch *b, int64_t *work_items, int64_t *total_points, uint64_t *candidate_pairs);

/* The k each job's grid uses (k_per_job[j], njobs entries): the job's own k,
 * or the autotuner's pick when the batch was built with GJ_AUTOTUNE. */
int gj_batch_get_k(const gj_batch *b, int32_t *k_per_job);

/* Release a batch.  NULL-safe. */
void gj_batch_free(gj_batch *b);

/* Facts about the index (k used, REORDER permutation, cell and candidate counts). */
int gj_index_get_info(const gj_index *h, gj_index_info_t *info);

/* Measurements of the last join on this handle. */
int gj_last_join_stats(const gj_index *h, gj_join_stats *st);

/* Release the handle and its device memory.  NULL-safe. */
void gj_free(gj_index *h);

/* Status of the last gj_index_build* on this thread. */
int gj_last_status(void);

/* Static English text for a status code. */
const char *gj_status_string(int status);

/* Library version, "major.minor.patch". */
const char *gj_version(void);

/* Measurement helper (no paper counterpart): FP64 fused multiply-add
 * throughput of the device in TFLOP/s (2 FLOPs per FMA), from independent
 * FMA chains timed with CUDA events; the denominator of the plain join's
 * roofline.  device = -1 for the current device. */
int gj_probe_fp64_tflops(int32_t device, double *tflops);

/* Diagnostic (no paper counterpart): one 128 x 128 tile D = A * B^T on the
 * tensor cores through the operand layout, descriptors and TMEM path of the
 * GJ_TC_FILTER join.  A and B are row-major [128][Kp] fp16 bit patterns in host
 * memory, Kp a multiple of 16 in [16, 128]; D is row-major [128][128] fp32 in
 * host memory.  The tile is read back with the join's reducing TMEM load
 * (values and per-lane minimum of each 32 columns); a minimum that differs from
 * the minimum of the values returned gives GJ_ERR_CUDA.  Runs on the current
 * device; returns GJ_OK or an error code. */
int gj_debug_tc_tile(const uint16_t *A, const uint16_t *B, int32_t Kp, float *D);

/* Diagnostic (no paper counterpart; host only, no device needed): the
 * tensor-core filter's survivor threshold.  For coordinates scaled by sigma
 * about a centre and held within radius R0 of it (h = rn16(sigma (x - c))),
 * every pair within eps has its computed t = |h_a|^2 + |h_b|^2 - 2 <h_a, h_b>
 * (fp16 products, fp32 accumulation, norms split hi/lo) at most *T.
 *   eps, sigma  > 0 and finite; R0 >= 0 and finite; 1 <= d <= 124.
 *   T           out: the fp32 value the kernel compares t with (the bound
 *               rounded up to fp32).
 * Returns GJ_OK or GJ_ERR_INVALID_ARG. */
int gj_tc_threshold(double eps, double sigma, double R0, int32_t d, float *T);

/* Diagnostic (no paper counterpart): the limit, in nanoseconds, of every
 * bounded device-side wait of the tensor-core joins launched after the call,
 * process-wide (0 restores the default, 4 s per wait).  A limit of a few
 * nanoseconds makes a join's waits run out: the kernel records the expiry,
 * lets its copies and MMAs in flight land, frees its tensor memory and
 * returns, and the join returns GJ_ERR_TIMEOUT with the context usable.  Used
 * by the tests to exercise that path without any device fault.  Returns GJ_OK. */
int gj_debug_set_wait_limit(uint64_t ns);

/* Measurement helper (no paper counterpart): number of CUDA kernels this
 * library has launched in this process so far (all handles, all threads). */
unsigned long long gj_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* GJ_H */
