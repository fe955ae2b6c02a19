// gj_internal.cuh -- shared declarations of the GB300 self-join library.
//
// Data kept in HBM by a built index (all device memory, library-owned):
//   X        FP64 [d][npad]  points in cell order (sorted by linear cell id,
//            then by the SORTIDU coordinate), dimensions in REORDER order,
//            structure-of-arrays so a tile of candidates is d coalesced rows.
//   orig     uint32 [n]      original row index of each sorted position.
//   cell_start int64 [G+1]   first sorted position of each non-empty cell
//            (Sec. 3.2.1: the "lookup array" ranges of the non-empty cells).
//   cell_id  int64 [G]       linearised cell ids, ascending (Sec. 3.2.1).
//   adj_start/adj            per cell, the non-empty adjacent cells b >= a
//            (3^k search of Sec. 3.2.1, halved by symmetry).
//   items    gj_item [nitems] query blocks of <= QB points of one cell.
//   order    uint32 [nitems] items by descending estimated load.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/gj.h"

namespace gj {

constexpr int QB = 128;            // most points of a work item the plain kernel holds
constexpr int QB_PLAIN = 120;      // query block of a plain-path index
constexpr int QB_TC = 120;         // query block of a tensor-core index (128-row A tile from qbeg & ~7)
constexpr int MAXK = 8;            // most indexed dimensions

struct Item {
    uint32_t cell;   // query cell index
    uint32_t qbeg;   // first sorted position of the block
    uint32_t qlen;   // points in the block (<= QB)
    uint32_t pad;
};

struct Deferred {    // resume point of an item whose results did not fit
    uint32_t item;
    uint32_t tile;   // first tile (in the item's tile order) not yet committed
};

// Device-side control block of one join launch.
struct JoinCtl {
    unsigned long long pos;        // pairs reserved in the output
    unsigned long long fail_base;  // lowest base of a reservation that did not fit
    unsigned long long counted;    // pairs counted (count-only launches)
    unsigned long long survivors;  // tensor-core filter survivors
    unsigned long long dims;       // dimensions evaluated (SHORTC depth summed over pairs)
    unsigned long long evaluated;  // candidate pairs evaluated
    unsigned int head;             // main-queue dequeue counter (monotone across launches)
    unsigned int full;             // output filled during this launch
    unsigned int din_head;         // deferred-in dequeue counter
    unsigned int dout_n;           // deferred-out entries
    unsigned int err;              // error bits (see kErr*)
    unsigned int pad[3];
};

constexpr unsigned kErrStaging = 1u;   // a tile's output did not fit the staging area
constexpr unsigned kErrTimeout = 2u;   // a bounded wait ran out
constexpr unsigned kErrDeferred = 4u;  // deferred list overflow

// Read-only geometry of an index, passed by value to kernels.
struct IndexView {
    const double *X;
    const uint32_t *orig;
    const int64_t *cell_start;
    const int64_t *adj_start;
    const uint32_t *adj;
    const Item *items;
    int64_t n, npad;
    int d;
    int u;          // SORTIDU dimension (reordered index), -1 = off
    double e2;      // fl(eps*eps)
    double ew;      // SORTIDU window half-width (eps widened)
    int ct;         // plain form: candidate tile (32 or 64), 0 = by d
    int qb;         // most points of a work item (sizes the plain kernel's query tile)
    // similarity join Q join E (asym != 0): queries come from XQ/qorig, items and
    // adjacency are the query side's, candidates the entries'; one orientation
    int asym;
    const double *XQ;
    const uint32_t *qorig;
    int64_t qnpad;
};

struct JoinLaunch {
    IndexView ix;
    const uint32_t *queue;      // item ids in dequeue order
    uint32_t qlimit;            // dequeue only while head < qlimit
    const Deferred *din;        // resume points from the previous launch
    uint32_t n_din;
    Deferred *dout;
    uint32_t dout_cap;
    JoinCtl *ctl;
    gj_pair *out;               // nullptr = count only
    unsigned long long cap;
    gj_pair *staging;           // per-CTA staging areas
    uint32_t stg_cap;           // pairs per CTA
    // optional (nullptr = not recorded): per SM slot (%smid mod kSmSlots), the
    // complement of the earliest CTA start [0, kSmSlots) and the latest CTA
    // exit [kSmSlots, 2 kSmSlots), in globaltimer ns; zero-initialised (the
    // complement turns the minimum into a maximum, whose identity is zero)
    unsigned long long *sm_span;
};

constexpr int kSmSlots = 256;

#ifdef __CUDACC__
// Record this CTA's start and exit in the launch's per-SM span slots.
__device__ __forceinline__ void note_sm_span(unsigned long long *span, unsigned long long t0,
                                             unsigned long long t1)
{
    uint32_t sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    sm %= (uint32_t)kSmSlots;
    atomicMax(&span[sm], ~t0);
    atomicMax(&span[kSmSlots + sm], t1);
}
#endif

// Index memory comes from the device's stream-ordered pool: an allocation or
// a free is queued on the build's stream and does not wait for the device
// (a build of many small indices, as for a many-jobs batch, would otherwise
// spend most of its time in the allocator).  pool_keep raises the pool's
// release threshold so that freed blocks are reused instead of returned.
template <class T>
inline cudaError_t dev_alloc(T **p, size_t bytes, cudaStream_t s)
{
    return cudaMallocAsync(reinterpret_cast<void **>(p), bytes, s);
}
inline void dev_free(void *p, cudaStream_t s)
{
    if (p)
        cudaFreeAsync(p, s);
}
void pool_keep(int device);
// An output buffer the kernels may write: device or managed memory as it is;
// nullptr for host memory (pageable or pinned), which the join fills by copies.
gj_pair *device_view(gj_pair *p);
// Device memory of `device` itself, or managed memory: a buffer the kernels of
// a handle on `device` may read and write.
bool device_memory_of(const void *p, int device);
// Device memory of another device: the kernels of a handle on `device` must
// not touch it (without peer access that is an illegal address), so the entry
// points reject it with GJ_ERR_INVALID_ARG.
bool foreign_device(const void *p, int device);

// Count of kernels this library has launched (process-wide); read through
// gj_kernel_launches().
void note_launch();
unsigned long long launches_so_far();

// ---- kernels and launchers (gj_index.cu) --------------------------------
cudaError_t launch_check_finite(const double *P, int64_t count, unsigned int *flag, cudaStream_t s);
cudaError_t launch_dim_stats(const double *P, int64_t n, int d, double *part, int nblk, double *stats,
                             cudaStream_t s);

struct Scratch;   // temporary device buffers of a build

// radix sort of (key64, val32) pairs on bits [lo, hi); result in (k0, v0)
cudaError_t radix_sort_pairs(uint64_t *k0, uint32_t *v0, uint64_t *k1, uint32_t *v1, int64_t n,
                             int lo, int hi, uint32_t *counts, int64_t counts_cap, cudaStream_t s);

// exclusive scan of int64 values in place; returns total via *total_dev (device)
cudaError_t exclusive_scan_i64(int64_t *data, int64_t n, int64_t *tmp, int64_t tmp_cap,
                               cudaStream_t s);

int64_t radix_counts_needed(int64_t n);
int64_t scan_tmp_needed(int64_t n);
int build_index(gj_index *h, const double *P, int64_t n, int d, double eps, int k_req, uint32_t flags,
                cudaStream_t s);

// ---- join kernels (gj_join.cu) -------------------------------------------
cudaError_t launch_join_plain(const JoinLaunch &L, int grid, cudaStream_t s);
cudaError_t launch_join_plain_direct(const JoinLaunch &L, int grid, cudaStream_t s);
int plain_ctas_per_sm(int d, int ct, int qb);
size_t plain_smem_bytes(int d, int ct, int qb);
cudaError_t launch_fp64_probe(double *out, int iters, int grid, cudaStream_t s);

// Per-job parameters of a many-jobs launch (gj_batch.cu).
struct TcJob {
    double e2, ew;       // fl(eps^2), SORTIDU window half-width
    int u;               // SORTIDU dimension or -1
    int Tbits;           // fp32 bits of the job's survivor threshold
    int d;               // the job's own dimensions (the combined layout pads to the largest)
    int pad;
    gj_pair *out;        // the job's device output (nullptr = count only)
    unsigned long long cap;
};

// ---- tensor-core filter (gj_tc.cu) -----------------------------------------
int tc_prepare(gj_index *h, const double *stats_host, const int *perm, cudaStream_t s);
// direct = true: pairs straight into L.out (device-addressable) with one
// reservation per warp, no staging and no resume (L.ctl->pos counts every
// pair, written or not); false: per-CTA staging committed per work item.
cudaError_t launch_join_tc(const gj_index *h, const JoinLaunch &L, int grid, cudaStream_t s, bool direct);
size_t tc_staging_pairs_per_cta();
int tc_threshold_bits(double eps, double sigma, double R0, int d, int Kp);
// XA or XB may be null (only the other operand is written)
cudaError_t tc_pack_into(const double *X, int64_t n, int64_t npad, int d, int Kp, double sigma, const double *centre,
                         int64_t row_off, void *XA, void *XB, cudaStream_t s);
// largest distance of n points (structure-of-arrays, row stride npad) from
// centre, widened by 1 + 2^-30; synchronous
cudaError_t tc_radius(const double *X, int64_t n, int64_t npad, int d, const double *centre, double *R0,
                      cudaStream_t s);
double tc_sigma_for(double R0);
// direct form over explicit operands (L.ix.asym: Q join_eps E)
cudaError_t launch_join_tc_ops(const JoinLaunch &L, const void *XA, const void *XB, const double *XR, int dr, int Kp,
                               int Tbits, int grid, cudaStream_t s);
// job_cycles (nullable): per-job SM cycles between the epilogue's item ends,
// summed over CTAs (the autotuner's per-job timing)
cudaError_t launch_join_tc_jobs(const JoinLaunch &L, const void *XA, const void *XB, int Kp, const TcJob *jobs,
                                unsigned long long *jpos, int grid, cudaStream_t s,
                                unsigned long long *job_cycles = nullptr);
cudaError_t tc_jobs_launch_attr(int Kp);
void set_last_status(int st);

// Query side of a similarity join Q join_eps E (gj_index.cu, gj_qjoin.cu): the
// queries sorted into the entry index's grid, with their own cells, the
// entry cells adjacent to each, and work items.
struct QuerySide {
    int64_t nq = 0, qnpad = 0;
    double *XQ = nullptr;           // FP64 [d][qnpad]: queries in (cell, u) order, dimensions in REORDER order
    uint32_t *qorig = nullptr;      // original query row of each sorted position
    int64_t Gq = 0;
    int64_t *qcell_start = nullptr; // [Gq + 1]
    int64_t *qcell_id = nullptr;    // [Gq] entry-grid linear ids
    int64_t *adj_start = nullptr;   // [Gq + 1] into adj
    uint32_t *adj = nullptr;        // entry cells adjacent to each query cell
    Item *items = nullptr;
    uint32_t *order = nullptr;      // items by descending load
    int64_t nitems = 0;
    unsigned long long candidates = 0;   // query x entry pairs in adjacent cells
};
int build_query_side(const gj_index *h, const double *Q, int64_t nq, int qb, QuerySide *qs, cudaStream_t s);
void free_query_side(QuerySide *qs, cudaStream_t s);

// Autotuner (gj_tune.cu): runs the trials; *best_out (nullable) receives the
// index of the pick, built, else it is freed.
int autotune_impl(const double *points, int64_t n, int d, double eps, const gj_config *cfg, gj_tune_result *out,
                  gj_index **best_out);

}  // namespace gj

namespace gj {
struct StagedState;   // gj_api.cu
}

// The handle (gj_api.cu)
struct gj_index {
    int device;
    cudaStream_t stream;
    bool own_stream;
    cudaStream_t drain_stream;
    gj_config cfg;
    gj_index_info_t info;
    gj_join_stats last;
    // device arrays
    double *X;
    uint32_t *orig;
    int64_t *cell_start;
    int64_t *cell_id;
    int64_t *adj_start;
    uint32_t *adj;
    gj::Item *items;
    uint32_t *order;     // items by descending load
    int64_t npad;
    int64_t G;
    int64_t nitems;
    int64_t nadj;        // adjacency entries (sum of the cells' lists)
    int u;
    double e2, ew;
    int sms;
    // the grid (for query sides of a similarity join)
    int grid_k, grid_bits;
    int grid_perm[gj::MAXK];
    double grid_origin[gj::MAXK], grid_invw[gj::MAXK];
    int64_t grid_nc[gj::MAXK], grid_stride[gj::MAXK];
    int *perm_dev;       // device: REORDER permutation of all d dimensions
    int qb;              // query block size the items were built with
    int q_align;         // > 0: items split at multiples of q_align positions
    int plain_ct;        // plain form: candidate tile, 0 = by d
    // tensor-core filter operands (GJ_TC_FILTER)
    bool tc_ready;
    void *XA, *XB;       // fp16 [npad + 512][Kp] in core-matrix order
    int tc_Kp;
    int tc_Tbits;        // fp32 bits of the survivor threshold (scaled units)
    double tc_sigma, tc_R0;
    double *tc_centre;   // device, the filter's centre per reordered dimension
    double *XR;          // device, the points row by row (n x XR_dr FP64) for the FP64 recheck
    int XR_dr;
    // launch state of the tensor-core join's direct form, allocated by the
    // first such join on the handle and kept until gj_free
    bool jd_ready;
    gj::JoinCtl *jd_ctl, *jd_hctl;          // device, pinned host
    uint32_t *jd_queue;                      // device, one entry per work item
    unsigned long long *jd_span, *jd_hspan;  // per-SM spans: device, pinned host
    cudaEvent_t jd_ev0, jd_ev1;
    // launch state of the staged join (result batches, plain form), allocated
    // by the first such join on the handle and kept until gj_free
    gj::StagedState *ss;
};
