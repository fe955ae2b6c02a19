// gj_tc.cu -- tensor-core candidate filter with an exact FP64 recheck.
//
// No paper counterpart: the paper computes every candidate distance on the
// FP32 cores (Sec. 4.4).  Here a candidate pair first meets a cheap,
// conservative test on the 5th-generation tensor cores; only survivors get
// the plain path's FP64 SHORTC distance, so the reported set is exactly the
// plain path's set.
//
// Filter.  With a common centre c (per-dimension midrange) and a power-of-two
// scale sigma, every point x gets fp16 coordinates h = rn16(sigma * (x - c)).
// The A row of a query is [-2h, |h|^2_hi, |h|^2_lo, 1, 1, 0...] and the B row
// of a candidate [h, 1, 1, |h|^2_hi, |h|^2_lo, 0...] (K = d + 4 padded to a
// multiple of 16), so one fp16 x fp16 -> fp32 MMA gives
//     t = |h_a|^2 + |h_b|^2 - 2 <h_a, h_b>  ~  sigma^2 |a - b|^2.
// A pair is kept iff t <= T.  T bounds, for every pair within eps, the fp16
// rounding of both points (|h - sigma(x-c)| <= 2^-11 |.| + 2^-25 per
// coordinate), the hi/lo split of the norms (<= 2^-22 relative) and the fp32
// accumulation (taken as <= (K+2) * 2^-22 * sum of |terms|, twice a
// truncating adder's bound).  Every pair of R therefore survives.
//
// Kernel (one persistent CTA per SM, 384 threads):
//   warp 0   producer: takes work items (query blocks of <= 128 points),
//            computes the SORTIDU windows of the adjacent cells (one per lane),
//            packs them into 256-row candidate tiles under a valid-row mask
//            (lane 0, state in registers; runs of whole tiles are pushed
//            warp-wide, one ring stage per lane), and loads the item's 128-row
//            A tile and each candidate tile with bulk asynchronous copies into
//            shared-memory stages, the tile descriptor beside each stage;
//   warps 1, 10  MMA issuers, one thread each, one 256-column fp32 TMEM
//            accumulator each (turns of parity 0 and 1): one M=128 x N=256
//            tcgen05.mma per K step, commits to the stage's and the
//            accumulator's mbarriers;
//   warps 2-9 epilogue: every warp reads its 32 TMEM lanes of one 128-column
//            half of each tile, 32 columns at a time with tcgen05.ld.red,
//            which also returns each lane's minimum, marks the values <= T of
//            a chunk whose minimum is <= T in per-lane bit masks and releases
//            its share of the accumulator.  Direct form: the warps hand their
//            survivors to
//   warp 11  the recheck warp, which runs the FP64 test and writes the exact
//            pairs straight to the output.  Staged form: the warps recheck
//            their own survivors and commit per-CTA staging per item (the
//            plain kernel's resume protocol).
// Every wait is bounded (globaltimer); on timeout the CTA flags the error,
// lets in-flight copies land, frees its TMEM and returns.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "gj_internal.cuh"
#include "gj_sm100.cuh"

namespace gj {

using namespace sm100;

constexpr int TC_THREADS = 384;   // producer, MMA issuer x2, epilogue x8, recheck
constexpr int TC_N = 256;        // candidate rows per tile (one M=128 x N=256 MMA per K step)
constexpr int TC_M = 128;        // query rows per A tile
constexpr int TC_MAXS = 8;       // most B-tile stages (one descriptor slot per stage)
constexpr uint32_t TC_STG = 1u << 18;   // staging pairs per half per CTA (4 tiles of worst-case output)
constexpr uint64_t TC_LIMIT_NS = 4000000000ull;   // 4 s per wait

// Diagnostic: the limit of every bounded wait in later tensor-core joins
// (0: TC_LIMIT_NS).  A short limit makes the waits run out, which exercises
// the timeout path (error status, copies in flight drained, TMEM freed)
// without any fault.
static std::atomic<unsigned long long> g_wait_limit_ns{0};
static unsigned long long wait_limit_ns()
{
    const unsigned long long v = g_wait_limit_ns.load(std::memory_order_relaxed);
    return v ? v : TC_LIMIT_NS;
}
constexpr int TC_SQ = 64;        // survivor queue per epilogue warp
constexpr int TC_RQ = 64;        // direct form: survivors handed to the recheck warp, per epilogue warp

// F_PAD: a no-op turn after an item that made one turn only, so that every
// item has a turn of each parity (each MMA issuer sees every item)
enum : uint32_t { F_FIRST = 1, F_LAST = 2, F_MARKER = 4, F_TRUNC = 8, F_TERM = 16, F_PAD = 32, F_FLUSH = 64 };

// One candidate tile: rows r0 .. r0+255 of the B operand, of which the rows
// in the searched windows are valid (bit c of mask = row r0 + c).  Windows of
// several adjacent cells share a tile when they lie within 256 rows of each
// other (the adjacent cells of a query cell come in ascending position order).
struct alignas(16) TileDesc {
    uint32_t item, tile, flags, aseq;   // aseq: the producer's item sequence number (A buffer aseq & 1)
    uint32_t qbeg, qlen, qa, r0;
    uint32_t p2, p3, pad2, pad3;
    uint32_t mask[8];
};

struct TcShared {
    uint64_t full_b[8], empty_b[8];
    uint64_t full_a[2], empty_a[2];
    // tmem_full: two arrivals per use, the MMA issuer's once the tile's
    // descriptor is written (release) and its commit once the MMAs land
    uint64_t tmem_full[2], tmem_empty[2];
    uint64_t epi_bar[2];
    uint64_t fin[2];         // per MMA issuer: its last commit has landed
    // the descriptor of a stage's current turn: the MMA issuer copies it
    // before the stage is released (by the MMA's commit, or a marker's
    // arrival), so the producer rewrites it only after the stage is free
    TileDesc ring[TC_MAXS];
    TileDesc tdesc[2];
    uint32_t tmem_base;
    uint32_t abort;
    uint32_t flush_req;   // staging passed its soft limit: commit at the next flagged turn
    uint32_t half;
    uint32_t cnt[2];
    uint32_t ok;
    uint32_t pad;
    unsigned long long base;
    uint32_t sq[8][TC_SQ];   // per epilogue warp: survivors waiting for the FP64 recheck
    uint32_t sc[8][TC_SQ];
    // direct form: per epilogue warp, a ring of survivors (query position,
    // candidate position, job) that the recheck warp takes; one writer, one
    // reader, positions counted from 0 (tail: written, head: taken)
    uint32_t rq_q[8][TC_RQ], rq_c[8][TC_RQ], rq_j[8][TC_RQ];
    uint32_t rq_tail[8], rq_head[8];
    uint32_t epi_done;       // epilogue warps that finished
    unsigned long long surv;     // survivors (statistics)
    unsigned long long counted;  // pairs counted (count-only launches)
    long long t_item;            // tuning launches: clock of the last item end
    long long t_start;           // clock at the CTA's start
    long long win[32][2];        // producer: one batch of SORTIDU windows [start, end)
};

struct TcLaunch {
    JoinLaunch J;
    const TcJob *jobs;           // many-jobs launch: per-job parameters (else nullptr)
    unsigned long long *jpos;    // many-jobs launch: per-job pair counters
    unsigned long long *job_cycles;   // many-jobs tuning launch: per-job SM cycles (else nullptr)
    const unsigned char *XA;
    const unsigned char *XB;
    const double *XR;            // entries row by row for the recheck (nullptr: from X)
    int dr;                      // XR's row stride in doubles
    int Kp;
    int NS;
    int Tbits;
    uint32_t a_bytes, b_bytes;
    uint32_t off_b, off_s;
    unsigned long long limit_ns;   // every bounded wait of the launch gives up after this
};

__device__ __forceinline__ int64_t tc_lower_u(const double *__restrict__ U, int64_t lo, int64_t hi, double ref,
                                              double ew)
{
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (U[mid] - ref < -ew)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int64_t tc_upper_u(const double *__restrict__ U, int64_t lo, int64_t hi, double ref,
                                              double ew)
{
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (U[mid] - ref <= ew)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Exact test of one surviving candidate: the plain path's FP64 SHORTC sum in
// REORDER order (same operations in the same order, so the same decision).
// Coordinates are fetched 16 dimensions at a time with independent loads, so
// a recheck costs about d/16 memory round trips instead of d.  The query
// comes from Xq (the entries themselves in a self-join, the query array in
// Q join_eps E), the candidate from the entries X.  With XR (the entries row
// by row, row stride dr a multiple of 4) the candidate's 16 coordinates are
// 128 contiguous bytes, four 32-byte sectors where the structure-of-arrays
// layout touches sixteen; in a self-join (qrows) the query is read there too.
__device__ __forceinline__ bool tc_exact(const double *__restrict__ Xq, int64_t qnpad,
                                         const double *__restrict__ X, int64_t npad,
                                         const double *__restrict__ XR, int dr, bool qrows,
                                         int d, long long e2bits, uint32_t qpos, uint32_t cpos)
{
    double s = 0.0;
    for (int j0 = 0; j0 < d; j0 += 16) {
        double a[16], b[16];
        if (XR) {
            // (a row holds dr >= d values, d rounded up to 4: each pair is in it)
            const double2 *rb = reinterpret_cast<const double2 *>(XR + (int64_t)cpos * dr + j0);
            const double2 *ra = reinterpret_cast<const double2 *>(XR + (int64_t)qpos * dr + j0);
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                if (j0 + 2 * t < d) {
                    const double2 vb = __ldg(rb + t);
                    b[2 * t] = vb.x;
                    b[2 * t + 1] = vb.y;
                    if (qrows) {
                        const double2 va = __ldg(ra + t);
                        a[2 * t] = va.x;
                        a[2 * t + 1] = va.y;
                    } else {
                        a[2 * t] = Xq[(int64_t)(j0 + 2 * t) * qnpad + qpos];
                        a[2 * t + 1] = Xq[(int64_t)min(j0 + 2 * t + 1, d - 1) * qnpad + qpos];
                    }
                }
            }
        } else {
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                if (j0 + t < d) {
                    a[t] = Xq[(int64_t)(j0 + t) * qnpad + qpos];
                    b[t] = X[(int64_t)(j0 + t) * npad + cpos];
                }
            }
        }
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            if (j0 + t < d) {
                const double dd = a[t] - b[t];
                s = __fma_rn(dd, dd, s);
                if (__double_as_longlong(s) > e2bits)
                    return false;
            }
        }
    }
    return true;
}

// Recheck the warp's queued survivors (one per lane per round) and emit the
// exact pairs into the staging half (or count them).  Called by all 32 lanes.
// A self-join emits both orientations of a pair (one for i = j); Q join_eps E
// (asym) emits (query, entry) once.
template <bool ASYM>
__device__ __noinline__ void tc_flush_survivors(const TcLaunch *__restrict__ T, const uint32_t *sq,
                                                const uint32_t *sc, uint32_t n, gj_pair *stg, uint32_t *cnt,
                                                uint32_t *flush_req, unsigned long long *counted, uint32_t job,
                                                unsigned long long *dpos = nullptr)
{
    const int lane = threadIdx.x & 31;
    const double *__restrict__ X = T->J.ix.X;
    const int64_t npad = T->J.ix.npad;
    const double *__restrict__ Xq = ASYM ? T->J.ix.XQ : X;
    const int64_t qnpad = ASYM ? T->J.ix.qnpad : npad;
    const uint32_t *__restrict__ qorig = ASYM ? T->J.ix.qorig : T->J.ix.orig;
    const TcJob *jp = T->jobs ? &T->jobs[job] : nullptr;
    const long long e2bits = __double_as_longlong(jp ? jp->e2 : T->J.ix.e2);
    // a job's dimensions past its own d are zero in the combined layout and
    // add exactly 0: the job's d suffices
    const int d = jp ? jp->d : T->J.ix.d;
    for (uint32_t base = 0; base < n; base += 32) {
        const uint32_t i = base + lane;
        bool keep = false;
        uint32_t qpos = 0, cpos = 0;
        if (i < n) {
            qpos = sq[i];
            cpos = sc[i];
            keep = tc_exact(Xq, qnpad, X, npad, jp ? nullptr : T->XR, T->dr, !ASYM, d, e2bits, qpos, cpos);
        }
        const uint32_t np = keep ? ((!ASYM && qpos != cpos) ? 2u : 1u) : 0u;
        if (stg == nullptr && jp == nullptr && dpos == nullptr) {
            *counted += np;
            continue;
        }
        uint32_t incl = np;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o)
                incl += y;
        }
        const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
        if (jp) {
            // many-jobs launch: straight into the job's buffer (pairs past its
            // capacity are counted, not written)
            unsigned long long o64 = 0;
            if (lane == 0 && tot)
                o64 = atomicAdd(&T->jpos[job], (unsigned long long)tot);
            o64 = __shfl_sync(0xffffffffu, o64, 0) + incl - np;
            if (np && jp->out) {
                const uint32_t a = T->J.ix.orig[qpos], b = T->J.ix.orig[cpos];
                if (o64 < jp->cap)
                    jp->out[o64] = gj_pair{a, b};
                if (np == 2 && o64 + 1 < jp->cap)
                    jp->out[o64 + 1] = gj_pair{b, a};
            }
            continue;
        }
        if (dpos) {
            // direct output: one reservation per warp; pairs past the
            // capacity are counted (the reservation), not written
            unsigned long long o64 = 0;
            if (lane == 0 && tot)
                o64 = atomicAdd(dpos, (unsigned long long)tot);
            o64 = __shfl_sync(0xffffffffu, o64, 0) + incl - np;
            if (np) {
                const uint32_t a = qorig[qpos], b = T->J.ix.orig[cpos];
                if (o64 < T->J.cap)
                    T->J.out[o64] = gj_pair{a, b};
                if (np == 2 && o64 + 1 < T->J.cap)
                    T->J.out[o64 + 1] = gj_pair{b, a};
            }
            continue;
        }
        uint32_t off = 0;
        if (lane == 0 && tot)
            off = atomicAdd(cnt, tot);
        off = __shfl_sync(0xffffffffu, off, 0) + incl - np;
        if (tot) {
            // soft limit: room for three more tiles of worst-case output (written
            // before the accumulator is released) plus the small post-release
            // output of up to four turns
            if (off + np > TC_STG - 3u * 2u * 128u * 256u - 4096u)
                *(volatile uint32_t *)flush_req = 1u;
            if (off + np > TC_STG) {
                atomicOr(&T->J.ctl->err, kErrStaging);
            } else if (np) {
                const uint32_t a = T->J.ix.orig[qpos], b = T->J.ix.orig[cpos];
                stg[off] = gj_pair{a, b};
                if (np == 2)
                    stg[off + 1] = gj_pair{b, a};
            }
        }
    }
}

// Bit i of the result: v[i] <= T (this lane's row against column i of a chunk).
__device__ __forceinline__ uint32_t hit_mask32(const uint32_t (&v)[32], float Tf)
{
    uint32_t m = 0;
#pragma unroll
    for (int i = 0; i < 32; ++i)
        m |= (__uint_as_float(v[i]) <= Tf ? 1u : 0u) << i;
    return m;
}

// Rare path of the epilogue, run after the accumulator is released: queue the
// valid survivors marked in each lane's hit mask (warp-aggregated), flushing
// the queue through the FP64 recheck when it would overflow.  Returns the new
// queue length.
template <bool ASYM>
__device__ __forceinline__ uint32_t tc_queue_bits(const TcLaunch *__restrict__ T, uint32_t mask, uint32_t col0,
                                               uint32_t qpos, uint32_t r0,
                                               uint32_t *sq, uint32_t *sc, uint32_t nq, gj_pair *stg, uint32_t *cnt,
                                               uint32_t *flush_req, uint32_t &surv,
                                               unsigned long long *counted_sh, uint32_t job,
                                               unsigned long long *dpos = nullptr)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t found = 0;
    for (;;) {
        const bool have = mask != 0u;
        if (!__any_sync(0xffffffffu, have))
            break;
        const uint32_t cpos = r0 + col0 + (have ? (uint32_t)(__ffs(mask) - 1) : 0u);
        mask &= mask - 1u;
        // the mask holds valid rows only; in a self-join j >= i keeps one
        // orientation (rows of the other searched cells all lie after the
        // query cell); Q join_eps E keeps every marked candidate
        const bool h = have && (ASYM || cpos >= qpos);
        const unsigned bal = __ballot_sync(0xffffffffu, h);
        if (!bal)
            continue;
        const uint32_t k = (uint32_t)__popc(bal);
        if (nq + k > (uint32_t)TC_SQ) {
            unsigned long long c = 0;
            __syncwarp();
            tc_flush_survivors<ASYM>(T, sq, sc, nq, stg, cnt, flush_req, &c, job, dpos);
            __syncwarp();
            if (c)
                atomicAdd(counted_sh, c);   // each lane counted its own pairs
            nq = 0;
        }
        if (h) {
            const uint32_t at = nq + (uint32_t)__popc(bal & lt);
            sq[at] = qpos;
            sc[at] = cpos;
        }
        nq += k;
        found += k;
    }
    if (lane == 0)
        surv += found;   // (summed into the launch statistics once, at the warp's exit)
    return nq;
}

// DIRECT = false: output through per-CTA staging committed per work item
// (exact resume; result batches for host output).  DIRECT = true: pairs go
// straight to the output (or a many-jobs launch's job buffers) with one
// reservation per warp, so the epilogue warps never agree on anything: each
// reads its share of every tile and moves on.
template <bool DIRECT, bool ASYM>
__global__ void __launch_bounds__(TC_THREADS, 1) k_join_tc(const TcLaunch T)
{
    static_assert(DIRECT || !ASYM, "Q join_eps E runs in the direct form");
    extern __shared__ __align__(1024) unsigned char smem[];
    TcShared &S = *reinterpret_cast<TcShared *>(smem + T.off_s);
    unsigned char *Abuf = smem;
    unsigned char *Bbuf = smem + T.off_b;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const JoinLaunch &L = T.J;
    const int NS = T.NS;
    const bool count_only = (L.out == nullptr);

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&S.full_b[s], 1);
            mbar_init(&S.empty_b[s], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&S.full_a[i], 1);
            mbar_init(&S.empty_a[i], 2);   // both MMA issuers commit at the item's end
            mbar_init(&S.tmem_full[i], 2);
            mbar_init(&S.tmem_empty[i], 8);   // the eight epilogue warps read every accumulator
            mbar_init(&S.epi_bar[i], 8);
            mbar_init(&S.fin[i], 1);
        }
        S.abort = 0;
        S.flush_req = 0;
        for (int w = 0; w < 8; ++w)
            S.rq_tail[w] = S.rq_head[w] = 0;
        S.epi_done = 0;
        S.half = 0;
        S.cnt[0] = S.cnt[1] = 0;
        S.surv = 0;
        S.counted = 0;
        S.t_start = (long long)globaltimer();
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(&S.tmem_base, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem_base;
    volatile uint32_t *abort = &S.abort;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        uint32_t seq = 0, nitem = 0;
        bool dead = false;
        unsigned long long slots = 0;   // candidate pairs of the pushed tiles (lane 0)
        auto push = [&](const TileDesc &D, bool tile) -> bool {   // lane 0 only
            const uint32_t stage = seq % (uint32_t)NS;
            if (!mbar_wait(&S.empty_b[stage], ((seq / NS) & 1u) ^ 1u, abort, T.limit_ns))
                return false;
            S.ring[stage] = D;
            if (tile) {
                mbar_arrive_expect_tx(&S.full_b[stage], T.b_bytes);
                bulk_g2s(Bbuf + (size_t)stage * T.b_bytes, T.XB + (size_t)D.r0 * T.Kp * 2, T.b_bytes,
                         &S.full_b[stage]);
            } else {
                mbar_arrive(&S.full_b[stage]);
            }
            ++seq;
            return true;
        };
        for (;;) {
            uint32_t item = 0xffffffffu, resume = 0;
            if (lane == 0) {
                if (count_only || !*(volatile unsigned int *)&L.ctl->full) {
                    uint32_t t = (L.n_din > 0) ? atomicAdd(&L.ctl->din_head, 1u) : 0xffffffffu;
                    if (t < L.n_din) {
                        item = L.din[t].item;
                        resume = L.din[t].tile;
                    } else {
                        uint32_t hq = atomicAdd(&L.ctl->head, 1u);
                        if (hq < L.qlimit)
                            item = L.queue[hq];
                    }
                }
            }
            item = __shfl_sync(0xffffffffu, item, 0);
            resume = __shfl_sync(0xffffffffu, resume, 0);
            if (item == 0xffffffffu || *abort)
                break;
            const Item it = L.ix.items[item];
            const uint32_t qa = it.qbeg & ~7u;
            const uint32_t aseq = nitem;
            const uint32_t abuf = nitem & 1u;
            if (lane == 0) {
                if (!mbar_wait(&S.empty_a[abuf], ((nitem >> 1) & 1u) ^ 1u, abort, T.limit_ns)) {
                    dead = true;
                } else {
                    mbar_arrive_expect_tx(&S.full_a[abuf], T.a_bytes);
                    bulk_g2s(Abuf + (size_t)abuf * T.a_bytes, T.XA + (size_t)qa * T.Kp * 2, T.a_bytes,
                             &S.full_a[abuf]);
                }
            }
            dead = __shfl_sync(0xffffffffu, dead, 0);
            if (dead)
                break;
            ++nitem;
            // Q join_eps E: the item's cell is a query cell (its adjacency lists
            // every adjacent entry cell; no own-cell window)
            const bool asym = ASYM;
            const int64_t cell_end = asym ? 0 : L.ix.cell_start[it.cell + 1];
            const int64_t nb_begin = L.ix.adj_start[it.cell], nb_end = L.ix.adj_start[it.cell + 1];
            const uint32_t job = T.jobs ? it.pad : 0u;
            const int u = T.jobs ? T.jobs[job].u : L.ix.u;
            const double ew = T.jobs ? T.jobs[job].ew : L.ix.ew;
            const uint32_t jtb = T.jobs ? (uint32_t)T.jobs[job].Tbits : (uint32_t)T.Tbits;
            double ulo = 0.0, uhi = 0.0;
            if (u >= 0) {
                const double *Uq = asym ? L.ix.XQ + (int64_t)u * L.ix.qnpad : L.ix.X + (int64_t)u * L.ix.npad;
                ulo = Uq[it.qbeg];
                uhi = Uq[it.qbeg + it.qlen - 1];
            }
            // Tile packing runs in lane 0 alone: the open tile [cr0, cr0 + TC_N),
            // its valid-row mask cm, the tile waiting to be pushed (pend) and
            // the flags live in lane 0's registers; the other lanes only compute
            // the windows and take part in the broadcasts once per batch.
            uint32_t tile_idx = 0;
            bool have = false, first = true, trunc = false;
            TileDesc pend{};
            bool open = false;
            uint32_t cr0 = 0;
            uint32_t cm[8];
            auto close_tile = [&](bool full) {   // lane 0 only
                if (!open)
                    return;
                open = false;
                if (tile_idx >= resume) {
                    // another CTA filled the output: stop (polled every 128 tiles;
                    // tiles made meanwhile are discarded by the failed commit)
                    if (!count_only && (tile_idx & 127u) == 0 && *(volatile unsigned int *)&L.ctl->full) {
                        trunc = true;
                    } else {
                        if (have) {
                            if (first)
                                pend.flags |= F_FIRST;
                            first = false;
                            if (!push(pend, true))
                                dead = true;
                        }
                        pend = TileDesc{item, tile_idx, 0u, aseq, it.qbeg, it.qlen, qa, cr0, job, jtb, 0u, 0u};
                        uint32_t nv = 0;
                        if (full) {
#pragma unroll
                            for (int w = 0; w < 8; ++w)
                                pend.mask[w] = 0xffffffffu;
                            nv = TC_N;
                        } else {
#pragma unroll
                            for (int w = 0; w < 8; ++w) {
                                pend.mask[w] = cm[w];
                                nv += __popc(cm[w]);
                            }
                        }
                        slots += (unsigned long long)it.qlen * nv;
                        have = true;
                    }
                }
                ++tile_idx;
            };
            // Pack rows [s0, e0) of one window into partial tiles.  Returns e0,
            // or the start of a run of whole tiles (no tile open, s0 a multiple
            // of 8, at least TC_N rows left), which the warp pushes together.
            auto pack_window = [&](int64_t s0, const int64_t e0) -> int64_t {   // lane 0 only
                while (s0 < e0 && !trunc && !dead) {
                    if (!open && (s0 & 7) == 0 && e0 - s0 >= TC_N)
                        return s0;
                    // (windows come in ascending order; one that does not
                    // starts a tile of its own)
                    if (open && (s0 >= (int64_t)cr0 + TC_N || s0 < (int64_t)cr0))
                        close_tile(false);
                    if (trunc || dead)
                        return e0;
                    if (!open) {
                        open = true;
                        cr0 = (uint32_t)(s0 & ~(int64_t)7);
#pragma unroll
                        for (int w = 0; w < 8; ++w)
                            cm[w] = 0u;
                    }
                    const int64_t hi = min(e0, (int64_t)cr0 + TC_N);
                    // rows [s0, hi) of the tile are valid
                    const int lo_r = (int)(s0 - cr0), hi_r = (int)(hi - cr0);
#pragma unroll
                    for (int w = 0; w < 8; ++w) {
                        const int a = max(lo_r - 32 * w, 0), b = min(hi_r - 32 * w, 32);
                        if (a < b)
                            cm[w] |= (b >= 32 ? 0xffffffffu : ((1u << b) - 1u)) & ~((1u << a) - 1u);
                    }
                    s0 = hi;
                    if (s0 < e0)
                        close_tile(false);   // the window runs on past this tile
                }
                return e0;
            };
            // A run of F whole tiles from row s0 (every row valid), warp-wide:
            // the pending tile goes first (lane 0), then the run's tiles but
            // its last, one per lane, in batches of at most NS turns (distinct
            // stages: no lane waits for a phase another lane's turn must pass);
            // the run's last tile becomes the pending one (its end flags are
            // known only when the item ends).
            auto push_run = [&](const int64_t r_s0, const uint32_t F) {
                const uint32_t ti0 = __shfl_sync(0xffffffffu, tile_idx, 0);
                const uint32_t skip = resume > ti0 ? min(F, resume - ti0) : 0u;   // tiles already committed
                if (lane == 0) {
                    tile_idx = ti0 + F;
                    // another CTA filled the output: stop (tiles made meanwhile
                    // are discarded by the failed commit)
                    if (!count_only && *(volatile unsigned int *)&L.ctl->full)
                        trunc = true;
                    else if (skip < F && have) {
                        if (first)
                            pend.flags |= F_FIRST;
                        first = false;
                        if (!push(pend, true))
                            dead = true;
                        have = false;
                    }
                }
                if (__shfl_sync(0xffffffffu, (trunc || dead) ? 1 : 0, 0) || skip == F)
                    return;
                const uint32_t sq0 = __shfl_sync(0xffffffffu, seq, 0);
                const bool fs = __shfl_sync(0xffffffffu, first ? 1 : 0, 0) != 0;
                const uint32_t m = F - skip - 1;   // pushed now
                // lane L pushes the run's tiles L, L + NS, ... : turns of one
                // stage, each as soon as the stage is free (a non-blocking
                // test per round, so the warp stays converged)
                bool bad = false;
                uint32_t kk = (uint32_t)lane;
                const uint32_t st = (sq0 + (uint32_t)lane) % (uint32_t)NS;
                const uint64_t t_start = globaltimer();
                uint32_t rounds = 0;
                while (__any_sync(0xffffffffu, kk < m && lane < NS)) {
                    if (kk < m && lane < NS) {
                        const uint32_t t = sq0 + kk;
                        if (mbar_test(&S.empty_b[st], ((t / NS) & 1u) ^ 1u)) {
                            const uint32_t i = skip + kk;
                            const uint32_t r0 = (uint32_t)r_s0 + i * (uint32_t)TC_N;
                            uint4 *dst = reinterpret_cast<uint4 *>(&S.ring[st]);
                            dst[0] = make_uint4(item, ti0 + i, (fs && kk == 0) ? F_FIRST : 0u, aseq);
                            dst[1] = make_uint4(it.qbeg, it.qlen, qa, r0);
                            dst[2] = make_uint4(job, jtb, 0u, 0u);
                            dst[3] = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
                            dst[4] = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
                            mbar_arrive_expect_tx(&S.full_b[st], T.b_bytes);
                            bulk_g2s(Bbuf + (size_t)st * T.b_bytes, T.XB + (size_t)r0 * T.Kp * 2, T.b_bytes,
                                     &S.full_b[st]);
                            kk += (uint32_t)NS;
                        }
                    }
                    // bounded like every other wait: the clock and the abort
                    // flag are read every 256 rounds
                    // (the warp leaves the loop together: the loop head is a vote)
                    if ((++rounds & 255u) == 0 &&
                        __any_sync(0xffffffffu, *abort || globaltimer() - t_start > T.limit_ns)) {
                        bad = true;
                        break;
                    }
                }
                bad = __any_sync(0xffffffffu, bad);
                if (lane == 0) {
                    if (bad)
                        dead = true;
                    seq = sq0 + m;
                    if (m)
                        first = false;
                    pend = TileDesc{item, ti0 + F - 1, 0u, aseq, it.qbeg, it.qlen, qa,
                                    (uint32_t)r_s0 + (F - 1) * (uint32_t)TC_N, job, jtb, 0u, 0u};
#pragma unroll
                    for (int w = 0; w < 8; ++w)
                        pend.mask[w] = 0xffffffffu;
                    have = true;
                    slots += (unsigned long long)it.qlen * TC_N * (m + 1);
                }
            };
            for (int64_t nb0 = nb_begin; nb0 < nb_end; nb0 += 32) {
                int64_t ws = 0, we = 0;
                if (nb0 + lane < nb_end) {
                    const uint32_t b = L.ix.adj[nb0 + lane];
                    if (!asym && b == it.cell) {
                        ws = it.qbeg;
                        we = cell_end;
                    } else {
                        ws = L.ix.cell_start[b];
                        we = L.ix.cell_start[b + 1];
                    }
                    if (u >= 0) {
                        const double *U = L.ix.X + (int64_t)u * L.ix.npad;
                        ws = tc_lower_u(U, ws, we, ulo, ew);
                        we = tc_upper_u(U, ws, we, uhi, ew);
                    }
                }
                S.win[lane][0] = ws;
                S.win[lane][1] = we;
                __syncwarp();
                const int nw = (int)min((int64_t)32, nb_end - nb0);
                for (int w = 0; w < nw; ++w) {
                    const int64_t e0 = S.win[w][1];
                    int64_t s0 = S.win[w][0];
                    for (;;) {
                        int64_t stop = e0;
                        if (lane == 0)
                            stop = pack_window(s0, e0);
                        stop = __shfl_sync(0xffffffffu, stop, 0);
                        trunc = __shfl_sync(0xffffffffu, trunc, 0);
                        dead = __shfl_sync(0xffffffffu, dead, 0);
                        if (trunc || dead || stop >= e0)
                            break;
                        const uint32_t F = (uint32_t)((e0 - stop) / TC_N);
                        push_run(stop, F);
                        trunc = __shfl_sync(0xffffffffu, trunc, 0);
                        dead = __shfl_sync(0xffffffffu, dead, 0);
                        if (trunc || dead)
                            break;
                        s0 = stop + (int64_t)F * TC_N;
                        if (s0 >= e0)
                            break;
                    }
                    if (trunc || dead)
                        break;
                }
                __syncwarp();
                if (trunc || dead)
                    break;
            }
            if (lane == 0 && !trunc && !dead)
                close_tile(false);
            if (lane == 0 && !dead) {
                const bool single = first;   // no turn pushed yet: the item ends with its only turn
                if (have && !trunc) {
                    pend.flags |= F_LAST | (first ? F_FIRST : 0u);
                    if (!push(pend, true))
                        dead = true;
                } else {
                    TileDesc M{item, first ? resume : 0u, F_MARKER | F_LAST | (first ? F_FIRST : 0u) |
                                                         (trunc ? F_TRUNC : 0u),
                               aseq, it.qbeg, it.qlen, qa, 0u, job, jtb, 0u, 0u};
                    if (!push(M, false))
                        dead = true;
                }
                if (single && !dead) {
                    TileDesc P{item, 0u, F_MARKER | F_PAD, aseq, it.qbeg, it.qlen, qa, 0u, job, jtb, 0u, 0u};
                    if (!push(P, false))
                        dead = true;
                }
            }
            dead = __shfl_sync(0xffffffffu, dead, 0);
            trunc = __shfl_sync(0xffffffffu, trunc, 0);
            if (trunc || dead)
                break;
        }
        if (lane == 0) {
            // one terminator per accumulator parity: each MMA issuer, and in
            // the direct form each epilogue group, stops at its own
            for (int t = 0; t < 2 && !dead; ++t) {
                TileDesc Tm{};
                Tm.flags = F_TERM;
                Tm.aseq = nitem;   // every item before this one is finished
                if (!push(Tm, false))
                    dead = true;
            }
            if (dead) {
                S.abort = 1;
                atomicOr(&L.ctl->err, kErrTimeout);
            }
            if (slots)
                atomicAdd(&L.ctl->evaluated, slots);
        }
        __syncwarp();
    } else if (warp == 1 || warp == 10) {
        // ------------------------------------------------------------ MMA issuers
        // Two issuing threads, one per accumulator: issuer j takes the turns
        // of parity j.  A thread waiting on a barrier or committing stalls its
        // own MMA stream, so with one issuer the tensor core idled for every
        // wait, fence and commit; with two, one issuer's bookkeeping overlaps
        // the other's MMAs.  Each issuer reads its own turns only (another
        // parity's stage barrier may already be a phase or more ahead).  An A
        // buffer is reused only after both issuers released it: when issuer
        // j's turn belongs to item a (the producer's item sequence number), j
        // has issued every MMA it will issue on items < a and commits their
        // release (the empty barrier counts 2 arrivals per item).  Every item
        // has a turn of each parity (the producer pads single-turn items), so
        // neither issuer holds a buffer the producer waits for.
        if (lane == 0) {
            const uint32_t j = (warp == 1) ? 0u : 1u;
            const uint32_t idesc = idesc_f16_f32(128, TC_N);
            const uint32_t lbo = 128, sbo = (uint32_t)T.Kp * 16;
            const uint32_t a0 = smem_addr(Abuf), b0 = smem_addr(Bbuf);
            const int ksteps = T.Kp / 16;
            // descriptors of buffer 0 / stage 0; an operand at byte offset o adds
            // o >> 4 to the start-address field (shared addresses stay < 2^18)
            const uint64_t adesc0 = desc_kmajor(a0, lbo, sbo), bdesc0 = desc_kmajor(b0, lbo, sbo);
            uint32_t a_seen = 0xffffffffu;   // item whose A load this thread has seen land
            uint32_t next_rel = 0;           // first item this thread has not released
            bool dead = false;
            // the A tile of item a has landed (its buffer is not reloaded before
            // this thread released it, so the parity cannot alias)
            auto wait_a = [&](uint32_t a) -> bool {
                if (a_seen == a)
                    return true;
                if (!mbar_wait(&S.full_a[a & 1u], (a >> 1) & 1u, abort, T.limit_ns))
                    return false;
                a_seen = a;
                return true;
            };
            for (uint32_t seq = j;; seq += 2) {
                const uint32_t stage = seq % (uint32_t)NS;
                if (!mbar_wait(&S.full_b[stage], (seq / NS) & 1u, abort, T.limit_ns)) {
                    dead = true;
                    break;
                }
                const TileDesc *R = &S.ring[stage];
                const uint32_t flags = R->flags;
                const uint32_t aseq = R->aseq;
                // release the A buffers of the items before this turn's (at a
                // terminator no item follows: only wait for their loads)
                while (next_rel < aseq) {
                    // (an item whose turns here were markers issued no MMA that
                    // waited for its load: wait before releasing the buffer)
                    if (!wait_a(next_rel)) {
                        dead = true;
                        break;
                    }
                    if (!(flags & F_TERM))
                        mma_commit(&S.empty_a[next_rel & 1u]);
                    ++next_rel;
                }
                if (dead)
                    break;
                const uint32_t acc = j, use = seq >> 1;   // this accumulator's use count
                if (!mbar_wait(&S.tmem_empty[acc], (use & 1u) ^ 1u, abort, T.limit_ns)) {
                    dead = true;
                    break;
                }
                TileDesc Dm = *R;
                if (*(volatile uint32_t *)&S.flush_req)
                    Dm.flags |= F_FLUSH;
                S.tdesc[acc] = Dm;
                if (!(flags & (F_MARKER | F_TERM))) {
                    if (!wait_a(aseq)) {
                        dead = true;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t ad = adesc0 + (((aseq & 1u) * T.a_bytes) >> 4);
                    const uint64_t bd = bdesc0 + ((stage * T.b_bytes) >> 4);
                    const uint32_t dcol = tmem + acc * 256u;
                    mma_f16(dcol, ad, bd, idesc, 0u);
                    for (int ks = 1; ks < ksteps; ++ks)
                        mma_f16(dcol, ad + (uint64_t)(ks * 16), bd + (uint64_t)(ks * 16), idesc, 1u);
                    mma_commit(&S.empty_b[stage]);
                    mbar_arrive(&S.tmem_full[acc]);   // the descriptor
                    mma_commit(&S.tmem_full[acc]);    // the accumulator
                } else {
                    mbar_arrive(&S.empty_b[stage]);
                    mbar_arrive(&S.tmem_full[acc]);
                    mbar_arrive(&S.tmem_full[acc]);
                }
                if (flags & F_TERM)
                    break;
            }
            // A commit's arrival lands asynchronously, after the MMAs before it
            // complete; one still in flight when the CTA exits could land in
            // the shared memory of the next CTA on this SM.  Commit once more
            // and wait: the earlier arrivals of this thread have then landed.
            if (!dead) {
                mma_commit(&S.fin[j]);
                if (!mbar_wait(&S.fin[j], 0u, abort, T.limit_ns))
                    dead = true;
            }
            if (dead) {
                S.abort = 1;
                atomicOr(&L.ctl->err, kErrTimeout);
            }
        }
        __syncwarp();
    } else if (warp == 11) {
        // ------------------------------------------------------------ recheck (direct form)
        // Takes the survivors the epilogue warps queue in their rings, 32 at a
        // time, runs the exact FP64 test and emits the pairs: the epilogue
        // warps go back to the accumulators without waiting for memory.  A
        // warp whose ring is full (dense data) rechecks its survivors itself.
        if constexpr (DIRECT) {
            unsigned long long *const dpos = (!T.jobs && !count_only) ? &L.ctl->pos : nullptr;
            uint32_t head[8];
#pragma unroll
            for (int w = 0; w < 8; ++w)
                head[w] = 0;
            unsigned long long counted = 0;
            bool last = false;
            for (;;) {
                // every epilogue warp done: one more pass takes what is left
                if (!last && *(volatile uint32_t *)&S.epi_done == 8u) {
                    __threadfence_block();
                    last = true;
                }
                bool worked = false;
#pragma unroll
                for (int w = 0; w < 8; ++w) {
                    const uint32_t tail = *(volatile uint32_t *)&S.rq_tail[w];
                    __threadfence_block();
                    while (head[w] != tail) {
                        const uint32_t pos = head[w] & (uint32_t)(TC_RQ - 1);
                        uint32_t n = min(min(tail - head[w], (uint32_t)TC_RQ - pos), 32u);
                        // a run of one job (a many-jobs launch mixes them)
                        const uint32_t j0 = S.rq_j[w][pos];
                        const unsigned same = __ballot_sync(0xffffffffu, (uint32_t)lane < n && S.rq_j[w][pos + lane] == j0);
                        n = (same == 0xffffffffu) ? 32u : (uint32_t)(__ffs(~same) - 1);
                        unsigned long long c = 0;
                        tc_flush_survivors<ASYM>(&T, &S.rq_q[w][pos], &S.rq_c[w][pos], n, nullptr, nullptr, nullptr,
                                                 &c, j0, dpos);
                        counted += c;
                        head[w] += n;
                        __syncwarp();
                        if (lane == 0)
                            *(volatile uint32_t *)&S.rq_head[w] = head[w];
                        __syncwarp();
                        worked = true;
                    }
                }
                if (last)
                    break;
                if (!worked) {
                    if (*abort)
                        break;
                    __nanosleep(2000);   // a ring fills in ~100 us of sparse data
                }
            }
            for (int o = 16; o; o >>= 1)
                counted += __shfl_xor_sync(0xffffffffu, counted, o);
            if (lane == 0 && counted)
                atomicAdd(&S.counted, counted);
        }
    } else if constexpr (DIRECT) {
        // ------------------------------------------------------------ epilogue (direct output)
        // All eight warps take every turn: warp e reads its 32 rows (TMEM
        // lane quadrant q) in the column half hh of the turn's accumulator,
        // two rounds of two 32-column loads, so a tile is read in half the
        // time one warp per quadrant would take; meanwhile the other
        // accumulator is refilled.  The warps never agree on anything: each
        // releases its share of the accumulator and queues its own hits.
        const int e = warp - 2, q = warp & 3, hh = e >> 2;
        uint32_t *const sq = S.sq[e], *const sc = S.sc[e];
        uint32_t nq = 0;
        const float Tf0 = __int_as_float(T.Tbits);
        uint32_t cur_aseq = 0xffffffffu;     // item whose values are cached
        uint32_t it_qpos = 0;                // this lane's query row
        uint32_t it_job = 0xffffffffu;       // the job of the queued survivors (none yet)
        bool it_rvalid = false;
        float it_Tf = Tf0;
        unsigned long long *const dpos = (!T.jobs && !count_only) ? &L.ctl->pos : nullptr;
        unsigned long long counted = 0;
        uint32_t surv_w = 0;                 // survivors this warp found (lane 0)
        uint32_t rq_tail = 0;                // this warp's ring: positions written
        bool dead = false;
        long long t_job = clock64();
        const bool lead = e == 0 && lane == 0;   // one lane of the epilogue (tuning launches)
        auto flush = [&]() {
            unsigned long long c = 0;
            __syncwarp();
            tc_flush_survivors<ASYM>(&T, sq, sc, nq, nullptr, nullptr, nullptr, &c, it_job, dpos);
            __syncwarp();
            counted += c;
            nq = 0;
        };
        for (uint32_t turn = 0;; ++turn) {
            const uint32_t acc = turn & 1u, par = (turn >> 1) & 1u;
            const bool ok = mbar_wait(&S.tmem_full[acc], par, abort, T.limit_ns);
            // one decision per warp: the TMEM loads below need all 32 lanes
            if (__any_sync(0xffffffffu, !ok)) {
                dead = true;
                break;
            }
            tc_fence_after();
            const TileDesc *Dp = &S.tdesc[acc];
            const uint32_t flags = Dp->flags;
            if (flags & F_TERM)
                break;
            const uint32_t aseq = Dp->aseq;
            uint32_t new_job = it_job;
            if (aseq != cur_aseq) {
                // per-item values (the same in every descriptor of the item)
                cur_aseq = aseq;
                const uint32_t qa = Dp->qa, qb = Dp->qbeg, ql = Dp->qlen;
                it_qpos = qa + (uint32_t)(q * 32 + lane);
                it_rvalid = it_qpos >= qb && it_qpos < qb + ql;
                new_job = Dp->p2;
                it_Tf = T.jobs ? __uint_as_float(Dp->p3) : Tf0;
            }
            uint32_t hm[4];   // this lane's hits in the 4 chunks of its column half
#pragma unroll
            for (int c = 0; c < 4; ++c)
                hm[c] = 0u;
            bool anyhit = false;
            uint32_t r0 = 0;
            const uint32_t cb = (uint32_t)hh * 128u;
            if (!(flags & F_MARKER)) {
                const float Tf = it_Tf;
                const bool rvalid = it_rvalid;
                const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + acc * 256u + cb;
#pragma unroll
                for (int rd = 0; rd < 2; ++rd) {
                    uint32_t va[32], vb[32];
                    float ma, mb;
                    tmem_ld32_min(tb + rd * 64u, va, ma);
                    tmem_ld32_min(tb + rd * 64u + 32u, vb, mb);
                    tmem_wait_ld();
                    const bool ha = rvalid && ma <= Tf, hb = rvalid && mb <= Tf;
                    if (__any_sync(0xffffffffu, ha || hb)) {
                        // valid rows of the tile: read only for a chunk with hits
                        const uint32_t *vmp = Dp->mask + hh * 4 + rd * 2;
                        anyhit = true;
                        if (ha)
                            hm[rd * 2 + 0] = hit_mask32(va, Tf) & vmp[0];
                        if (hb)
                            hm[rd * 2 + 1] = hit_mask32(vb, Tf) & vmp[1];
                    }
                }
                if (anyhit)
                    r0 = Dp->r0;
            }
            // release this warp's share of the accumulator (and with the last
            // share the descriptor slot)
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&S.tmem_empty[acc]);
            // reconverge: otherwise lanes 1-31 run ahead into the next wait's
            // polling loop and lane 0's remaining work interleaves with it
            __syncwarp();
            if (new_job != it_job) {
                // survivors queued for another job are rechecked with its values
                if (nq)
                    flush();
                if (T.job_cycles && lead) {
                    const long long t_now = clock64();
                    if (it_job != 0xffffffffu)
                        atomicAdd(&T.job_cycles[it_job], (unsigned long long)(t_now - t_job));
                    t_job = t_now;
                }
                it_job = new_job;
            }
            if (anyhit) {
                // this lane's survivors: marked columns, in a self-join those
                // with cpos >= qpos (one orientation; rows of the other
                // searched cells lie after the query cell)
                uint32_t k = 0;
                const bool sym = !ASYM;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const uint32_t col0 = r0 + cb + (uint32_t)c * 32u;
                    if (sym) {
                        if (col0 + 31u < it_qpos)
                            hm[c] = 0u;
                        else if (col0 < it_qpos)
                            hm[c] &= ~((1u << (it_qpos - col0)) - 1u);
                    }
                    k += (uint32_t)__popc(hm[c]);
                }
                uint32_t incl = k;
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o)
                        incl += y;
                }
                const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
                if (tot) {
                    const uint32_t rhead = *(volatile uint32_t *)&S.rq_head[e];
                    if (rq_tail + tot - rhead <= (uint32_t)TC_RQ) {
                        // room in the ring: hand them to the recheck warp
                        uint32_t at = rq_tail + incl - k;
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            uint32_t mm = hm[c];
                            while (mm) {
                                const uint32_t b = (uint32_t)(__ffs(mm) - 1);
                                mm &= mm - 1u;
                                const uint32_t slot = at & (uint32_t)(TC_RQ - 1);
                                S.rq_q[e][slot] = it_qpos;
                                S.rq_c[e][slot] = r0 + cb + (uint32_t)c * 32u + b;
                                S.rq_j[e][slot] = it_job;
                                ++at;
                            }
                        }
                        __syncwarp();
                        __threadfence_block();
                        rq_tail += tot;
                        if (lane == 0) {
                            *(volatile uint32_t *)&S.rq_tail[e] = rq_tail;
                            surv_w += tot;
                        }
                        __syncwarp();
                    } else {
                        // ring full (dense data): recheck them here
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            if (__any_sync(0xffffffffu, hm[c] != 0u))
                                nq = tc_queue_bits<ASYM>(&T, hm[c], cb + (uint32_t)c * 32u, it_qpos, r0, sq, sc, nq, nullptr,
                                                   nullptr, nullptr, surv_w, &S.counted, it_job, dpos);
                    }
                }
            }
            if (nq >= 32u)
                flush();
        }
        if (!dead && nq)
            flush();
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();   // the ring's last tail is visible before the count
            atomicAdd(&S.epi_done, 1u);
            if (surv_w)
                atomicAdd(&S.surv, (unsigned long long)surv_w);
        }
        if (T.job_cycles && lead && it_job != 0xffffffffu)
            atomicAdd(&T.job_cycles[it_job], (unsigned long long)(clock64() - t_job));
        for (int o = 16; o; o >>= 1)
            counted += __shfl_xor_sync(0xffffffffu, counted, o);
        if (lane == 0 && counted)
            atomicAdd(&S.counted, counted);
        if (dead) {
            S.abort = 1;
            atomicOr(&L.ctl->err, kErrTimeout);
        }
    } else {
        // ------------------------------------------------------------ epilogue (staged output)
        const int e = warp - 2, q = warp & 3, hh = e >> 2;
        const int etid = threadIdx.x - 64;
        uint32_t turn = 0, es = 0, commit_tile = 0;
        bool failed = false, dead = false;
        uint32_t *const sq = S.sq[e], *const sc = S.sc[e];
        uint32_t nq = 0;
        uint32_t surv_w = 0;   // survivors this warp found (lane 0)
        // tuning launches: the cycles from one item end to the next are the
        // cost of the later item in the steady state (the epilogue is the
        // pipeline's last stage); summed per job
        if (etid == 0)
            S.t_item = clock64();
        const float Tf0 = __int_as_float(T.Tbits);
        uint32_t it_qpos = 0, it_job = 0;   // per-item: this lane's query row, its job
        bool it_rvalid = false;              // the row belongs to the item
        float it_Tf = Tf0;                   // the item's survivor threshold
        gj_pair *stg0 = count_only ? nullptr : L.staging + (size_t)blockIdx.x * 2 * TC_STG;
        // Cross-warp agreement only where a decision is needed: at the end of
        // an item and when the MMA thread flags a flush in the descriptor (a
        // uniform signal).  Two barriers: A (every warp finished the tile),
        // read the shared counters, leader reserves and flips the staging
        // half, B (every warp has read); then the old half is copied out
        // while later tiles write the new half.
        auto epi_sync = [&]() -> bool {
            __threadfence_block();
            __syncwarp();
            uint64_t *b = &S.epi_bar[es & 1u];
            if (lane == 0)
                mbar_arrive(b);
            const bool ok = mbar_wait(b, (es >> 1) & 1u, abort, T.limit_ns);
            ++es;
            return __all_sync(0xffffffffu, ok);   // one decision per warp
        };
        for (;;) {
            const uint32_t acc = turn & 1u, par = (turn >> 1) & 1u;
            const bool ok = mbar_wait(&S.tmem_full[acc], par, abort, T.limit_ns);
            // one decision per warp: the TMEM loads below need all 32 lanes
            if (__any_sync(0xffffffffu, !ok)) {
                dead = true;
                break;
            }
            tc_fence_after();
            // the descriptor slot is reused once the accumulator is released:
            // what is needed afterwards is read now
            const TileDesc *Dp = &S.tdesc[acc];
            const uint32_t flags = Dp->flags, d_tile = Dp->tile, d_item = Dp->item;
            if (flags & F_FIRST) {
                // per-item values, the same in every descriptor of the item
                commit_tile = d_tile;
                failed = false;
                const uint32_t qa = Dp->qa, qb = Dp->qbeg, ql = Dp->qlen;
                it_qpos = qa + (uint32_t)(q * 32 + lane);
                it_rvalid = it_qpos >= qb && it_qpos < qb + ql;
                it_job = Dp->p2;
                it_Tf = T.jobs ? __uint_as_float(Dp->p3) : Tf0;
            }
            const bool is_tile = !(flags & (F_MARKER | F_TERM));
            const float Tf = it_Tf;
            const uint32_t qpos = it_qpos;
            const bool rvalid = it_rvalid;
            uint32_t hm0 = 0, hm1 = 0, hm2 = 0, hm3 = 0;   // per-lane hit masks of the 4 chunks
            bool anyhit = false;
            uint32_t r0 = 0;
            if (is_tile && !failed) {
                // valid rows of this thread's 128 columns: read only for a chunk
                // with hits, before the accumulator (and with it the descriptor
                // slot) is released
                const uint32_t *vmp = Dp->mask + hh * 4;
                const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + acc * 256u + (uint32_t)hh * 128u;
                {
                    uint32_t va[32], vb[32];
                    float ma, mb;
                    tmem_ld32_min(tb, va, ma);
                    tmem_ld32_min(tb + 32u, vb, mb);
                    tmem_wait_ld();
                    const bool ha = rvalid && ma <= Tf, hb = rvalid && mb <= Tf;
                    if (__any_sync(0xffffffffu, ha || hb)) {
                        anyhit = true;
                        if (ha)
                            hm0 = hit_mask32(va, Tf) & vmp[0];
                        if (hb)
                            hm1 = hit_mask32(vb, Tf) & vmp[1];
                    }
                }
                {
                    uint32_t va[32], vb[32];
                    float ma, mb;
                    tmem_ld32_min(tb + 64u, va, ma);
                    tmem_ld32_min(tb + 96u, vb, mb);
                    tmem_wait_ld();
                    const bool ha = rvalid && ma <= Tf, hb = rvalid && mb <= Tf;
                    if (__any_sync(0xffffffffu, ha || hb)) {
                        anyhit = true;
                        if (ha)
                            hm2 = hit_mask32(va, Tf) & vmp[2];
                        if (hb)
                            hm3 = hit_mask32(vb, Tf) & vmp[3];
                    }
                }
            }
            if (anyhit)
                r0 = Dp->r0;
            // A warp with few hits queues them after releasing the accumulator.
            // A warp with many (dense data) queues and rechecks them before, so
            // that its staging output is seen by the flush logic in time.
            bool early = false;
            if (anyhit) {
                const int hits =
                    __reduce_add_sync(0xffffffffu, __popc(hm0) + __popc(hm1) + __popc(hm2) + __popc(hm3));
                early = hits > 32;
            }
            if (!early) {
                tc_fence_before();
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(&S.tmem_empty[acc]);
                __syncwarp();
            }
            const uint32_t half = S.half;
            gj_pair *stg = stg0 ? stg0 + (size_t)half * TC_STG : nullptr;
            if (anyhit) {
                const uint32_t cb = (uint32_t)hh * 128u;
                if (__any_sync(0xffffffffu, hm0 != 0u))
                    nq = tc_queue_bits<ASYM>(&T, hm0, cb + 0u, qpos, r0, sq, sc, nq, stg, &S.cnt[half],
                                       &S.flush_req, surv_w, &S.counted, it_job);
                if (__any_sync(0xffffffffu, hm1 != 0u))
                    nq = tc_queue_bits<ASYM>(&T, hm1, cb + 32u, qpos, r0, sq, sc, nq, stg, &S.cnt[half],
                                       &S.flush_req, surv_w, &S.counted, it_job);
                if (__any_sync(0xffffffffu, hm2 != 0u))
                    nq = tc_queue_bits<ASYM>(&T, hm2, cb + 64u, qpos, r0, sq, sc, nq, stg, &S.cnt[half],
                                       &S.flush_req, surv_w, &S.counted, it_job);
                if (__any_sync(0xffffffffu, hm3 != 0u))
                    nq = tc_queue_bits<ASYM>(&T, hm3, cb + 96u, qpos, r0, sq, sc, nq, stg, &S.cnt[half],
                                       &S.flush_req, surv_w, &S.counted, it_job);
                if (early && nq) {
                    unsigned long long c = 0;
                    __syncwarp();
                    tc_flush_survivors<ASYM>(&T, sq, sc, nq, stg, &S.cnt[half], &S.flush_req, &c, it_job);
                    __syncwarp();
                    if (c)
                        atomicAdd(&S.counted, c);
                    nq = 0;
                }
            }
            if (early) {
                tc_fence_before();
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(&S.tmem_empty[acc]);
                __syncwarp();
            }
            ++turn;
            // the accumulator is released; recheck queued survivors now when the
            // queue is half full, or when the item's results must be complete
            const bool item_end = (flags & F_LAST) != 0;   // (every marker but a pad ends its item)
            const bool flush = (flags & F_FLUSH) != 0;
            if (nq >= 32u || ((item_end || flush || (flags & F_TERM)) && nq)) {
                unsigned long long c = 0;
                __syncwarp();
                tc_flush_survivors<ASYM>(&T, sq, sc, nq, stg, &S.cnt[half], &S.flush_req, &c, it_job);
                __syncwarp();
                if (c)
                    atomicAdd(&S.counted, c);
                nq = 0;
            }
            if (flags & F_TERM)
                break;
            if (T.job_cycles && item_end && etid == 0) {
                const long long t_now = clock64();
                atomicAdd(&T.job_cycles[L.ix.items[d_item].pad], (unsigned long long)(t_now - S.t_item));
                S.t_item = t_now;
            }
            if (count_only)
                continue;
            if (!item_end && !flush)
                continue;
            if (!epi_sync()) {   // A
                dead = true;
                break;
            }
            const uint32_t cnt = S.cnt[half];
            const bool commit = !failed && !(flags & F_TRUNC);
            if (etid == 0) {
                uint32_t ok = 0;
                unsigned long long b = 0;
                if (commit) {
                    ok = 1;
                    if (cnt) {
                        b = atomicAdd(&L.ctl->pos, (unsigned long long)cnt);
                        ok = (b + cnt <= L.cap) ? 1u : 0u;
                        if (!ok) {
                            atomicMin(&L.ctl->fail_base, b);
                            atomicExch(&L.ctl->full, 1u);
                        }
                    }
                }
                if (item_end && !(commit && ok)) {
                    uint32_t slot = atomicAdd(&L.ctl->dout_n, 1u);
                    if (slot < L.dout_cap)
                        L.dout[slot] = Deferred{d_item, commit_tile};
                    else
                        atomicOr(&L.ctl->err, kErrDeferred);
                }
                S.ok = ok;
                S.base = b;
                S.cnt[half ^ 1u] = 0;
                S.half = half ^ 1u;
                S.flush_req = 0;
            }
            if (!epi_sync()) {   // B
                dead = true;
                break;
            }
            if (commit) {
                if (S.ok) {
                    const unsigned long long b = S.base;
                    for (uint32_t i = (uint32_t)etid; i < cnt; i += 256u)
                        L.out[b + i] = stg[i];
                    if (!item_end && is_tile)
                        commit_tile = d_tile + 1;
                } else {
                    failed = true;
                }
            }
        }
        if (lane == 0 && surv_w)
            atomicAdd(&S.surv, (unsigned long long)surv_w);
        if (dead) {
            S.abort = 1;
            atomicOr(&L.ctl->err, kErrTimeout);
        }
    }

    __syncthreads();
    if (threadIdx.x == 0) {
        if (S.surv)
            atomicAdd(&L.ctl->survivors, S.surv);
        if (S.counted)
            atomicAdd(&L.ctl->counted, S.counted);
        if (L.sm_span)
            note_sm_span(L.sm_span, (unsigned long long)S.t_start, globaltimer());
    }
    if (S.abort) {
        // let copies and MMAs already issued land before the memory goes away
        const uint64_t t0 = globaltimer();
        while (globaltimer() - t0 < 2000000ull) {
        }
    }
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// ---------------------------------------------------------------------------
// Operand preparation
// ---------------------------------------------------------------------------
struct TcPrepParams {
    int d, Kp;
    double sigma;
    const double *centre;   // device, reordered dims
    int64_t row_off;        // output row of point 0 (many-jobs layouts)
};

__global__ void k_tc_radius(const double *__restrict__ X, int64_t n, int64_t npad, int d,
                            const double *__restrict__ centre, unsigned long long *__restrict__ rmax)
{
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double r2 = 0.0;
    if (p < n)
        for (int j = 0; j < d; ++j) {
            double t = X[(int64_t)j * npad + p] - centre[j];
            r2 = __fma_rn(t, t, r2);
        }
    for (int o = 16; o; o >>= 1)
        r2 = fmax(r2, __shfl_xor_sync(0xffffffffu, r2, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(rmax, (unsigned long long)__double_as_longlong(r2));
}

__device__ __forceinline__ __half tc_coord(const double *__restrict__ X, int64_t npad, int64_t p, int j,
                                           const double *__restrict__ centre, double sigma)
{
    return __double2half((X[(int64_t)j * npad + p] - centre[j]) * sigma);
}

// XA/XB: row p at core matrix ((p/8)*(Kp/8) + k/8), row p%8, element k%8.
// Either may be null (Q join_eps E packs its queries as A rows only).
__global__ void k_tc_pack(const double *__restrict__ X, int64_t n, int64_t npad, TcPrepParams P,
                          uint4 *__restrict__ XA, uint4 *__restrict__ XB)
{
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n)
        return;
    const int d = P.d, Kp = P.Kp;
    double nrm = 0.0;
    for (int j = 0; j < d; ++j) {
        double h = (double)__half2float(tc_coord(X, npad, p, j, P.centre, P.sigma));
        nrm = __fma_rn(h, h, nrm);
    }
    const __half hi = __double2half(nrm);
    const __half lo = __double2half(nrm - (double)__half2float(hi));
    const __half one = __float2half(1.0f), zero = __float2half(0.0f);
    for (int kc = 0; kc < Kp / 8; ++kc) {
        __align__(16) __half a[8], b[8];
        for (int e = 0; e < 8; ++e) {
            const int k = kc * 8 + e;
            if (k < d) {
                __half h = tc_coord(X, npad, p, k, P.centre, P.sigma);
                b[e] = h;
                a[e] = __float2half(-2.0f * __half2float(h));
            } else if (k == d) {
                a[e] = hi;
                b[e] = one;
            } else if (k == d + 1) {
                a[e] = lo;
                b[e] = one;
            } else if (k == d + 2) {
                a[e] = one;
                b[e] = hi;
            } else if (k == d + 3) {
                a[e] = one;
                b[e] = lo;
            } else {
                a[e] = zero;
                b[e] = zero;
            }
        }
        const int64_t r = p + P.row_off;
        const int64_t idx = ((r >> 3) * (Kp / 8) + kc) * 8 + (r & 7);   // in 16-byte units
        if (XA)
            XA[idx] = *reinterpret_cast<const uint4 *>(a);
        if (XB)
            XB[idx] = *reinterpret_cast<const uint4 *>(b);
    }
}

// XR[p * dr + j] = X[j * npad + p]: the points row by row (rows padded with
// zeros to dr values), for the recheck's contiguous reads.
__global__ void k_tc_rows(const double *__restrict__ X, int64_t n, int64_t npad, int d, int dr,
                          double *__restrict__ XR)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n * dr)
        return;
    const int64_t p = i / dr;
    const int j = (int)(i - p * dr);
    XR[i] = j < d ? X[(int64_t)j * npad + p] : 0.0;
}

// Survivor threshold in scaled units (see the file header for the terms).
double tc_threshold(double eps, double sigma, double R0, int d, int Kp)
{
    const double sd = sqrt((double)d);
    const double Rh = sigma * R0 * (1.0 + ldexp(1.0, -10)) + sd * ldexp(1.0, -24);
    const double quant = 2.0 * (ldexp(1.0, -11) * Rh + sd * ldexp(1.0, -25));
    const double D = sigma * eps * (1.0 + ldexp(1.0, -40)) + quant * (1.0 + ldexp(1.0, -40));
    const double E = (Kp + 2) * ldexp(1.0, -22) * 4.04 * Rh * Rh + 2.0 * ldexp(1.0, -21) * Rh * Rh * 1.01 +
                     (2.0 * d + 8.0) * ldexp(1.0, -50) * Rh * Rh;
    return (D * D + E) * (1.0 + ldexp(1.0, -20));
}

int tc_prepare(gj_index *h, const double *stats_host, const int *perm, cudaStream_t s)
{
    const int d = h->info.d;
    const int64_t n = h->info.n;
    const int Kp = ((d + 4 + 15) / 16) * 16;
    if (Kp > 128 || n == 0) {
        h->tc_ready = false;
        return GJ_OK;
    }
    std::vector<double> c(d);
    for (int j = 0; j < d; ++j)
        c[j] = 0.5 * (stats_host[(size_t)perm[j] * 4 + 2] + stats_host[(size_t)perm[j] * 4 + 3]);
    double *centre = nullptr;
    cudaError_t e = dev_alloc(&centre, d * sizeof(double), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(centre, c.data(), d * sizeof(double), cudaMemcpyHostToDevice, s);
    double R0 = 0.0;
    if (e == cudaSuccess)
        e = tc_radius(h->X, n, h->npad, d, centre, &R0, s);
    const double sigma = tc_sigma_for(R0);
    const int64_t rows = h->npad + 512;
    const size_t bytes = (size_t)rows * Kp * 2;
    if (e == cudaSuccess)
        e = dev_alloc(&h->XA, bytes, s);
    if (e == cudaSuccess)
        e = dev_alloc(&h->XB, bytes, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(h->XA, 0, bytes, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(h->XB, 0, bytes, s);
    if (e == cudaSuccess) {
        TcPrepParams P{d, Kp, sigma, centre, 0};
        note_launch();
        k_tc_pack<<<(int)((n + 127) / 128), 128, 0, s>>>(h->X, n, h->npad, P, (uint4 *)h->XA, (uint4 *)h->XB);
        e = cudaGetLastError();
    }
    // the recheck's copy of the points, row by row
    const int dr = (d + 3) & ~3;
    if (e == cudaSuccess)
        e = dev_alloc(&h->XR, (size_t)n * dr * sizeof(double), s);
    if (e == cudaSuccess) {
        note_launch();
        k_tc_rows<<<(int)((n * dr + 255) / 256), 256, 0, s>>>(h->X, n, h->npad, d, dr, h->XR);
        e = cudaGetLastError();
    }
    h->XR_dr = dr;
    h->tc_centre = centre;   // kept: a many-jobs layout and Q join_eps E re-pack from it
    if (e != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? GJ_ERR_OOM : GJ_ERR_CUDA;
    const double Td = tc_threshold(h->info.eps, sigma, R0, d, Kp);
    float Tf = (float)Td;
    if ((double)Tf < Td)
        Tf = nextafterf(Tf, INFINITY);
    int Tb;
    memcpy(&Tb, &Tf, sizeof(Tb));
    h->tc_Kp = Kp;
    h->tc_Tbits = Tb;
    h->tc_sigma = sigma;
    h->tc_R0 = R0;
    h->tc_ready = true;
    return GJ_OK;
}

static int tc_stages(int Kp, uint32_t *a_bytes, uint32_t *b_bytes, uint32_t *off_b, uint32_t *off_s,
                     size_t *smem)
{
    *a_bytes = (uint32_t)TC_M * Kp * 2;
    *b_bytes = (uint32_t)TC_N * Kp * 2;
    const size_t budget = 227 * 1024 - 1024;
    const size_t fixed = 2 * (size_t)(*a_bytes) + ((sizeof(TcShared) + 1023) & ~size_t(1023));
    int ns = (int)((budget - fixed) / *b_bytes);
    if (ns > 8)
        ns = 8;
    *off_b = 2 * *a_bytes;
    *off_s = *off_b + (uint32_t)ns * *b_bytes;
    *smem = *off_s + sizeof(TcShared);
    if (*smem < 120 * 1024)
        *smem = 120 * 1024;   // one CTA per SM: each holds all 512 TMEM columns
    return ns;
}

size_t tc_staging_pairs_per_cta() { return 2 * (size_t)TC_STG; }

int tc_threshold_bits(double eps, double sigma, double R0, int d, int Kp)
{
    const double Td = tc_threshold(eps, sigma, R0, d, Kp);
    float Tf = (float)Td;
    if ((double)Tf < Td)
        Tf = nextafterf(Tf, INFINITY);
    int Tb;
    memcpy(&Tb, &Tf, sizeof(Tb));
    return Tb;
}

cudaError_t tc_pack_into(const double *X, int64_t n, int64_t npad, int d, int Kp, double sigma, const double *centre,
                         int64_t row_off, void *XA, void *XB, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    TcPrepParams P{d, Kp, sigma, centre, row_off};
    note_launch();
    k_tc_pack<<<(int)((n + 127) / 128), 128, 0, s>>>(X, n, npad, P, (uint4 *)XA, (uint4 *)XB);
    return cudaGetLastError();
}

cudaError_t tc_jobs_launch_attr(int Kp)
{
    uint32_t a, b, ob, os;
    size_t sm = 0;
    if (tc_stages(Kp, &a, &b, &ob, &os, &sm) < 2)
        return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(k_join_tc<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

// (call tc_jobs_launch_attr first: this launcher sets no attribute, so it can
// run inside a stream capture)
cudaError_t launch_join_tc_jobs(const JoinLaunch &L, const void *XA, const void *XB, int Kp, const TcJob *jobs,
                                unsigned long long *jpos, int grid, cudaStream_t s, unsigned long long *job_cycles)
{
    TcLaunch T{};
    T.J = L;
    T.jobs = jobs;
    T.jpos = jpos;
    T.job_cycles = jobs ? job_cycles : nullptr;
    T.XA = (const unsigned char *)XA;
    T.XB = (const unsigned char *)XB;
    T.Kp = Kp;
    T.Tbits = 0;
    T.limit_ns = wait_limit_ns();
    size_t sm = 0;
    T.NS = tc_stages(T.Kp, &T.a_bytes, &T.b_bytes, &T.off_b, &T.off_s, &sm);
    if (T.NS < 2)
        return cudaErrorInvalidValue;
    k_join_tc<true, false><<<grid, TC_THREADS, sm, s>>>(T);   // every job writes its own buffer directly
    return cudaGetLastError();
}

cudaError_t launch_join_tc(const gj_index *h, const JoinLaunch &L, int grid, cudaStream_t s, bool direct)
{
    TcLaunch T{};
    T.J = L;
    T.XA = (const unsigned char *)h->XA;
    T.XB = (const unsigned char *)h->XB;
    T.XR = h->XR;
    T.dr = h->XR_dr;
    T.Kp = h->tc_Kp;
    T.Tbits = h->tc_Tbits;
    T.limit_ns = wait_limit_ns();
    size_t sm = 0;
    T.NS = tc_stages(T.Kp, &T.a_bytes, &T.b_bytes, &T.off_b, &T.off_s, &sm);
    if (T.NS < 2)
        return cudaErrorInvalidValue;
    cudaError_t e = direct
                        ? cudaFuncSetAttribute(k_join_tc<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)
                        : cudaFuncSetAttribute(k_join_tc<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)sm);
    if (e != cudaSuccess)
        return e;
    note_launch();
    if (direct)
        k_join_tc<true, false><<<grid, TC_THREADS, sm, s>>>(T);
    else
        k_join_tc<false, false><<<grid, TC_THREADS, sm, s>>>(T);
    return cudaGetLastError();
}

// Direct form over explicit operand arrays and threshold (Q join_eps E: query
// A rows, entry B rows, both under one centre and scale; XR: the entries row by
// row, nullable).
cudaError_t launch_join_tc_ops(const JoinLaunch &L, const void *XA, const void *XB, const double *XR, int dr, int Kp,
                               int Tbits, int grid, cudaStream_t s)
{
    TcLaunch T{};
    T.J = L;
    T.XA = (const unsigned char *)XA;
    T.XB = (const unsigned char *)XB;
    T.XR = XR;
    T.dr = dr;
    T.Kp = Kp;
    T.Tbits = Tbits;
    T.limit_ns = wait_limit_ns();
    size_t sm = 0;
    T.NS = tc_stages(T.Kp, &T.a_bytes, &T.b_bytes, &T.off_b, &T.off_s, &sm);
    if (T.NS < 2)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_join_tc<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess)
        return e;
    note_launch();
    k_join_tc<true, true><<<grid, TC_THREADS, sm, s>>>(T);
    return cudaGetLastError();
}

// Radius of a point set about a centre: sqrt of the largest squared distance
// (times 1 + 2^-30, the same widening as the index build's).
cudaError_t tc_radius(const double *X, int64_t n, int64_t npad, int d, const double *centre, double *R0,
                      cudaStream_t s)
{
    *R0 = 0.0;
    if (n <= 0)
        return cudaSuccess;
    unsigned long long *rmax = nullptr;
    unsigned long long rbits = 0;
    cudaError_t e = dev_alloc(&rmax, sizeof(unsigned long long), s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(rmax, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
        note_launch();
        k_tc_radius<<<(int)((n + 255) / 256), 256, 0, s>>>(X, n, npad, d, centre, rmax);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&rbits, rmax, sizeof(rbits), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    dev_free(rmax, s);
    double R2 = 0.0;
    memcpy(&R2, &rbits, sizeof(R2));
    *R0 = sqrt(R2) * (1.0 + ldexp(1.0, -30));
    return e;
}

// The power-of-two scale that keeps every |h| of a set of radius R0 at most 250.
double tc_sigma_for(double R0)
{
    int sexp = 0;
    if (R0 > 0.0)
        sexp = (int)floor(log2(250.0 / R0));
    return ldexp(1.0, sexp);
}

// ---------------------------------------------------------------------------
// Diagnostic: one 128x128 tile D = A * B^T through the same operand layout,
// descriptors and TMEM path as the join (used by the tests to check the
// layout and the accumulation error model).
// ---------------------------------------------------------------------------
__global__ void k_tc_debug(const unsigned char *__restrict__ A, const unsigned char *__restrict__ B, int Kp,
                           float *__restrict__ D, unsigned int *__restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar_ld, bar_mma;
    __shared__ uint32_t tbase, abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t bytes = 128u * Kp * 2;
    if (threadIdx.x == 0) {
        mbar_init(&bar_ld, 1);
        mbar_init(&bar_mma, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&tbase, 128);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tbase;
    bool ok = true;
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar_ld, 2 * bytes);
        bulk_g2s(smem, A, bytes, &bar_ld);
        bulk_g2s(smem + bytes, B, bytes, &bar_ld);
        ok = mbar_wait(&bar_ld, 0, &abort_flag, TC_LIMIT_NS);
        if (ok) {
            tc_fence_after();
            const uint32_t a0 = smem_addr(smem), b0 = a0 + bytes;
            const uint32_t idesc = idesc_f16_f32(128, 128);
            for (int ks = 0; ks < Kp / 16; ++ks)
                mma_f16(tmem, desc_kmajor(a0 + ks * 256u, 128, Kp * 16), desc_kmajor(b0 + ks * 256u, 128, Kp * 16),
                        idesc, ks > 0 ? 1u : 0u);
            mma_commit(&bar_mma);
        } else {
            abort_flag = 1;
        }
    }
    __syncthreads();
    if (!abort_flag) {
        if (mbar_wait(&bar_mma, 0, &abort_flag, TC_LIMIT_NS)) {
            tc_fence_after();
            const int row = warp * 32 + lane;
            for (int c = 0; c < 4; ++c) {
                // the join's load: the 32 values of this lane's row and their
                // minimum, which must equal the minimum of the values returned
                uint32_t v[32];
                float mn;
                tmem_ld32_min(tmem + ((uint32_t)(warp * 32) << 16) + c * 32u, v, mn);
                tmem_wait_ld();
                float m = __uint_as_float(v[0]);
                for (int i = 0; i < 32; ++i) {
                    m = fminf(m, __uint_as_float(v[i]));
                    D[row * 128 + c * 32 + i] = __uint_as_float(v[i]);
                }
                if (m != mn)
                    atomicOr(err, 2u);
            }
        } else {
            atomicOr(err, 1u);
        }
    } else {
        atomicOr(err, 1u);
    }
    tc_fence_before();
    __syncthreads();
    if (abort_flag) {
        const uint64_t t0 = globaltimer();
        while (globaltimer() - t0 < 2000000ull) {
        }
    }
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 128);
    }
}

}  // namespace gj

extern "C" int gj_debug_tc_tile(const uint16_t *A, const uint16_t *B, int32_t Kp, float *D)
{
    using namespace gj;
    if (!A || !B || !D || Kp < 16 || Kp > 128 || Kp % 16)
        return GJ_ERR_INVALID_ARG;
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess ||
        prop.major != 10 || prop.minor != 3)
        return GJ_ERR_UNSUPPORTED;
    // pack row-major [128][Kp] into the core-matrix layout
    std::vector<uint16_t> pa((size_t)128 * Kp), pb((size_t)128 * Kp);
    for (int r = 0; r < 128; ++r)
        for (int k = 0; k < Kp; ++k) {
            size_t idx = (((size_t)(r >> 3) * (Kp / 8) + (k >> 3)) * 8 + (r & 7)) * 8 + (k & 7);
            pa[idx] = A[(size_t)r * Kp + k];
            pb[idx] = B[(size_t)r * Kp + k];
        }
    unsigned char *dA = nullptr, *dB = nullptr;
    float *dD = nullptr;
    unsigned int *derr = nullptr, herr = 0;
    const size_t bytes = (size_t)128 * Kp * 2;
    cudaError_t e = cudaMalloc(&dA, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&dB, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&dD, 128 * 128 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&derr, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemcpy(dA, pa.data(), bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, pb.data(), bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(derr, 0, sizeof(unsigned int));
    if (e == cudaSuccess) {
        const int sm = (int)(2 * bytes);
        e = cudaFuncSetAttribute(k_tc_debug, cudaFuncAttributeMaxDynamicSharedMemorySize, sm < 48 * 1024 ? 48 * 1024 : sm);
        if (e == cudaSuccess) {
            note_launch();
            k_tc_debug<<<1, 128, sm < 48 * 1024 ? 48 * 1024 : sm>>>(dA, dB, Kp, dD, derr);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(D, dD, 128 * 128 * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(herr), cudaMemcpyDeviceToHost);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dD);
    cudaFree(derr);
    if (e != cudaSuccess)
        return GJ_ERR_CUDA;
    if (herr & 2u)
        return GJ_ERR_CUDA;
    return herr ? GJ_ERR_TIMEOUT : GJ_OK;
}

extern "C" int gj_tc_threshold(double eps, double sigma, double R0, int32_t d, float *T)
{
    if (!T || !(eps > 0.0) || !isfinite(eps) || !(sigma > 0.0) || !isfinite(sigma) || !(R0 >= 0.0) ||
        !isfinite(R0) || d < 1)
        return GJ_ERR_INVALID_ARG;
    const int Kp = ((d + 4 + 15) / 16) * 16;
    if (Kp > 128)
        return GJ_ERR_INVALID_ARG;
    const int bits = gj::tc_threshold_bits(eps, sigma, R0, d, Kp);
    memcpy(T, &bits, sizeof(float));
    return GJ_OK;
}

extern "C" int gj_debug_set_wait_limit(uint64_t ns)
{
    gj::g_wait_limit_ns.store(ns, std::memory_order_relaxed);
    return GJ_OK;
}
