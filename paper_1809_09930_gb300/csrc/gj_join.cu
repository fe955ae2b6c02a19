// gj_join.cu -- the plain FP64 join (Alg. 1 SelfJoinKernel with SORTIDU,
// Sec. 4.3, and SHORTC, Sec. 4.4) and the sampled result-size estimate
// (Sec. 3.2.2).
//
// Design (GB300-first, not the paper's thread-per-point kernel):
//  * persistent CTAs pull work items (a query block of one cell) from a queue
//    ordered by descending load; a per-launch deferred list carries the resume
//    point of items whose results did not fit the output (exact resume);
//  * the query block and one candidate tile of the searched cells sit in
//    shared memory, dimension-major, in REORDER order;
//  * each lane owns one (query, candidate) pair at a time and advances it one
//    dimension per step: d = x_q - x_c, s = fma(d, d, s), stop when s > eps^2
//    (compared as integers: s >= 0, so the IEEE bit order is the numeric
//    order).  A lane whose pair stopped or finished takes the next pair of the
//    tile at once (warp ballot + shared counter), so the FP64 pipe only ever
//    computes dimensions some pair needs -- the depth each pair needs under a
//    per-dimension SHORTC check, no warp-wide "slowest lane" cost;
//  * result pairs are compacted with a warp ballot + popcount prefix and one
//    shared-memory atomic per warp into a per-CTA staging area, which is
//    committed to the output with one global atomic per item (or when nearly
//    full); a commit that does not fit marks the launch full and defers the
//    item from its first uncommitted tile.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gj_internal.cuh"

namespace gj {

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr int JT = 256;               // threads per CTA
constexpr unsigned FULL = 0xffffffffu;
constexpr unsigned NONE = 0xffffffffu;
constexpr int NBCHUNK = JT;           // neighbour windows computed per round

struct SmemHdr {
    uint32_t item, resume, cell, qbeg, qlen;
    int64_t cell_end;
    int64_t nb_begin, nb_end;
    uint32_t next;            // pair counter of the current tile
    uint32_t stg_cnt;         // pairs in the staging area
    uint32_t stop;            // abandon the current item (deferred)
    unsigned long long base;
    int ok;
    long long t_start;        // clock at the CTA's start
    int64_t win_s[NBCHUNK];
    int64_t win_e[NBCHUNK];
    uint32_t win_b[NBCHUNK];
};

__device__ __forceinline__ int64_t lower_u(const double *__restrict__ U, int64_t lo, int64_t hi, double ref,
                                           double ew)
{
    // first q in [lo,hi) with fl(U[q] - ref) >= -ew
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (U[mid] - ref < -ew)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int64_t upper_u(const double *__restrict__ U, int64_t lo, int64_t hi, double ref,
                                           double ew)
{
    // first q in [lo,hi) with fl(U[q] - ref) > ew
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (U[mid] - ref <= ew)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// DIRECT = true: pairs go straight to the output through one global atomic
// per warp (no staging, no commit/defer protocol); pairs past `cap` are
// counted but not written.
template <int CT, int QBT, bool DIRECT = false, bool ASYM = false>
__global__ void __launch_bounds__(JT) k_join_plain(JoinLaunch L)
{
    constexpr int LOGCT = (CT == 64) ? 6 : (CT == 32 ? 5 : 4);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemHdr &H = *reinterpret_cast<SmemHdr *>(smem_raw);
    const int d = L.ix.d;
    double *Qs = reinterpret_cast<double *>(smem_raw + ((sizeof(SmemHdr) + 15) & ~size_t(15)));
    double *Cs = Qs + (size_t)d * QBT;

    const int tid = threadIdx.x, lane = tid & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t npad = L.ix.npad;
    const double *__restrict__ X = L.ix.X;
    const long long e2bits = __double_as_longlong(L.ix.e2);
    const bool count_only = (L.out == nullptr);
    const bool staged = !count_only && !DIRECT;
    gj_pair *stg = staged ? L.staging + (size_t)blockIdx.x * L.stg_cap : nullptr;
    const uint32_t flush_at = L.stg_cap > 2u * QBT * CT ? L.stg_cap - 2u * QBT * CT : 0u;

    unsigned long long my_count = 0, my_dims = 0, my_pairs = 0;

    if (tid == 0) {
        H.stg_cnt = 0;
        H.t_start = (long long)globaltimer_ns();
    }

    for (;;) {
        // ---- next item: deferred resume points first, then the main queue
        if (tid == 0) {
            uint32_t item = NONE, resume = 0;
            if (!count_only && *(volatile unsigned int *)&L.ctl->full) {
                item = NONE;
            } else {
                uint32_t t = (L.n_din > 0) ? atomicAdd(&L.ctl->din_head, 1u) : NONE;
                if (t < L.n_din) {
                    item = L.din[t].item;
                    resume = L.din[t].tile;
                } else {
                    uint32_t hq = atomicAdd(&L.ctl->head, 1u);
                    if (hq < L.qlimit)
                        item = L.queue[hq];
                }
            }
            H.item = item;
            H.resume = resume;
            H.stop = 0;
            if (item != NONE) {
                Item it = L.ix.items[item];
                H.cell = it.cell;
                H.qbeg = it.qbeg;
                H.qlen = it.qlen;
                H.cell_end = ASYM ? 0 : L.ix.cell_start[it.cell + 1];
                H.nb_begin = L.ix.adj_start[it.cell];
                H.nb_end = L.ix.adj_start[it.cell + 1];
            }
        }
        __syncthreads();
        if (H.item == NONE)
            break;
        const uint32_t cell = H.cell, qbeg = H.qbeg, qlen = H.qlen;
        const int64_t nb_begin = H.nb_begin, nb_end = H.nb_end;

        // ---- query block -> shared memory, Qs[j][qi] (a similarity join's
        // queries live in their own array)
        const double *__restrict__ XQ = ASYM ? L.ix.XQ : X;
        const int64_t qstride = ASYM ? L.ix.qnpad : npad;
        for (int idx = tid; idx < d * QBT; idx += JT) {
            int j = idx / QBT, qi = idx - j * QBT;
            Qs[idx] = (qi < (int)qlen) ? XQ[(int64_t)j * qstride + qbeg + qi] : 0.0;
        }

        uint32_t tile_idx = 0, commit_tile = H.resume;
        const int u = L.ix.u;
        double ulo = 0.0, uhi = 0.0;
        if (u >= 0) {
            ulo = XQ[(int64_t)u * qstride + qbeg];
            uhi = XQ[(int64_t)u * qstride + qbeg + qlen - 1];
        }

        for (int64_t nb0 = nb_begin; nb0 < nb_end && !H.stop; nb0 += NBCHUNK) {
            // ---- windows of up to NBCHUNK searched cells (SORTIDU, Sec. 4.3)
            __syncthreads();
            if (nb0 + tid < nb_end) {
                uint32_t b = L.ix.adj[nb0 + tid];
                int64_t cs, ce;
                if (!ASYM && b == cell) {
                    cs = qbeg;
                    ce = H.cell_end;
                } else {
                    cs = L.ix.cell_start[b];
                    ce = L.ix.cell_start[b + 1];
                }
                if (u >= 0) {
                    const double *U = X + (int64_t)u * npad;
                    cs = lower_u(U, cs, ce, ulo, L.ix.ew);
                    ce = upper_u(U, cs, ce, uhi, L.ix.ew);
                }
                H.win_s[tid] = cs;
                H.win_e[tid] = ce;
                H.win_b[tid] = b;
            }
            __syncthreads();
            const int nwin = (int)min((int64_t)NBCHUNK, nb_end - nb0);
            for (int w = 0; w < nwin && !H.stop; ++w) {
                const int64_t ws = H.win_s[w], we = H.win_e[w];
                const bool self = !ASYM && (H.win_b[w] == cell);
                for (int64_t t0 = ws; t0 < we; t0 += CT, ++tile_idx) {
                    if (tile_idx < commit_tile)
                        continue;   // committed by an earlier launch
                    const int tlen = (int)min((int64_t)CT, we - t0);
                    // ---- stop if another CTA filled the output
                    if (tid == 0) {
                        H.next = 0;
                        if (!count_only && *(volatile unsigned int *)&L.ctl->full)
                            H.stop = 1;
                    }
                    // ---- candidate tile -> Cs[j][c]
                    for (int idx = tid; idx < d * CT; idx += JT) {
                        int j = idx >> LOGCT, c = idx & (CT - 1);
                        Cs[idx] = (c < tlen) ? X[(int64_t)j * npad + t0 + c] : 0.0;
                    }
                    __syncthreads();
                    if (H.stop)
                        break;
                    // ---- pairs of the tile, one dimension per step per lane
                    {
                        const uint32_t P = qlen << LOGCT;
                        int qi = 0, cj = 0, j = 0;
                        double s = 0.0;
                        bool act = false, exhausted = false;
                        for (;;) {
                            if (!exhausted) {
                                unsigned need = __ballot_sync(FULL, !act);
                                if (need) {
                                    uint32_t base = 0;
                                    if (lane == 0)
                                        base = atomicAdd(&H.next, (uint32_t)__popc(need));
                                    base = __shfl_sync(FULL, base, 0);
                                    if (base + (uint32_t)__popc(need) >= P)
                                        exhausted = true;
                                    if (!act) {
                                        uint32_t p = base + __popc(need & lt);
                                        if (p < P) {
                                            qi = (int)(p >> LOGCT);
                                            cj = (int)(p & (CT - 1));
                                            bool ok = cj < tlen &&
                                                      (!self || t0 + cj >= (int64_t)qbeg + qi);
                                            if (ok) {
                                                act = true;
                                                j = 0;
                                                s = 0.0;
                                            }
                                        }
                                    }
                                }
                            }
                            if (!__any_sync(FULL, act)) {
                                if (exhausted)
                                    break;
                                continue;
                            }
                            bool fin = false;
                            if (act) {
                                double t = Qs[j * QBT + qi] - Cs[(j << LOGCT) + cj];
                                s = __fma_rn(t, t, s);
                                ++j;
                                ++my_dims;
                                if (__double_as_longlong(s) > e2bits) {
                                    act = false;
                                    ++my_pairs;
                                } else if (j == d) {
                                    act = false;
                                    fin = true;
                                    ++my_pairs;
                                }
                            }
                            unsigned em = __ballot_sync(FULL, fin);
                            if (em) {
                                const uint32_t qpos = qbeg + qi;
                                const uint32_t cpos = (uint32_t)(t0 + cj);
                                // both orientations, except a self-pair and a similarity join's (q, e)
                                const bool two = fin && !ASYM && (qpos != cpos);
                                unsigned em2 = __ballot_sync(FULL, two);
                                if (count_only) {
                                    my_count += (fin ? 1 : 0) + (two ? 1 : 0);
                                } else if constexpr (DIRECT) {
                                    const uint32_t cnt = __popc(em) + __popc(em2);
                                    unsigned long long off = 0;
                                    if (lane == 0)
                                        off = atomicAdd(&L.ctl->pos, (unsigned long long)cnt);
                                    off = __shfl_sync(FULL, off, 0);
                                    if (fin) {
                                        const uint32_t a = ASYM ? L.ix.qorig[qpos] : L.ix.orig[qpos];
                                        const uint32_t b = L.ix.orig[cpos];
                                        const unsigned long long i1 = off + __popc(em & lt);
                                        if (i1 < L.cap)
                                            L.out[i1] = gj_pair{a, b};
                                        if (two) {
                                            const unsigned long long i2 = off + __popc(em) + __popc(em2 & lt);
                                            if (i2 < L.cap)
                                                L.out[i2] = gj_pair{b, a};
                                        }
                                    }
                                } else {
                                    uint32_t cnt = __popc(em) + __popc(em2);
                                    uint32_t off = 0;
                                    if (lane == 0)
                                        off = atomicAdd(&H.stg_cnt, cnt);
                                    off = __shfl_sync(FULL, off, 0);
                                    if (off + cnt > L.stg_cap) {
                                        if (lane == 0)
                                            atomicOr(&L.ctl->err, kErrStaging);
                                    } else if (fin) {
                                        uint32_t a = ASYM ? L.ix.qorig[qpos] : L.ix.orig[qpos];
                                        uint32_t b = L.ix.orig[cpos];
                                        stg[off + __popc(em & lt)] = gj_pair{a, b};
                                        if (two)
                                            stg[off + __popc(em) + __popc(em2 & lt)] = gj_pair{b, a};
                                    }
                                }
                            }
                        }
                    }
                    __syncthreads();
                    // ---- commit when the staging area could not hold another tile
                    if (staged && H.stg_cnt > flush_at) {
                        if (tid == 0) {
                            uint32_t cnt = H.stg_cnt;
                            unsigned long long b = atomicAdd(&L.ctl->pos, (unsigned long long)cnt);
                            H.ok = (b + cnt <= L.cap);
                            H.base = b;
                            if (!H.ok) {
                                atomicMin(&L.ctl->fail_base, b);
                                atomicExch(&L.ctl->full, 1u);
                            }
                        }
                        __syncthreads();
                        if (H.ok) {
                            const uint32_t cnt = H.stg_cnt;
                            for (uint32_t i = tid; i < cnt; i += JT)
                                L.out[H.base + i] = stg[i];
                            commit_tile = tile_idx + 1;
                        } else if (tid == 0) {
                            H.stop = 1;
                        }
                        __syncthreads();
                        if (tid == 0)
                            H.stg_cnt = 0;
                    }
                }
            }
        }
        __syncthreads();
        // ---- end of item: commit the rest, or defer from the first uncommitted tile
        if (staged) {
            if (tid == 0 && !H.stop) {
                uint32_t cnt = H.stg_cnt;
                H.ok = 1;
                if (cnt) {
                    unsigned long long b = atomicAdd(&L.ctl->pos, (unsigned long long)cnt);
                    H.ok = (b + cnt <= L.cap);
                    H.base = b;
                    if (!H.ok) {
                        atomicMin(&L.ctl->fail_base, b);
                        atomicExch(&L.ctl->full, 1u);
                    }
                }
            }
            __syncthreads();
            if (!H.stop && H.ok) {
                const uint32_t cnt = H.stg_cnt;
                for (uint32_t i = tid; i < cnt; i += JT)
                    L.out[H.base + i] = stg[i];
            } else if (tid == 0) {
                uint32_t slot = atomicAdd(&L.ctl->dout_n, 1u);
                if (slot < L.dout_cap)
                    L.dout[slot] = Deferred{H.item, commit_tile};
                else
                    atomicOr(&L.ctl->err, kErrDeferred);
            }
            __syncthreads();
            if (tid == 0)
                H.stg_cnt = 0;
        }
    }

    // ---- per-CTA statistics
    for (int o = 16; o; o >>= 1) {
        my_count += __shfl_xor_sync(FULL, my_count, o);
        my_dims += __shfl_xor_sync(FULL, my_dims, o);
        my_pairs += __shfl_xor_sync(FULL, my_pairs, o);
    }
    if (lane == 0) {
        if (my_count)
            atomicAdd(&L.ctl->counted, my_count);
        atomicAdd(&L.ctl->dims, my_dims);
        atomicAdd(&L.ctl->evaluated, my_pairs);
    }
    if (tid == 0 && L.sm_span)
        note_sm_span(L.sm_span, (unsigned long long)H.t_start, globaltimer_ns());
}

// Query tile rows held in shared memory: 64 when the work items hold at most
// 64 points (a smaller footprint, more CTAs per SM at large d), else 128.
static int plain_qbt(int qb) { return qb > 0 && qb <= 64 ? 64 : QB; }

static size_t plain_smem(int d, int ct, int qbt)
{
    return ((sizeof(SmemHdr) + 15) & ~size_t(15)) + (size_t)d * (qbt + ct) * sizeof(double);
}

static int plain_ct(int d, int ct = 0) { return ct == 32 || ct == 64 ? ct : (d <= 32 ? 64 : 32); }

int plain_ctas_per_sm(int d, int ct_req, int qb)
{
    int ct = plain_ct(d, ct_req);
    size_t sm = plain_smem(d, ct, plain_qbt(qb));
    int per = (int)((227 * 1024) / (sm + 1024));
    if (per > 4)
        per = 4;
    return per < 1 ? 0 : per;
}

size_t plain_smem_bytes(int d, int ct, int qb) { return plain_smem(d, plain_ct(d, ct), plain_qbt(qb)); }

template <int CT, int QBT, bool DIRECT, bool ASYM>
static cudaError_t launch_one(const JoinLaunch &L, int grid, size_t sm, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_join_plain<CT, QBT, DIRECT, ASYM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess)
        return e;
    note_launch();
    k_join_plain<CT, QBT, DIRECT, ASYM><<<grid, JT, sm, s>>>(L);
    return cudaGetLastError();
}

template <bool DIRECT, bool ASYM>
static cudaError_t launch_by_shape(const JoinLaunch &L, int grid, cudaStream_t s)
{
    const int ct = plain_ct(L.ix.d, L.ix.ct);
    const int qbt = plain_qbt(L.ix.qb);
    const size_t sm = plain_smem(L.ix.d, ct, qbt);
    if (ct == 64)
        return qbt == 64 ? launch_one<64, 64, DIRECT, ASYM>(L, grid, sm, s)
                         : launch_one<64, QB, DIRECT, ASYM>(L, grid, sm, s);
    return qbt == 64 ? launch_one<32, 64, DIRECT, ASYM>(L, grid, sm, s)
                     : launch_one<32, QB, DIRECT, ASYM>(L, grid, sm, s);
}

cudaError_t launch_join_plain_direct(const JoinLaunch &L, int grid, cudaStream_t s)
{
    return L.ix.asym ? launch_by_shape<true, true>(L, grid, s) : launch_by_shape<true, false>(L, grid, s);
}

cudaError_t launch_join_plain(const JoinLaunch &L, int grid, cudaStream_t s)
{
    return launch_by_shape<false, false>(L, grid, s);
}

// ---------------------------------------------------------------------------
// FP64 pipe probe: independent DFMA chains, 8 per thread; returns nothing
// useful except through `out` (kept so the work is not optimised away).
// FLOPs = 2 * 8 * iters * threads.
// ---------------------------------------------------------------------------
__global__ void k_fp64_probe(double *out, int iters)
{
    double a0 = threadIdx.x * 1e-9, a1 = a0 + 1e-9, a2 = a0 + 2e-9, a3 = a0 + 3e-9;
    double a4 = a0 + 4e-9, a5 = a0 + 5e-9, a6 = a0 + 6e-9, a7 = a0 + 7e-9;
    const double m = 0.9999999, c = 1e-12;
    for (int i = 0; i < iters; ++i) {
        a0 = __fma_rn(a0, m, c);
        a1 = __fma_rn(a1, m, c);
        a2 = __fma_rn(a2, m, c);
        a3 = __fma_rn(a3, m, c);
        a4 = __fma_rn(a4, m, c);
        a5 = __fma_rn(a5, m, c);
        a6 = __fma_rn(a6, m, c);
        a7 = __fma_rn(a7, m, c);
    }
    double r = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
    if (r == 12345.678)
        out[blockIdx.x] = r;
}

cudaError_t launch_fp64_probe(double *out, int iters, int grid, cudaStream_t s)
{
    k_fp64_probe<<<grid, 256, 0, s>>>(out, iters);
    return cudaGetLastError();
}

}  // namespace gj
