// gj_index.cu -- index construction on the GPU (Alg. 1: reorderVariance,
// constructIndex) and the load-ordered work queue.
//
// Stages, each a kernel:
//   (a) REORDER (Sec. 4.2): per-dimension mean and population variance over all
//       points (two deterministic passes: fixed block partition, fixed
//       reduction order), dimensions sorted by descending variance.
//   (b) grid (Sec. 3.2.1, 4.1): cell coordinate floor((y - m_j) / w_j) of the
//       first k reordered dimensions, row-major linear id (dimension 0 most
//       significant, as in Fig. 1), stable LSD radix sort of the points by id
//       (after a stable sort by the SORTIDU coordinate, Sec. 4.3, so points are
//       ordered by u inside each cell), compaction of the non-empty cells.
//   (c) adjacent cells (Sec. 3.2.1, Fig. 1): for every non-empty cell, the 3^k
//       neighbouring ids are searched by binary search among the sorted
//       non-empty ids; only neighbours b >= a are kept (each unordered pair of
//       cells is joined once and both orientations are emitted).
//   (e) work items: query blocks of <= QB points of one cell, with an estimated
//       load |Q| * (points in the searched cells), sorted by descending load so
//       that a persistent join pulls the heaviest blocks first.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include "gj_internal.cuh"

namespace gj {

// ---------------------------------------------------------------------------
// Finite check
// ---------------------------------------------------------------------------
__global__ void k_check_finite(const double *__restrict__ P, int64_t count, unsigned int *flag)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (; i < count; i += stride) {
        unsigned long long b = (unsigned long long)__double_as_longlong(P[i]);
        bad |= ((b >> 52) & 0x7FF) == 0x7FF;   // Inf or NaN
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0)
        atomicOr(flag, 1u);
}

cudaError_t launch_check_finite(const double *P, int64_t count, unsigned int *flag, cudaStream_t s)
{
    if (count <= 0)
        return cudaSuccess;
    int64_t blocks = (count + 255) / 256;
    if (blocks > 4096)
        blocks = 4096;
    note_launch();
    k_check_finite<<<(int)blocks, 256, 0, s>>>(P, count, flag);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-dimension statistics: pass 0 -> sum/min/max, pass 1 -> sum of squared
// deviations from the mean.  Block b reduces rows [b*R, (b+1)*R) with a fixed
// partition and fixed reduction order, so the result is reproducible.
// part layout: [blk][d][3]
// ---------------------------------------------------------------------------
__global__ void k_dim_partial(const double *__restrict__ P, int64_t n, int d, int64_t rows_per_blk,
                              int pass, const double *__restrict__ mean, double *__restrict__ part)
{
    __shared__ double red[8][32][3];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t r0 = blockIdx.x * rows_per_blk;
    int64_t r1 = r0 + rows_per_blk;
    if (r1 > n)
        r1 = n;
    for (int j0 = 0; j0 < d; j0 += 32) {
        const int j = j0 + tx;
        double a = 0.0, mn = INFINITY, mx = -INFINITY;
        if (j < d) {
            const double m = pass ? mean[j] : 0.0;
            for (int64_t r = r0 + ty; r < r1; r += 8) {
                double v = P[r * d + j];
                if (pass) {
                    double t = v - m;
                    a += t * t;
                } else {
                    a += v;
                    mn = fmin(mn, v);
                    mx = fmax(mx, v);
                }
            }
        }
        red[ty][tx][0] = a;
        red[ty][tx][1] = mn;
        red[ty][tx][2] = mx;
        __syncthreads();
        if (ty == 0 && j < d) {
            double s = 0.0, lo = INFINITY, hi = -INFINITY;
            for (int y = 0; y < 8; ++y) {
                s += red[y][tx][0];
                lo = fmin(lo, red[y][tx][1]);
                hi = fmax(hi, red[y][tx][2]);
            }
            double *o = part + ((size_t)blockIdx.x * d + j) * 3;
            o[0] = s;
            o[1] = lo;
            o[2] = hi;
        }
        __syncthreads();
    }
}

// stats layout: [d][4] = mean, var, min, max.  One thread per dimension,
// blocks summed in index order.
__global__ void k_dim_final(const double *__restrict__ part, int nblk, int d, int64_t n, int pass,
                            double *__restrict__ stats)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d)
        return;
    double s = 0.0, lo = INFINITY, hi = -INFINITY;
    for (int b = 0; b < nblk; ++b) {
        const double *o = part + ((size_t)b * d + j) * 3;
        s += o[0];
        lo = fmin(lo, o[1]);
        hi = fmax(hi, o[2]);
    }
    if (pass == 0) {
        stats[j * 4 + 0] = s / (double)n;
        stats[j * 4 + 2] = lo;
        stats[j * 4 + 3] = hi;
    } else {
        stats[j * 4 + 1] = s / (double)n;
    }
}

cudaError_t launch_dim_stats(const double *P, int64_t n, int d, double *part, int nblk, double *stats,
                             cudaStream_t s)
{
    int64_t rows = (n + nblk - 1) / nblk;
    double *mean_col = nullptr;   // mean is read from stats[j*4], strided: copy into part tail
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            // gather means contiguously after the partials
            mean_col = part + (size_t)nblk * d * 3;
            cudaError_t e = cudaMemcpy2DAsync(mean_col, sizeof(double), stats, 4 * sizeof(double),
                                              sizeof(double), d, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess)
                return e;
        }
        note_launch();
        k_dim_partial<<<nblk, 256, 0, s>>>(P, n, d, rows, pass, mean_col, part);
        note_launch();
        k_dim_final<<<(d + 127) / 128, 128, 0, s>>>(part, nblk, d, n, pass, stats);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Keys
// ---------------------------------------------------------------------------
struct GridParams {
    int k;
    int d;
    int perm[MAXK];        // original column of reordered dimension j < k
    double origin[MAXK];
    double invw[MAXK];     // 1 / w_j (0: dimension not indexed)
    int64_t nc[MAXK];
    int64_t stride[MAXK];
};

__device__ __forceinline__ uint64_t orderable(double v)
{
    uint64_t b = (uint64_t)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// key[t] = orderable(P[t][col]), val[t] = t
__global__ void k_ukeys(const double *__restrict__ P, int64_t n, int d, int col,
                        uint64_t *__restrict__ key, uint32_t *__restrict__ val)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        key[i] = orderable(P[i * d + col]);
        val[i] = (uint32_t)i;
    }
}

__device__ __forceinline__ int64_t cell_coord(double y, double origin, double invw, int64_t nc)
{
    if (invw == 0.0)
        return 0;
    double t = __dmul_rn(__dsub_rn(y, origin), invw);
    int64_t c = (int64_t)floor(t);
    if (c < 0)
        c = 0;
    if (c >= nc)
        c = nc - 1;
    return c;
}

// ckey[t] = linear cell id of point val[t]; if val == nullptr the point is t.
__global__ void k_cellkeys(const double *__restrict__ P, int64_t n, GridParams g,
                           const uint32_t *__restrict__ val, uint64_t *__restrict__ key,
                           uint32_t *__restrict__ valout)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n)
        return;
    int64_t i = val ? (int64_t)val[t] : t;
    int64_t id = 0;
    for (int j = 0; j < g.k; ++j)
        id += cell_coord(P[i * g.d + g.perm[j]], g.origin[j], g.invw[j], g.nc[j]) * g.stride[j];
    key[t] = (uint64_t)id;
    if (!val)
        valout[t] = (uint32_t)t;
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort, 8 bits per pass.
// counts layout: [256][nblocks] (digit-major) followed by 256 digit totals.
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_PER_THREAD = 16;
constexpr int RS_TILE = RS_THREADS * RS_PER_THREAD;   // 4096 keys per block

__global__ void k_rs_count(const uint64_t *__restrict__ key, int64_t n, int shift,
                           uint32_t *__restrict__ counts, int nblocks)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_PER_THREAD; ++r) {
        int64_t i = base + r * RS_THREADS + threadIdx.x;
        if (i < n)
            atomicAdd(&h[(key[i] >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    counts[(size_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// one block per digit: exclusive scan of counts[digit][*]; total -> counts[256*nblocks + digit]
__global__ void k_rs_scan(uint32_t *__restrict__ counts, int nblocks)
{
    __shared__ uint32_t part[1024];
    uint32_t *row = counts + (size_t)blockIdx.x * nblocks;
    const int per = (nblocks + 1023) / 1024;
    const int b0 = threadIdx.x * per;
    uint32_t s = 0;
    for (int b = b0; b < b0 + per && b < nblocks; ++b)
        s += row[b];
    part[threadIdx.x] = s;
    __syncthreads();
    // Hillis-Steele inclusive scan over 1024 partials
    for (int off = 1; off < 1024; off <<= 1) {
        uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (int b = b0; b < b0 + per && b < nblocks; ++b) {
        uint32_t c = row[b];
        row[b] = run;
        run += c;
    }
    if (threadIdx.x == 1023)
        counts[(size_t)256 * nblocks + blockIdx.x] = part[1023];
}

__global__ void __launch_bounds__(RS_THREADS)
k_rs_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
             uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n, int shift,
             const uint32_t *__restrict__ counts, int nblocks)
{
    __shared__ uint32_t dbase[256];
    __shared__ uint32_t wcnt[RS_THREADS / 32][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // digit bases: exclusive scan of the 256 totals (small, done per block)
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        const uint32_t *tot = counts + (size_t)256 * nblocks;
        for (int dg = 0; dg < 256; ++dg) {
            dbase[dg] = run;
            run += tot[dg];
        }
    }
    for (int dg = lane; dg < 256; dg += 32)
        wcnt[w][dg] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)w * (32 * RS_PER_THREAD);
    uint32_t dig[RS_PER_THREAD], rk[RS_PER_THREAD];
    uint64_t kk[RS_PER_THREAD];
    uint32_t vv[RS_PER_THREAD];
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < RS_PER_THREAD; ++r) {
        int64_t i = base + r * 32 + lane;
        bool ok = i < n;
        uint64_t kv = ok ? kin[i] : ~0ull;
        uint32_t dg = ok ? (uint32_t)((kv >> shift) & 0xFF) : 256u;
        kk[r] = kv;
        vv[r] = ok ? vin[i] : 0u;
        unsigned peers = __match_any_sync(0xffffffffu, dg);
        uint32_t before = ok ? wcnt[w][dg] : 0u;
        rk[r] = before + __popc(peers & lt);
        dig[r] = dg;
        __syncwarp();
        if (ok && (peers & lt) == 0)
            wcnt[w][dg] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps, per digit
    {
        int dg = threadIdx.x;   // 256 threads == 256 digits
        uint32_t run = 0;
        for (int y = 0; y < RS_THREADS / 32; ++y) {
            uint32_t c = wcnt[y][dg];
            wcnt[y][dg] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int r = 0; r < RS_PER_THREAD; ++r) {
        uint32_t dg = dig[r];
        if (dg < 256) {
            uint32_t pos = dbase[dg] + counts[(size_t)dg * nblocks + blockIdx.x] + wcnt[w][dg] + rk[r];
            kout[pos] = kk[r];
            vout[pos] = vv[r];
        }
    }
}

int64_t radix_counts_needed(int64_t n)
{
    int64_t nb = (n + RS_TILE - 1) / RS_TILE;
    return 256 * (nb > 0 ? nb : 1) + 256;
}

cudaError_t radix_sort_pairs(uint64_t *k0, uint32_t *v0, uint64_t *k1, uint32_t *v1, int64_t n,
                             int lo, int hi, uint32_t *counts, int64_t counts_cap, cudaStream_t s)
{
    if (n <= 1 || hi <= lo)
        return cudaSuccess;
    int nblocks = (int)((n + RS_TILE - 1) / RS_TILE);
    if (radix_counts_needed(n) > counts_cap)
        return cudaErrorInvalidValue;
    uint64_t *ka = k0, *kb = k1;
    uint32_t *va = v0, *vb = v1;
    int passes = 0;
    for (int shift = lo; shift < hi; shift += 8) {
        note_launch();
        k_rs_count<<<nblocks, RS_THREADS, 0, s>>>(ka, n, shift, counts, nblocks);
        note_launch();
        k_rs_scan<<<256, 1024, 0, s>>>(counts, nblocks);
        note_launch();
        k_rs_scatter<<<nblocks, RS_THREADS, 0, s>>>(ka, va, kb, vb, n, shift, counts, nblocks);
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
        ++passes;
    }
    if (passes & 1) {
        cudaMemcpyAsync(k0, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(v0, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Exclusive scan of int64 (in place), 4096 elements per block, recursive.
// tmp must hold scan_tmp_needed(n) elements.
// ---------------------------------------------------------------------------
constexpr int SC_THREADS = 1024;
constexpr int SC_PER = 4;
constexpr int SC_TILE = SC_THREADS * SC_PER;

__global__ void k_scan_block(int64_t *__restrict__ data, int64_t n, int64_t *__restrict__ sums)
{
    __shared__ int64_t part[SC_THREADS];
    const int64_t b0 = (int64_t)blockIdx.x * SC_TILE + threadIdx.x * SC_PER;
    int64_t v[SC_PER];
    int64_t s = 0;
    for (int r = 0; r < SC_PER; ++r) {
        v[r] = (b0 + r < n) ? data[b0 + r] : 0;
        s += v[r];
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < SC_THREADS; off <<= 1) {
        int64_t t = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += t;
        __syncthreads();
    }
    int64_t run = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (int r = 0; r < SC_PER; ++r) {
        if (b0 + r < n)
            data[b0 + r] = run;
        run += v[r];
    }
    if (threadIdx.x == SC_THREADS - 1 && sums)
        sums[blockIdx.x] = part[SC_THREADS - 1];
}

__global__ void k_scan_add(int64_t *__restrict__ data, int64_t n, const int64_t *__restrict__ sums)
{
    const int64_t b0 = (int64_t)blockIdx.x * SC_TILE;
    const int64_t add = sums[blockIdx.x];
    for (int r = threadIdx.x; r < SC_TILE; r += SC_THREADS)
        if (b0 + r < n)
            data[b0 + r] += add;
}

int64_t scan_tmp_needed(int64_t n)
{
    int64_t need = 0;
    while (n > SC_TILE) {
        n = (n + SC_TILE - 1) / SC_TILE;
        need += n + 1;
    }
    return need + 1;
}

cudaError_t exclusive_scan_i64(int64_t *data, int64_t n, int64_t *tmp, int64_t tmp_cap, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    int64_t nb = (n + SC_TILE - 1) / SC_TILE;
    if (nb == 1) {
        note_launch();
        k_scan_block<<<1, SC_THREADS, 0, s>>>(data, n, nullptr);
        return cudaGetLastError();
    }
    if (tmp_cap < nb + 1)
        return cudaErrorInvalidValue;
    note_launch();
    k_scan_block<<<(int)nb, SC_THREADS, 0, s>>>(data, n, tmp);
    cudaError_t e = exclusive_scan_i64(tmp, nb, tmp + nb + 1, tmp_cap - nb - 1, s);
    if (e != cudaSuccess)
        return e;
    note_launch();
    k_scan_add<<<(int)nb, SC_THREADS, 0, s>>>(data, n, tmp);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gather points into the sorted, reordered, structure-of-arrays layout.
// A block moves 32 sorted positions: rows are read coalesced into shared
// memory, columns written coalesced.
// ---------------------------------------------------------------------------
__global__ void k_gather_soa(const double *__restrict__ P, int64_t n, int d, int64_t npad,
                             const uint32_t *__restrict__ order, const int *__restrict__ perm,
                             double *__restrict__ X, uint32_t *__restrict__ orig)
{
    __shared__ double tile[32][65];
    const int64_t p0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 256 threads: 8 x 32
    for (int j0 = 0; j0 < d; j0 += 64) {
        const int dj = min(64, d - j0);
        // load: row p0+r, reordered dims j0..j0+dj
        for (int r = ty; r < 32; r += 8) {
            int64_t p = p0 + r;
            if (p < n) {
                const double *row = P + (int64_t)order[p] * d;
                for (int c = tx; c < dj; c += 32)
                    tile[r][c] = row[perm[j0 + c]];
            }
        }
        __syncthreads();
        for (int c = ty; c < dj; c += 8) {
            int64_t p = p0 + tx;
            if (p < n)
                X[(int64_t)(j0 + c) * npad + p] = tile[tx][c];
        }
        __syncthreads();
    }
    if (threadIdx.x < 32 && p0 + threadIdx.x < n)
        orig[p0 + threadIdx.x] = order[p0 + threadIdx.x];
}

// ---------------------------------------------------------------------------
// Cells
// ---------------------------------------------------------------------------
__global__ void k_heads(const uint64_t *__restrict__ key, int64_t n, int64_t *__restrict__ flag)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n)
        flag[i] = (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
}

// flag holds the exclusive scan of the head flags
__global__ void k_cells(const uint64_t *__restrict__ key, int64_t n, const int64_t *__restrict__ pre,
                        int64_t *__restrict__ cell_start, int64_t *__restrict__ cell_id)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && (i == 0 || key[i] != key[i - 1])) {
        cell_start[pre[i]] = i;
        cell_id[pre[i]] = (int64_t)key[i];
    }
}

__global__ void k_set_i64(int64_t *p, int64_t v) { *p = v; }

// ---------------------------------------------------------------------------
// Adjacent non-empty cells (b >= a), one warp per cell.  Offsets t in
// [0, 3^k) are read as base-3 digits (dimension 0 most significant), each
// digit minus one giving the step in that dimension.
// mode 0: count and sum neighbour sizes; mode 1: write the list.
// ---------------------------------------------------------------------------
struct AdjParams {
    int k;
    int64_t nc[MAXK];
    int64_t stride[MAXK];
    int64_t pow3;
};

__device__ __forceinline__ int64_t find_id(const int64_t *__restrict__ ids, int64_t G, int64_t x)
{
    int64_t lo = 0, hi = G;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (ids[mid] < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < G && ids[lo] == x) ? lo : -1;
}

__global__ void k_adjacent(const int64_t *__restrict__ cell_id, const int64_t *__restrict__ cell_start,
                           int64_t G, AdjParams a, int mode, int64_t *__restrict__ cnt,
                           int64_t *__restrict__ nbsum, const int64_t *__restrict__ adj_start,
                           uint32_t *__restrict__ adj)
{
    const int lane = threadIdx.x & 31;
    const int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (c >= G)
        return;
    const int64_t id = cell_id[c];
    int64_t coord[MAXK];
    for (int j = 0; j < a.k; ++j)
        coord[j] = (id / a.stride[j]) % a.nc[j];
    int64_t found = 0, sz = 0;
    int64_t out = mode ? adj_start[c] : 0;
    for (int64_t t0 = 0; t0 < a.pow3; t0 += 32) {
        int64_t t = t0 + lane;
        int64_t b = -1;
        if (t < a.pow3) {
            int64_t r = t, nid = 0;
            bool ok = true;
            for (int j = a.k - 1; j >= 0; --j) {
                int64_t cj = coord[j] + (r % 3) - 1;
                r /= 3;
                ok &= (cj >= 0 && cj < a.nc[j]);
                nid += cj * a.stride[j];
            }
            if (ok)
                b = find_id(cell_id, G, nid);
            if (b < c)
                b = -1;
        }
        unsigned m = __ballot_sync(0xffffffffu, b >= 0);
        if (b >= 0) {
            if (mode)
                adj[out + found + __popc(m & ((1u << lane) - 1u))] = (uint32_t)b;
            else if (b != c)
                sz += cell_start[b + 1] - cell_start[b];
        }
        found += __popc(m);
    }
    if (!mode) {
        for (int o = 16; o; o >>= 1)
            sz += __shfl_xor_sync(0xffffffffu, sz, o);
        if (lane == 0) {
            cnt[c] = found;
            nbsum[c] = sz;
        }
    }
}

// Similarity join: the entry cells adjacent to each query cell (all of them,
// no symmetry), one warp per query cell.  mode 0: count and sum the entry
// cells' sizes; mode 1: write the list.
__global__ void k_adjacent_qe(const int64_t *__restrict__ qcell_id, int64_t Gq, const int64_t *__restrict__ cell_id,
                              const int64_t *__restrict__ cell_start, int64_t G, AdjParams a, int mode,
                              int64_t *__restrict__ cnt, int64_t *__restrict__ nbsum,
                              const int64_t *__restrict__ adj_start, uint32_t *__restrict__ adj)
{
    const int lane = threadIdx.x & 31;
    const int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (c >= Gq)
        return;
    const int64_t id = qcell_id[c];
    int64_t coord[MAXK];
    for (int j = 0; j < a.k; ++j)
        coord[j] = (id / a.stride[j]) % a.nc[j];
    int64_t found = 0, sz = 0;
    const int64_t out = mode ? adj_start[c] : 0;
    for (int64_t t0 = 0; t0 < a.pow3; t0 += 32) {
        const int64_t t = t0 + lane;
        int64_t b = -1;
        if (t < a.pow3) {
            int64_t r = t, nid = 0;
            bool ok = true;
            for (int j = a.k - 1; j >= 0; --j) {
                const int64_t cj = coord[j] + (r % 3) - 1;
                r /= 3;
                ok &= (cj >= 0 && cj < a.nc[j]);
                nid += cj * a.stride[j];
            }
            if (ok)
                b = find_id(cell_id, G, nid);
        }
        const unsigned m = __ballot_sync(0xffffffffu, b >= 0);
        if (b >= 0) {
            if (mode)
                adj[out + found + __popc(m & ((1u << lane) - 1u))] = (uint32_t)b;
            else
                sz += cell_start[b + 1] - cell_start[b];
        }
        found += __popc(m);
    }
    if (!mode) {
        for (int o = 16; o; o >>= 1)
            sz += __shfl_xor_sync(0xffffffffu, sz, o);
        if (lane == 0) {
            cnt[c] = found;
            nbsum[c] = sz;
        }
    }
}

// ---------------------------------------------------------------------------
// Work items
// ---------------------------------------------------------------------------
// Items of a cell: blocks of qb points from the cell's start, or (align > 0)
// the pieces of the cell between multiples of align in sorted position, so
// that every block but a cell's first starts on a multiple of align.
__global__ void k_item_counts(const int64_t *__restrict__ cell_start, int64_t G, int qb, int align,
                              int64_t *__restrict__ cnt)
{
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c < G) {
        const int64_t s = cell_start[c], e = cell_start[c + 1];
        if (align > 0)
            cnt[c] = e > s ? (e - 1) / align - s / align + 1 : 0;
        else
            cnt[c] = (e - s + qb - 1) / qb;
    }
}

// items of cell c at [istart[c], ...); cost key = ~float bits of the load
// estimate (ascending key = descending load); also sums candidate pairs.
// One warp per cell, its lanes taking the cell's items in turn (a large
// cell holds thousands of items).
__global__ void k_items(const int64_t *__restrict__ cell_start, int64_t G, int qb, int align,
                        const int64_t *__restrict__ istart, const int64_t *__restrict__ nbsum,
                        Item *__restrict__ items, uint64_t *__restrict__ key, uint32_t *__restrict__ val,
                        unsigned long long *__restrict__ cand)
{
    const int lane = threadIdx.x & 31;
    const int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (c >= G)
        return;
    const int64_t s = cell_start[c], e = cell_start[c + 1], len = e - s;
    const int64_t nb = nbsum[c];
    const int64_t cnt = align > 0 ? (len > 0 ? (e - 1) / align - s / align + 1 : 0) : (len + qb - 1) / qb;
    for (int64_t i = lane; i < cnt; i += 32) {
        int64_t q, qe;
        if (align > 0) {
            q = i == 0 ? s : (s / align + i) * align;
            qe = min(e, (s / align + i + 1) * align);
        } else {
            q = s + i * qb;
            qe = min(e, q + qb);
        }
        const int64_t it = istart[c] + i;
        const uint32_t ql = (uint32_t)(qe - q);
        items[it] = Item{(uint32_t)c, (uint32_t)q, ql, 0u};
        const float load = (float)ql * (float)(nb + (e - q));
        key[it] = (uint64_t)(~__float_as_uint(load));
        val[it] = (uint32_t)it;
    }
    if (lane == 0)
        atomicAdd(cand, (unsigned long long)(len * (len - 1) / 2) + (unsigned long long)(len * nb));
}

// Similarity join: query blocks of qb points per query cell; load = block
// size x points of the adjacent entry cells; candidate pairs = |Q cell| x
// points of the adjacent entry cells.
__global__ void k_qe_items(const int64_t *__restrict__ qcell_start, int64_t Gq, int qb,
                           const int64_t *__restrict__ istart, const int64_t *__restrict__ nbsum,
                           Item *__restrict__ items, uint64_t *__restrict__ key, uint32_t *__restrict__ val,
                           unsigned long long *__restrict__ cand)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= Gq)
        return;
    const int64_t s = qcell_start[c], e = qcell_start[c + 1];
    const int64_t nb = nbsum[c];
    int64_t it = istart[c];
    for (int64_t q = s; q < e; q += qb, ++it) {
        const uint32_t ql = (uint32_t)min((int64_t)qb, e - q);
        items[it] = Item{(uint32_t)c, (uint32_t)q, ql, 0u};
        const float load = (float)ql * (float)nb;
        key[it] = (uint64_t)(~__float_as_uint(load));
        val[it] = (uint32_t)it;
    }
    atomicAdd(cand, (unsigned long long)((e - s) * nb));
}

// ---------------------------------------------------------------------------
// Host orchestration of the build.
// ---------------------------------------------------------------------------
#define GJ_TRY(x)                                                                           \
    do {                                                                                    \
        cudaError_t _e = (x);                                                               \
        if (_e != cudaSuccess) {                                                            \
            st = (_e == cudaErrorMemoryAllocation) ? GJ_ERR_OOM : GJ_ERR_CUDA;              \
            goto done;                                                                      \
        }                                                                                   \
    } while (0)

static int64_t grid_blocks(int64_t n, int t) { return (n + t - 1) / t; }

// Choice of k when the caller passes 0 (Sec. 4.1 trade-off, Sec. 5.4 cost
// comparison): per candidate k, the candidate pairs under a uniform-density
// model (each indexed dimension keeps at most 3 of nc_j cells) against the
// index search cost |G| * 3^k * log2|G|; the cheaper wins.
static int choose_k(int d, const std::vector<int64_t> &nc_all, int64_t n, int kmax)
{
    double best = INFINITY;
    int bk = 1;
    double frac = 1.0, cells = 1.0;
    for (int k = 1; k <= kmax && k <= d; ++k) {
        double ncj = (double)nc_all[k - 1];
        frac *= std::min(1.0, 3.0 / ncj);
        cells = std::min((double)n, cells * ncj);
        double pairs = 0.5 * (double)n * (double)n * frac;
        double search = cells * pow(3.0, k) * log2(std::max(2.0, cells));
        double cost = pairs * 4.0 + search * 8.0;
        if (cost < best * 0.98) {
            best = cost;
            bk = k;
        }
    }
    return bk;
}

int build_index(gj_index *h, const double *P, int64_t n, int d, double eps, int k_req,
                uint32_t flags, cudaStream_t s)
{
    int st = GJ_OK;
    const int nblk_stats = (int)std::max<int64_t>(1, std::min<int64_t>(1024, (n + 2047) / 2048));
    double *part = nullptr, *stats = nullptr;
    uint64_t *k0 = nullptr, *k1 = nullptr;
    uint32_t *v0 = nullptr, *v1 = nullptr, *counts = nullptr;
    int64_t *flagbuf = nullptr, *tmp = nullptr, *cnt = nullptr, *nbsum = nullptr;
    int *perm_dev = nullptr;
    unsigned long long *cand_dev = nullptr;
    int64_t counts_cap = 0, tmp_cap = 0, G = 0, nitems = 0, nadj = 0;
    std::vector<double> hs((size_t)d * 4);
    std::vector<int> perm(d);
    GridParams gp{};
    AdjParams ap{};
    int k = 0;
    const int64_t maxn = std::max<int64_t>(n, 1);

    h->npad = ((n + 31) / 32) * 32;
    if (h->npad == 0)
        h->npad = 32;

    // (a) REORDER statistics
    GJ_TRY(dev_alloc(&part, ((size_t)nblk_stats * d * 3 + d) * sizeof(double), s));
    GJ_TRY(dev_alloc(&stats, (size_t)d * 4 * sizeof(double), s));
    if (n > 0) {
        GJ_TRY(launch_dim_stats(P, n, d, part, nblk_stats, stats, s));
        GJ_TRY(cudaMemcpyAsync(hs.data(), stats, (size_t)d * 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
        GJ_TRY(cudaStreamSynchronize(s));
    } else {
        std::fill(hs.begin(), hs.end(), 0.0);
    }
    for (int j = 0; j < d; ++j)
        perm[j] = j;
    if (flags & GJ_REORDER)
        std::stable_sort(perm.begin(), perm.end(),
                         [&](int a, int b) { return hs[(size_t)a * 4 + 1] > hs[(size_t)b * 4 + 1]; });
    for (int j = 0; j < d; ++j)
        h->info.perm[j] = perm[j];

    // (b) grid geometry on the host (k, widths, cell counts, strides)
    {
        const double w0 = eps * (1.0 + ldexp(1.0, -24));
        std::vector<int64_t> nc_all(std::min(d, MAXK));
        std::vector<double> invw_all(nc_all.size()), org_all(nc_all.size());
        for (size_t j = 0; j < nc_all.size(); ++j) {
            double lo = hs[(size_t)perm[j] * 4 + 2], hi = hs[(size_t)perm[j] * 4 + 3];
            double range = hi - lo;
            org_all[j] = lo;
            if (!(range < 1e300) || n == 0) {
                nc_all[j] = 1;
                invw_all[j] = 0.0;
                continue;
            }
            double w = std::max(w0, range * ldexp(1.0, -24));
            double iw = 1.0 / w;
            double tmax = (range)*iw;   // same rounding shape as the kernel: fl(fl(M-m)*iw)
            int64_t cmax = (int64_t)floor(tmax);
            nc_all[j] = cmax + 1;
            invw_all[j] = (nc_all[j] > 1) ? iw : 0.0;
            if (nc_all[j] == 1)
                invw_all[j] = 0.0;
        }
        const bool tc = (flags & GJ_TC_FILTER) && ((d + 4 + 15) / 16) * 16 <= 128;
        // tensor-core form, default blocks: pieces of a cell between multiples of
        // 128 positions, so that the 128-row A tile starts at the block itself
        h->q_align = (tc && h->cfg.query_block == 0) ? QB : 0;
        h->qb = h->q_align ? QB : (tc ? QB_TC : QB_PLAIN);
        // plain form above 32 dimensions: blocks of 64, so the query tile
        // (d x 64 doubles) leaves room for four CTAs per SM
        if (!tc && d > 32 && h->cfg.query_block == 0)
            h->qb = 64;
        if (h->cfg.query_block > 0)
            h->qb = std::min(h->cfg.query_block, tc ? QB_TC : QB);
        h->plain_ct = tc ? 0 : h->cfg.tile;
        int kmax = std::min(d, MAXK);
        // the tensor-core filter wants large cells (full 128 x 128 tiles): index at most 3 dims
        k = (k_req > 0) ? std::min(k_req, kmax) : choose_k(d, nc_all, n, tc ? std::min(kmax, 3) : kmax);
        // cap k so the linear id fits in 62 bits
        while (k > 0) {
            long double prod = 1.0L;
            for (int j = 0; j < k; ++j)
                prod *= (long double)nc_all[j];
            if (prod < 4.0e18L)
                break;
            --k;
        }
        gp.k = k;
        gp.d = d;
        int64_t strd = 1;
        for (int j = k - 1; j >= 0; --j) {
            gp.perm[j] = perm[j];
            gp.origin[j] = org_all[j];
            gp.invw[j] = invw_all[j];
            gp.nc[j] = nc_all[j];
            gp.stride[j] = strd;
            strd *= nc_all[j];
        }
        ap.k = k;
        ap.pow3 = 1;
        for (int j = 0; j < k; ++j) {
            ap.nc[j] = gp.nc[j];
            ap.stride[j] = gp.stride[j];
            ap.pow3 *= 3;
        }
        h->info.k = k;
        int bits = 0;
        while (bits < 63 && (((int64_t)1 << bits) < strd))
            ++bits;
        h->grid_k = k;
        h->grid_bits = bits;
        for (int j = 0; j < MAXK; ++j) {
            h->grid_perm[j] = j < k ? gp.perm[j] : 0;
            h->grid_origin[j] = j < k ? gp.origin[j] : 0.0;
            h->grid_invw[j] = j < k ? gp.invw[j] : 0.0;
            h->grid_nc[j] = j < k ? gp.nc[j] : 1;
            h->grid_stride[j] = j < k ? gp.stride[j] : 0;
        }
        // SORTIDU dimension: first un-indexed reordered dimension (or 0 when k == d)
        h->u = (flags & GJ_SORTIDU) ? (k < d ? k : 0) : -1;
        h->info.sortidu_dim = h->u;

        // key buffers
        counts_cap = radix_counts_needed(maxn);
        GJ_TRY(dev_alloc(&k0, maxn * sizeof(uint64_t), s));
        GJ_TRY(dev_alloc(&k1, maxn * sizeof(uint64_t), s));
        GJ_TRY(dev_alloc(&v0, maxn * sizeof(uint32_t), s));
        GJ_TRY(dev_alloc(&v1, maxn * sizeof(uint32_t), s));
        GJ_TRY(dev_alloc(&counts, counts_cap * sizeof(uint32_t), s));
        GJ_TRY(dev_alloc(&perm_dev, d * sizeof(int), s));
        GJ_TRY(cudaMemcpyAsync(perm_dev, perm.data(), d * sizeof(int), cudaMemcpyHostToDevice, s));

        if (n > 0) {
            const uint32_t *vin = nullptr;
            if (h->u >= 0) {
                note_launch();
                k_ukeys<<<(int)grid_blocks(n, 256), 256, 0, s>>>(P, n, d, perm[h->u], k0, v0);
                GJ_TRY(cudaGetLastError());
                GJ_TRY(radix_sort_pairs(k0, v0, k1, v1, n, 0, 64, counts, counts_cap, s));
                // v0 = point ids ordered by u; cell keys in that order (v1 gets a copy)
                GJ_TRY(cudaMemcpyAsync(v1, v0, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
                vin = v1;
                note_launch();
                k_cellkeys<<<(int)grid_blocks(n, 256), 256, 0, s>>>(P, n, gp, vin, k0, nullptr);
            } else {
                note_launch();
                k_cellkeys<<<(int)grid_blocks(n, 256), 256, 0, s>>>(P, n, gp, nullptr, k0, v0);
            }
            GJ_TRY(cudaGetLastError());
            GJ_TRY(radix_sort_pairs(k0, v0, k1, v1, n, 0, ((bits + 7) / 8) * 8, counts, counts_cap, s));
        }

        // sorted SoA points
        GJ_TRY(dev_alloc(&h->X, (size_t)d * h->npad * sizeof(double), s));
        GJ_TRY(dev_alloc(&h->orig, maxn * sizeof(uint32_t), s));
        GJ_TRY(cudaMemsetAsync(h->X, 0, (size_t)d * h->npad * sizeof(double), s));
        if (n > 0) {
            note_launch();
            k_gather_soa<<<(int)grid_blocks(n, 32), 256, 0, s>>>(P, n, d, h->npad, v0, perm_dev, h->X, h->orig);
            GJ_TRY(cudaGetLastError());
        }

        // (b) non-empty cells
        tmp_cap = scan_tmp_needed(maxn) + 64;
        GJ_TRY(dev_alloc(&tmp, tmp_cap * sizeof(int64_t), s));
        GJ_TRY(dev_alloc(&flagbuf, (maxn + 1) * sizeof(int64_t), s));
        if (n > 0) {
            note_launch();
            k_heads<<<(int)grid_blocks(n, 256), 256, 0, s>>>(k0, n, flagbuf);
            int64_t last_flag = 0;
            GJ_TRY(cudaMemcpyAsync(&last_flag, flagbuf + n - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            GJ_TRY(exclusive_scan_i64(flagbuf, n, tmp, tmp_cap, s));
            int64_t last_pre = 0;
            GJ_TRY(cudaMemcpyAsync(&last_pre, flagbuf + n - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            GJ_TRY(cudaStreamSynchronize(s));
            G = last_pre + last_flag;
        }
        h->G = G;
        GJ_TRY(dev_alloc(&h->cell_start, (G + 1) * sizeof(int64_t), s));
        GJ_TRY(dev_alloc(&h->cell_id, std::max<int64_t>(G, 1) * sizeof(int64_t), s));
        if (n > 0) {
            note_launch();
            k_cells<<<(int)grid_blocks(n, 256), 256, 0, s>>>(k0, n, flagbuf, h->cell_start, h->cell_id);
            note_launch();
            k_set_i64<<<1, 1, 0, s>>>(h->cell_start + G, n);
            GJ_TRY(cudaGetLastError());
        } else {
            note_launch();
            k_set_i64<<<1, 1, 0, s>>>(h->cell_start, 0);
        }

        // (c) adjacency
        GJ_TRY(dev_alloc(&cnt, (G + 1) * sizeof(int64_t), s));
        GJ_TRY(dev_alloc(&nbsum, std::max<int64_t>(G, 1) * sizeof(int64_t), s));
        GJ_TRY(dev_alloc(&h->adj_start, (G + 1) * sizeof(int64_t), s));
        if (G > 0) {
            int64_t thr = G * 32;
            note_launch();
            k_adjacent<<<(int)grid_blocks(thr, 256), 256, 0, s>>>(h->cell_id, h->cell_start, G, ap, 0, cnt,
                                                                  nbsum, nullptr, nullptr);
            GJ_TRY(cudaGetLastError());
            GJ_TRY(cudaMemcpyAsync(h->adj_start, cnt, G * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
            int64_t last_cnt = 0, last_pre = 0;
            GJ_TRY(cudaMemcpyAsync(&last_cnt, cnt + G - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            GJ_TRY(exclusive_scan_i64(h->adj_start, G, tmp, tmp_cap, s));
            GJ_TRY(cudaMemcpyAsync(&last_pre, h->adj_start + G - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            GJ_TRY(cudaStreamSynchronize(s));
            nadj = last_pre + last_cnt;
            h->nadj = nadj;
            note_launch();
            k_set_i64<<<1, 1, 0, s>>>(h->adj_start + G, nadj);
            GJ_TRY(dev_alloc(&h->adj, std::max<int64_t>(nadj, 1) * sizeof(uint32_t), s));
            note_launch();
            k_adjacent<<<(int)grid_blocks(thr, 256), 256, 0, s>>>(h->cell_id, h->cell_start, G, ap, 1, nullptr,
                                                                  nullptr, h->adj_start, h->adj);
            GJ_TRY(cudaGetLastError());
        } else {
            note_launch();
            k_set_i64<<<1, 1, 0, s>>>(h->adj_start, 0);
            GJ_TRY(dev_alloc(&h->adj, sizeof(uint32_t), s));
        }

        // (e) items, ordered by descending load
        GJ_TRY(dev_alloc(&cand_dev, sizeof(unsigned long long), s));
        GJ_TRY(cudaMemsetAsync(cand_dev, 0, sizeof(unsigned long long), s));
        if (G > 0) {
            note_launch();
            k_item_counts<<<(int)grid_blocks(G, 256), 256, 0, s>>>(h->cell_start, G, h->qb, h->q_align, cnt);
            int64_t last_cnt = 0, last_pre = 0;
            GJ_TRY(cudaMemcpyAsync(&last_cnt, cnt + G - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            GJ_TRY(exclusive_scan_i64(cnt, G, tmp, tmp_cap, s));
            GJ_TRY(cudaMemcpyAsync(&last_pre, cnt + G - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            GJ_TRY(cudaStreamSynchronize(s));
            nitems = last_pre + last_cnt;
        }
        h->nitems = nitems;
        GJ_TRY(dev_alloc(&h->items, std::max<int64_t>(nitems, 1) * sizeof(Item), s));
        GJ_TRY(dev_alloc(&h->order, std::max<int64_t>(nitems, 1) * sizeof(uint32_t), s));
        if (nitems > 0) {
            if (nitems > maxn) {   // cannot happen (items <= points), guard the key buffers
                st = GJ_ERR_CUDA;
                goto done;
            }
            note_launch();
            k_items<<<(int)grid_blocks(G * 32, 256), 256, 0, s>>>(h->cell_start, G, h->qb, h->q_align, cnt, nbsum,
                                                                  h->items, k0, v0, cand_dev);
            GJ_TRY(cudaGetLastError());
            GJ_TRY(radix_sort_pairs(k0, v0, k1, v1, nitems, 0, 32, counts, counts_cap, s));
            GJ_TRY(cudaMemcpyAsync(h->order, v0, nitems * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
        }
        unsigned long long cand = 0;
        GJ_TRY(cudaMemcpyAsync(&cand, cand_dev, sizeof(cand), cudaMemcpyDeviceToHost, s));
        GJ_TRY(cudaStreamSynchronize(s));
        h->info.candidate_pairs = cand;
        if ((flags & GJ_TC_FILTER) && n > 0) {
            st = tc_prepare(h, hs.data(), perm.data(), s);
            if (st != GJ_OK)
                goto done;
        }
    }
    h->info.nonempty_cells = G;
    h->info.work_items = nitems;

done:
    dev_free(part, s);
    dev_free(stats, s);
    dev_free(k0, s);
    dev_free(k1, s);
    dev_free(v0, s);
    dev_free(v1, s);
    dev_free(counts, s);
    dev_free(flagbuf, s);
    dev_free(tmp, s);
    dev_free(cnt, s);
    dev_free(nbsum, s);
    if (st == GJ_OK && !h->perm_dev) {
        h->perm_dev = perm_dev;   // kept: a similarity join gathers its queries with it
        perm_dev = nullptr;
    }
    dev_free(perm_dev, s);
    dev_free(cand_dev, s);
    return st;
}

void free_query_side(QuerySide *qs, cudaStream_t s)
{
    dev_free(qs->XQ, s);
    dev_free(qs->qorig, s);
    dev_free(qs->qcell_start, s);
    dev_free(qs->qcell_id, s);
    dev_free(qs->adj_start, s);
    dev_free(qs->adj, s);
    dev_free(qs->items, s);
    dev_free(qs->order, s);
    *qs = QuerySide{};
}

// The query side of Q join_eps E over the entry index h: queries (device,
// row-major nq x d, finite) keyed into the entry grid exactly as entries are
// (cell_coord clamps a coordinate into [0, nc): a query within eps of an entry
// is at most one cell away from it before the clamp, and clamping keeps it so),
// sorted by (cell, u), gathered into the REORDER structure-of-arrays layout;
// query cells, their adjacent entry cells, and load-ordered work items of at
// most qb queries.
int build_query_side(const gj_index *h, const double *Q, int64_t nq, int qb, QuerySide *qs, cudaStream_t s)
{
    int st = GJ_OK;
    const int d = h->info.d;
    const int64_t maxn = std::max<int64_t>(nq, 1);
    uint64_t *k0 = nullptr, *k1 = nullptr;
    uint32_t *v0 = nullptr, *v1 = nullptr, *counts = nullptr;
    int64_t *flagbuf = nullptr, *tmp = nullptr, *cnt = nullptr, *nbsum = nullptr;
    unsigned long long *cand_dev = nullptr;
    int64_t Gq = 0, nitems = 0, nadj = 0;
    GridParams gp{};
    AdjParams ap{};
    gp.k = h->grid_k;
    gp.d = d;
    ap.k = h->grid_k;
    ap.pow3 = 1;
    for (int j = 0; j < h->grid_k; ++j) {
        gp.perm[j] = h->grid_perm[j];
        gp.origin[j] = h->grid_origin[j];
        gp.invw[j] = h->grid_invw[j];
        gp.nc[j] = h->grid_nc[j];
        gp.stride[j] = h->grid_stride[j];
        ap.nc[j] = gp.nc[j];
        ap.stride[j] = gp.stride[j];
        ap.pow3 *= 3;
    }
    *qs = QuerySide{};
    qs->nq = nq;
    qs->qnpad = std::max<int64_t>(32, ((nq + 31) / 32) * 32);
    const int64_t counts_cap = radix_counts_needed(maxn);
    const int64_t tmp_cap = scan_tmp_needed(maxn + 1) + 64;
    GJ_TRY(dev_alloc(&k0, maxn * sizeof(uint64_t), s));
    GJ_TRY(dev_alloc(&k1, maxn * sizeof(uint64_t), s));
    GJ_TRY(dev_alloc(&v0, maxn * sizeof(uint32_t), s));
    GJ_TRY(dev_alloc(&v1, maxn * sizeof(uint32_t), s));
    GJ_TRY(dev_alloc(&counts, counts_cap * sizeof(uint32_t), s));
    GJ_TRY(dev_alloc(&tmp, tmp_cap * sizeof(int64_t), s));
    GJ_TRY(dev_alloc(&flagbuf, (maxn + 1) * sizeof(int64_t), s));
    GJ_TRY(dev_alloc(&cand_dev, sizeof(unsigned long long), s));
    GJ_TRY(cudaMemsetAsync(cand_dev, 0, sizeof(unsigned long long), s));
    // (1) keys: cell of the entry grid, then the SORTIDU coordinate inside a cell
    if (nq > 0) {
        if (h->u >= 0) {
            note_launch();
            k_ukeys<<<(int)grid_blocks(nq, 256), 256, 0, s>>>(Q, nq, d, h->info.perm[h->u], k0, v0);
            GJ_TRY(cudaGetLastError());
            GJ_TRY(radix_sort_pairs(k0, v0, k1, v1, nq, 0, 64, counts, counts_cap, s));
            GJ_TRY(cudaMemcpyAsync(v1, v0, nq * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
            note_launch();
            k_cellkeys<<<(int)grid_blocks(nq, 256), 256, 0, s>>>(Q, nq, gp, v1, k0, nullptr);
        } else {
            note_launch();
            k_cellkeys<<<(int)grid_blocks(nq, 256), 256, 0, s>>>(Q, nq, gp, nullptr, k0, v0);
        }
        GJ_TRY(cudaGetLastError());
        GJ_TRY(radix_sort_pairs(k0, v0, k1, v1, nq, 0, ((h->grid_bits + 7) / 8) * 8, counts, counts_cap, s));
    }
    // (2) queries in the reordered structure-of-arrays layout
    GJ_TRY(dev_alloc(&qs->XQ, (size_t)d * qs->qnpad * sizeof(double), s));
    GJ_TRY(dev_alloc(&qs->qorig, maxn * sizeof(uint32_t), s));
    GJ_TRY(cudaMemsetAsync(qs->XQ, 0, (size_t)d * qs->qnpad * sizeof(double), s));
    if (nq > 0) {
        note_launch();
        k_gather_soa<<<(int)grid_blocks(nq, 32), 256, 0, s>>>(Q, nq, d, qs->qnpad, v0, h->perm_dev, qs->XQ,
                                                             qs->qorig);
        GJ_TRY(cudaGetLastError());
        // (3) query cells
        note_launch();
        k_heads<<<(int)grid_blocks(nq, 256), 256, 0, s>>>(k0, nq, flagbuf);
        int64_t last_flag = 0, last_pre = 0;
        GJ_TRY(cudaMemcpyAsync(&last_flag, flagbuf + nq - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        GJ_TRY(exclusive_scan_i64(flagbuf, nq, tmp, tmp_cap, s));
        GJ_TRY(cudaMemcpyAsync(&last_pre, flagbuf + nq - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        GJ_TRY(cudaStreamSynchronize(s));
        Gq = last_pre + last_flag;
    }
    qs->Gq = Gq;
    GJ_TRY(dev_alloc(&qs->qcell_start, (Gq + 1) * sizeof(int64_t), s));
    GJ_TRY(dev_alloc(&qs->qcell_id, std::max<int64_t>(Gq, 1) * sizeof(int64_t), s));
    GJ_TRY(dev_alloc(&qs->adj_start, (Gq + 1) * sizeof(int64_t), s));
    GJ_TRY(dev_alloc(&cnt, std::max<int64_t>(Gq, 1) * sizeof(int64_t), s));
    GJ_TRY(dev_alloc(&nbsum, std::max<int64_t>(Gq, 1) * sizeof(int64_t), s));
    note_launch();
    k_set_i64<<<1, 1, 0, s>>>(qs->qcell_start + Gq, nq);
    if (Gq > 0) {
        note_launch();
        k_cells<<<(int)grid_blocks(nq, 256), 256, 0, s>>>(k0, nq, flagbuf, qs->qcell_start, qs->qcell_id);
        // (4) entry cells adjacent to each query cell
        const int64_t thr = Gq * 32;
        note_launch();
        k_adjacent_qe<<<(int)grid_blocks(thr, 256), 256, 0, s>>>(qs->qcell_id, Gq, h->cell_id, h->cell_start, h->G,
                                                                 ap, 0, cnt, nbsum, nullptr, nullptr);
        GJ_TRY(cudaGetLastError());
        GJ_TRY(cudaMemcpyAsync(qs->adj_start, cnt, Gq * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
        int64_t last_cnt = 0, last_pre = 0;
        GJ_TRY(cudaMemcpyAsync(&last_cnt, cnt + Gq - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        GJ_TRY(exclusive_scan_i64(qs->adj_start, Gq, tmp, tmp_cap, s));
        GJ_TRY(cudaMemcpyAsync(&last_pre, qs->adj_start + Gq - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        GJ_TRY(cudaStreamSynchronize(s));
        nadj = last_pre + last_cnt;
        note_launch();
        k_set_i64<<<1, 1, 0, s>>>(qs->adj_start + Gq, nadj);
        GJ_TRY(dev_alloc(&qs->adj, std::max<int64_t>(nadj, 1) * sizeof(uint32_t), s));
        if (nadj > 0) {
            note_launch();
            k_adjacent_qe<<<(int)grid_blocks(thr, 256), 256, 0, s>>>(qs->qcell_id, Gq, h->cell_id, h->cell_start,
                                                                     h->G, ap, 1, nullptr, nullptr, qs->adj_start,
                                                                     qs->adj);
            GJ_TRY(cudaGetLastError());
        }
        // (5) work items by descending load
        note_launch();
        k_item_counts<<<(int)grid_blocks(Gq, 256), 256, 0, s>>>(qs->qcell_start, Gq, qb, 0, cnt);
        GJ_TRY(cudaMemcpyAsync(&last_cnt, cnt + Gq - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        GJ_TRY(exclusive_scan_i64(cnt, Gq, tmp, tmp_cap, s));
        GJ_TRY(cudaMemcpyAsync(&last_pre, cnt + Gq - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        GJ_TRY(cudaStreamSynchronize(s));
        nitems = last_pre + last_cnt;
    } else {
        GJ_TRY(dev_alloc(&qs->adj, sizeof(uint32_t), s));
        note_launch();
        k_set_i64<<<1, 1, 0, s>>>(qs->adj_start, 0);
    }
    qs->nitems = nitems;
    GJ_TRY(dev_alloc(&qs->items, std::max<int64_t>(nitems, 1) * sizeof(Item), s));
    GJ_TRY(dev_alloc(&qs->order, std::max<int64_t>(nitems, 1) * sizeof(uint32_t), s));
    if (nitems > 0) {
        note_launch();
        k_qe_items<<<(int)grid_blocks(Gq, 256), 256, 0, s>>>(qs->qcell_start, Gq, qb, cnt, nbsum, qs->items,
                                                             k0, v0, cand_dev);
        GJ_TRY(cudaGetLastError());
        GJ_TRY(radix_sort_pairs(k0, v0, k1, v1, nitems, 0, 32, counts, counts_cap, s));
        GJ_TRY(cudaMemcpyAsync(qs->order, v0, nitems * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
    GJ_TRY(cudaMemcpyAsync(&qs->candidates, cand_dev, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    GJ_TRY(cudaStreamSynchronize(s));
done:
    dev_free(k0, s);
    dev_free(k1, s);
    dev_free(v0, s);
    dev_free(v1, s);
    dev_free(counts, s);
    dev_free(flagbuf, s);
    dev_free(tmp, s);
    dev_free(cnt, s);
    dev_free(nbsum, s);
    dev_free(cand_dev, s);
    if (st != GJ_OK)
        free_query_side(qs, s);
    return st;
}

}  // namespace gj
