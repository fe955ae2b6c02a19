// gj_table.cu -- the neighbour table of a self-join result.
//
// Alg. 1 keeps a batch's key/value result pairs (key = query point, value = a
// point within eps) and folds them into the result with constructNeighborTable,
// which stores each key once (Sec. 3.2.2).  Here the table is built on the
// device in compressed sparse row form, rows in original point order and each
// row's neighbours ascending, so the table is a deterministic function of R:
//   1. the join writes R into a device buffer;
//   2. every pair (a, b) becomes the 64-bit key (a << B) | b, B = bits of n - 1,
//      with value b, and a stable LSD radix sort orders the keys -- rows by a,
//      neighbours by b;
//   3. per-row counts (one atomic per pair) and their exclusive scan give the
//      row starts; the sorted values are the neighbour lists.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "gj_internal.cuh"

namespace gj {
namespace {

__global__ void k_table_keys(const gj_pair *__restrict__ pairs, int64_t m, int bb, uint64_t *__restrict__ key,
                             uint32_t *__restrict__ val)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m) {
        const gj_pair p = pairs[i];
        key[i] = ((uint64_t)p.a << bb) | (uint64_t)p.b;
        val[i] = p.b;
    }
}

__global__ void k_row_counts(const uint64_t *__restrict__ key, int64_t m, int bb, int64_t n,
                             unsigned long long *__restrict__ cnt)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m) {
        const uint64_t a = key[i] >> bb;
        if (a < (uint64_t)n)
            atomicAdd(&cnt[a], 1ull);
    }
}

int status_of(cudaError_t e)
{
    if (e == cudaSuccess)
        return GJ_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GJ_ERR_OOM : GJ_ERR_CUDA;
}

}  // namespace
}  // namespace gj

using namespace gj;

extern "C" int gj_neighbor_table(gj_index *h, int64_t *row_start, uint32_t *nbr, uint64_t cap, uint64_t *count)
{
    if (!h || !count || !row_start || (cap > 0 && !nbr))
        return GJ_ERR_INVALID_ARG;
    *count = 0;
    if (cudaSetDevice(h->device) != cudaSuccess)
        return GJ_ERR_CUDA;
    if (!device_memory_of(row_start, h->device) || (cap > 0 && !device_memory_of(nbr, h->device)))
        return GJ_ERR_INVALID_ARG;
    const int64_t n = h->info.n;
    cudaStream_t s = h->stream;

    // 1. |R|, then R itself into a device buffer
    uint64_t total = 0;
    int st = gj_self_join(h, nullptr, 0, &total);
    if (st != GJ_OK)
        return st;
    *count = total;
    if (total > cap)
        return GJ_ERR_CAPACITY;
    gj_pair *pairs = nullptr;
    uint64_t *k0 = nullptr, *k1 = nullptr;
    uint32_t *v1 = nullptr, *counts = nullptr;
    int64_t *tmp = nullptr;
    cudaError_t e = cudaSuccess;
    int bb = 1;
    while (bb < 32 && ((int64_t)1 << bb) < n)
        ++bb;
    const int64_t m = (int64_t)total;
    const int64_t counts_cap = radix_counts_needed(std::max<int64_t>(m, 1));
    const int64_t tmp_cap = scan_tmp_needed(n + 1) + 64;
    if (m > 0) {
        e = cudaMalloc(&pairs, (size_t)m * sizeof(gj_pair));
        if (e != cudaSuccess)
            return status_of(e);
        uint64_t c2 = 0;
        st = gj_self_join(h, pairs, total, &c2);
        if (st == GJ_OK && c2 != total)
            st = GJ_ERR_CUDA;
        if (st != GJ_OK) {
            cudaFree(pairs);
            return st;
        }
    }
    // 2. keys and the radix sort (the sorted values land in nbr)
    if (e == cudaSuccess && m > 0) e = cudaMalloc(&k0, (size_t)m * sizeof(uint64_t));
    if (e == cudaSuccess && m > 0) e = cudaMalloc(&k1, (size_t)m * sizeof(uint64_t));
    if (e == cudaSuccess && m > 0) e = cudaMalloc(&v1, (size_t)m * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&counts, (size_t)counts_cap * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&tmp, (size_t)tmp_cap * sizeof(int64_t));
    if (e == cudaSuccess && m > 0) {
        note_launch();
        k_table_keys<<<(int)((m + 255) / 256), 256, 0, s>>>(pairs, m, bb, k0, nbr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && m > 1)
        e = radix_sort_pairs(k0, nbr, k1, v1, m, 0, ((2 * bb + 7) / 8) * 8, counts, counts_cap, s);
    // 3. row counts -> row starts
    if (e == cudaSuccess) e = cudaMemsetAsync(row_start, 0, (size_t)(n + 1) * sizeof(int64_t), s);
    if (e == cudaSuccess && m > 0) {
        note_launch();
        k_row_counts<<<(int)((m + 255) / 256), 256, 0, s>>>(k0, m, bb, n, (unsigned long long *)row_start);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = exclusive_scan_i64(row_start, n + 1, tmp, tmp_cap, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(pairs);
    cudaFree(k0);
    cudaFree(k1);
    cudaFree(v1);
    cudaFree(counts);
    cudaFree(tmp);
    return status_of(e);
}
