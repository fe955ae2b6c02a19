// gj_qjoin.cu -- the similarity join Q join_eps E of Sec. 3.1.
//
// The paper states the self-join as the case Q = E of the similarity join
// that finds, for every query point of Q, the entry points of E within eps.
// Here E is an index built by gj_index_build* (REORDER, grid, cells); the
// queries of a call are keyed into E's grid (build_query_side: same REORDER
// permutation, cell widths and origin, sorted by cell and by the SORTIDU
// dimension, gathered into the structure-of-arrays layout), every query cell
// gets the list of all adjacent non-empty entry cells (no symmetry to exploit),
// and a join kernel runs in its asymmetric mode: queries from the query array,
// candidates from the entries, one orientation (q, e) per pair.  The kernel is
// the index's own form: the plain FP64 SHORTC kernel, or for an index built
// with GJ_TC_FILTER the tensor-core filter with its FP64 recheck (query A rows
// and entry B rows packed under one centre and one scale that covers both
// sets, so the filter's margin holds for every query-entry pair).  One launch
// writes the pairs straight into the caller's device buffer, or into a device
// buffer of cap pairs that is then copied to the host, with warp-aggregated
// atomics, and counts every pair, so a result larger than cap is reported with
// its size.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "gj_internal.cuh"

namespace gj {
namespace {

__global__ void k_qe_queue(const uint32_t *__restrict__ order, int64_t n, uint32_t *__restrict__ queue)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n)
        queue[i] = order[i];
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

extern "C" int gj_join_qe(gj_index *h, const double *queries, int64_t nq, gj_pair *pairs_out, uint64_t cap,
                          uint64_t *count)
{
    if (!h || !count || nq < 0 || (nq > 0 && !queries) || (!pairs_out && cap > 0))
        return GJ_ERR_INVALID_ARG;
    if (nq >= ((int64_t)1 << 32))
        return GJ_ERR_TOO_LARGE;
    *count = 0;
    if (cudaSetDevice(h->device) != cudaSuccess)
        return GJ_ERR_CUDA;
    if (pairs_out && foreign_device(pairs_out, h->device))
        return GJ_ERR_INVALID_ARG;   // another device's memory
    cudaStream_t s = h->stream;
    const int d = h->info.d;
    const bool tc = h->tc_ready;
    // query blocks small enough that every CTA of the persistent grid gets
    // about eight (few queries against many entries would otherwise leave
    // most of the grid idle behind a few long blocks); blocks of at most 64
    // also shrink the plain kernel's query tile, which may fit more CTAs per
    // SM.  Tensor-core blocks hold at most 120 queries, so the 128-row A tile
    // from the block's first row rounded down to 8 covers the block.
    int qb = 0, grid = 0;
    if (tc) {
        qb = (int)std::max<int64_t>(32, std::min<int64_t>(120, (nq / (8 * (int64_t)h->sms)) & ~7));
        grid = h->sms;
    } else {
        int per_sm = plain_ctas_per_sm(d, h->plain_ct, QB);
        if (per_sm < 1)
            return GJ_ERR_UNSUPPORTED;
        qb = (int)std::max<int64_t>(32, std::min<int64_t>(QB_PLAIN, (nq / (8 * (int64_t)h->sms * per_sm)) & ~7));
        per_sm = plain_ctas_per_sm(d, h->plain_ct, qb);
        grid = h->sms * per_sm;
    }

    // queries on the device, finite
    double *Qd = nullptr;
    unsigned int *flag = nullptr;
    unsigned int hflag = 0;
    // host memory or another device's memory is copied to this device first
    const bool q_on_dev = device_memory_of(queries, h->device);
    cudaError_t e = cudaSuccess;
    if (nq > 0 && !q_on_dev) {
        e = cudaMalloc(&Qd, (size_t)nq * d * sizeof(double));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(Qd, queries, (size_t)nq * d * sizeof(double), cudaMemcpyDefault, s);
    }
    const double *Q = (nq > 0 && !q_on_dev) ? Qd : queries;
    if (e == cudaSuccess) e = cudaMalloc(&flag, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess && nq > 0) e = launch_check_finite(Q, nq * (int64_t)d, flag, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(flag);
    if (e != cudaSuccess) {
        cudaFree(Qd);
        return status_of(e);
    }
    if (hflag) {
        cudaFree(Qd);
        return GJ_ERR_NONFINITE;
    }

    // the query side
    QuerySide qs;
    int st = build_query_side(h, Q, nq, qb, &qs, s);
    cudaFree(Qd);
    if (st != GJ_OK)
        return st;
    if (qs.nitems == 0 || h->info.n == 0) {
        free_query_side(&qs, s);
        return GJ_OK;
    }

    // tensor-core operands: the scale must keep every |h| of both sets at
    // most 250, so it comes from the larger radius about the entries' centre;
    // the entries' B rows are reused when that scale is theirs
    void *XAq = nullptr, *XBt = nullptr;
    const void *XBop = nullptr;
    int Tbits = 0;
    if (tc) {
        double R0q = 0.0;
        const int Kp = h->tc_Kp;
        e = tc_radius(qs.XQ, nq, qs.qnpad, d, h->tc_centre, &R0q, s);
        const double R0 = std::max(h->tc_R0, R0q);
        const double sigma = tc_sigma_for(R0);
        const size_t abytes = (size_t)(qs.qnpad + 512) * Kp * 2;
        if (e == cudaSuccess) e = dev_alloc(&XAq, abytes, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(XAq, 0, abytes, s);
        if (e == cudaSuccess) e = tc_pack_into(qs.XQ, nq, qs.qnpad, d, Kp, sigma, h->tc_centre, 0, XAq, nullptr, s);
        XBop = h->XB;
        if (e == cudaSuccess && sigma != h->tc_sigma) {
            const size_t bbytes = (size_t)(h->npad + 512) * Kp * 2;
            e = dev_alloc(&XBt, bbytes, s);
            if (e == cudaSuccess) e = cudaMemsetAsync(XBt, 0, bbytes, s);
            if (e == cudaSuccess)
                e = tc_pack_into(h->X, h->info.n, h->npad, d, Kp, sigma, h->tc_centre, 0, nullptr, XBt, s);
            XBop = XBt;
        }
        Tbits = tc_threshold_bits(h->info.eps, sigma, R0, d, Kp);
        if (e != cudaSuccess) {
            dev_free(XAq, s);
            dev_free(XBt, s);
            free_query_side(&qs, s);
            return status_of(e);
        }
    }

    // the asymmetric join kernel
    JoinCtl *ctl = nullptr;
    uint32_t *queue = nullptr;
    gj_pair *dbuf = nullptr;
    JoinCtl hctl{};
    gj_pair *const direct = device_view(pairs_out);   // host output: a device buffer, then a copy
    const bool dev_out = direct != nullptr;
    uint64_t total = 0;
    e = cudaMalloc(&ctl, sizeof(JoinCtl));
    if (e == cudaSuccess) e = cudaMalloc(&queue, qs.nitems * sizeof(uint32_t));
    if (e == cudaSuccess) {
        note_launch();
        k_qe_queue<<<(int)((qs.nitems + 255) / 256), 256, 0, s>>>(qs.order, qs.nitems, queue);
        e = cudaGetLastError();
    }
    JoinLaunch L{};
    L.ix.X = h->X;
    L.ix.orig = h->orig;
    L.ix.cell_start = h->cell_start;
    L.ix.adj_start = qs.adj_start;
    L.ix.adj = qs.adj;
    L.ix.items = qs.items;
    L.ix.n = h->info.n;
    L.ix.npad = h->npad;
    L.ix.d = d;
    L.ix.u = h->u;
    L.ix.e2 = h->e2;
    L.ix.ew = h->ew;
    L.ix.ct = h->plain_ct;
    L.ix.qb = qb;
    L.ix.asym = 1;
    L.ix.XQ = qs.XQ;
    L.ix.qorig = qs.qorig;
    L.ix.qnpad = qs.qnpad;
    L.queue = queue;
    L.qlimit = (uint32_t)qs.nitems;
    L.ctl = ctl;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double kms = 0.0;
    if (e == cudaSuccess) e = cudaEventCreate(&ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ev1);
    // one launch: pairs go straight to the output (device memory, or a device
    // buffer of cap pairs for host output) while every pair is counted, so a
    // result larger than cap is reported with its size
    gj_pair *out = nullptr;
    if (e == cudaSuccess && cap > 0) {
        if (dev_out) {
            out = direct;
        } else {
            e = cudaMalloc(&dbuf, cap * sizeof(gj_pair));
            out = dbuf;
        }
    }
    L.out = out;
    L.cap = out ? cap : 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, sizeof(JoinCtl), s);
    if (e == cudaSuccess) e = cudaEventRecord(ev0, s);
    if (e == cudaSuccess)
        e = tc ? launch_join_tc_ops(L, XAq, XBop, h->XR, h->XR_dr, h->tc_Kp, Tbits, grid, s)
               : launch_join_plain_direct(L, grid, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev1, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hctl, ctl, sizeof(JoinCtl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        kms = ms;
        if (hctl.err & kErrTimeout)
            st = GJ_ERR_TIMEOUT;
        else if (hctl.err)
            st = GJ_ERR_CUDA;
        total = out ? hctl.pos : hctl.counted;
        h->last = gj_join_stats{};
        h->last.pairs = total;
        h->last.evaluated = hctl.evaluated;
        h->last.dims = hctl.dims;
        h->last.tc_survivors = hctl.survivors;
        h->last.candidates = qs.candidates;
    }
    h->last.join_ms = kms;
    h->last.launches = 1;
    if (e == cudaSuccess && st == GJ_OK && dbuf && total <= cap && total > 0)
        e = cudaMemcpy(pairs_out, dbuf, total * sizeof(gj_pair), cudaMemcpyDeviceToHost);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    cudaFree(ctl);
    cudaFree(queue);
    cudaFree(dbuf);
    dev_free(XAq, s);
    dev_free(XBt, s);
    free_query_side(&qs, s);
    if (e != cudaSuccess)
        return status_of(e);
    *count = total;
    if (st != GJ_OK)
        return st;
    return (pairs_out && total > cap) ? GJ_ERR_CAPACITY : GJ_OK;
}
