// gj_batch.cu -- many independent self-joins in one persistent launch.
//
// No paper counterpart (the paper runs one self-join at a time).  Each job's
// index is built with the single-job builder (REORDER, grid, adjacency, work
// items, fp16 filter operands), then the jobs are concatenated into one
// combined index:
//   * points back to back in one FP64 structure-of-arrays, zero-padded to the
//     largest d (a zero dimension adds exactly 0 to an FP64 running sum, so no
//     distance decision changes);
//   * cells, adjacency lists and work items shifted by each job's offsets,
//     every work item tagged with its job;
//   * the filter operands re-packed with one common K (each job keeps its own
//     centre, scale and survivor threshold);
//   * one queue of all work items in descending estimated load.
// A join is then one launch of the tensor-core kernel in which every job
// writes its pairs straight into its own device buffer through its own
// counter.  The launch has no host decisions in it, so it is captured once in
// a CUDA graph (parameter upload, counter reset, kernel, counter download) and
// replayed on every later call.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "gj_internal.cuh"

using namespace gj;

struct gj_batch {
    int device;
    cudaStream_t stream;
    bool own_stream;
    int sms;
    int32_t njobs;
    int d_max, Kp;
    int64_t n_total, npad, G_total, nitems;
    double *X;
    uint32_t *orig;
    int64_t *cell_start, *adj_start;
    uint32_t *adj;
    Item *items;
    uint32_t *order;
    void *XA, *XB;
    TcJob *jobs_dev;
    TcJob *jobs_host;           // pinned: the launch parameters uploaded by the graph
    unsigned long long *jpos;   // device counters
    unsigned long long *jpos_host;   // pinned
    JoinCtl *ctl;
    cudaGraphExec_t graph;
    bool graph_ready;
    std::vector<uint64_t> n_job;
    std::vector<int32_t> k_job;   // k of each job's grid
    uint64_t candidates;        // sum over jobs of the unordered candidate pairs of the grid
    JoinCtl *ctl_host;          // pinned: the control block read back by the graph
};

namespace {

__global__ void k_shift_i64(const int64_t *__restrict__ src, int64_t count, int64_t add, int64_t *__restrict__ dst)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count)
        dst[i] = src[i] + add;
}

__global__ void k_shift_u32(const uint32_t *__restrict__ src, int64_t count, uint32_t add, uint32_t *__restrict__ dst)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count)
        dst[i] = src[i] + add;
}

__global__ void k_shift_items(const Item *__restrict__ src, int64_t count, uint32_t cell_add, uint32_t pos_add,
                              uint32_t job, Item *__restrict__ dst)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count) {
        Item it = src[i];
        dst[i] = Item{it.cell + cell_add, it.qbeg + pos_add, it.qlen, job};
    }
}

__global__ void k_set_one_i64(int64_t *p, int64_t v) { *p = v; }

// key = ~float bits of the estimated load qlen * (points in the searched cells)
__global__ void k_item_loads(const Item *__restrict__ items, int64_t nitems, const int64_t *__restrict__ cell_start,
                             const int64_t *__restrict__ adj_start, const uint32_t *__restrict__ adj,
                             uint64_t *__restrict__ key, uint32_t *__restrict__ val)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nitems)
        return;
    const Item it = items[i];
    int64_t pts = cell_start[it.cell + 1] - it.qbeg;
    for (int64_t a = adj_start[it.cell]; a < adj_start[it.cell + 1]; ++a) {
        const uint32_t b = adj[a];
        if (b != it.cell)
            pts += cell_start[b + 1] - cell_start[b];
    }
    const float load = (float)it.qlen * (float)pts;
    key[i] = (uint64_t)(~__float_as_uint(load));
    val[i] = (uint32_t)i;
}

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess)
        return GJ_OK;
    return e == cudaErrorMemoryAllocation ? GJ_ERR_OOM : GJ_ERR_CUDA;
}

int64_t blocks(int64_t n, int t) { return (n + t - 1) / t; }

}  // namespace

extern "C" {

void gj_batch_free(gj_batch *b)
{
    if (!b)
        return;
    cudaSetDevice(b->device);
    if (b->stream)
        cudaStreamSynchronize(b->stream);
    if (b->graph_ready)
        cudaGraphExecDestroy(b->graph);
    cudaFree(b->X);
    cudaFree(b->orig);
    cudaFree(b->cell_start);
    cudaFree(b->adj_start);
    cudaFree(b->adj);
    cudaFree(b->items);
    cudaFree(b->order);
    cudaFree(b->XA);
    cudaFree(b->XB);
    cudaFree(b->jobs_dev);
    cudaFreeHost(b->jobs_host);
    cudaFree(b->jpos);
    cudaFreeHost(b->jpos_host);
    cudaFree(b->ctl);
    cudaFreeHost(b->ctl_host);
    if (b->own_stream && b->stream)
        cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"

namespace {

// The combined structure of the jobs, job j's grid on ks[j] dimensions
// (0 = the builder's own choice).
gj_batch *build_batch(const gj_job *jobs, int32_t njobs, const gj_config &cfg, const int32_t *ks)
{
    int d_max = 1;
    int64_t n_total = 0;
    for (int32_t j = 0; j < njobs; ++j) {
        if (jobs[j].d < 1 || jobs[j].n < 0 || !(jobs[j].eps > 0.0)) {
            gj::set_last_status(GJ_ERR_INVALID_ARG);
            return nullptr;
        }
        d_max = std::max(d_max, (int)jobs[j].d);
        n_total += jobs[j].n;
    }
    const int Kp = ((d_max + 4 + 15) / 16) * 16;
    if (Kp > 128 || n_total >= ((int64_t)1 << 31)) {
        gj::set_last_status(GJ_ERR_TOO_LARGE);
        return nullptr;
    }
    gj_batch *b = new (std::nothrow) gj_batch();
    if (!b) {
        gj::set_last_status(GJ_ERR_OOM);
        return nullptr;
    }
    int st = GJ_OK;
    cudaError_t e = cudaSuccess;
    int dev = cfg.device;
    if (dev < 0)
        cudaGetDevice(&dev);
    else
        cudaSetDevice(dev);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess || prop.major != 10 || prop.minor != 3) {
        delete b;
        gj::set_last_status(GJ_ERR_UNSUPPORTED);
        return nullptr;
    }
    b->device = dev;
    b->sms = prop.multiProcessorCount;
    b->njobs = njobs;
    b->d_max = d_max;
    b->Kp = Kp;
    b->n_total = n_total;
    b->npad = ((n_total + 31) / 32) * 32 + 32;
    if (cfg.stream) {
        b->stream = (cudaStream_t)cfg.stream;
    } else {
        cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        b->own_stream = true;
    }
    cudaStream_t s = b->stream;

    // 1. per-job indices
    std::vector<gj_index *> hs(njobs, nullptr);
    gj_config jc = cfg;
    jc.flags = cfg.flags | GJ_TC_FILTER;
    jc.stream = (void *)s;
    jc.device = dev;
    int64_t G_total = 0, A_total = 0, I_total = 0;
    jc.flags &= ~(GJ_AUTOTUNE | GJ_TUNE_FORM);
    // fixed 120-point blocks: a job's positions are shifted in the combined
    // layout, so blocks aligned within the job would not stay aligned
    jc.query_block = QB_TC;
    jc.tile = 0;
    // The jobs' indices are built by a few host threads, each on its own
    // stream, largest jobs first: a build is a chain of short kernels and
    // host round trips, so several chains overlap on the device.
    {
        std::vector<int32_t> by_size((size_t)njobs);
        for (int32_t j = 0; j < njobs; ++j)
            by_size[j] = j;
        std::stable_sort(by_size.begin(), by_size.end(),
                         [&](int32_t a, int32_t c) { return jobs[a].n > jobs[c].n; });
        const int nthreads = (int)std::min<int32_t>(8, njobs);
        std::vector<cudaStream_t> streams((size_t)nthreads, nullptr);
        std::vector<int> tst((size_t)nthreads, GJ_OK);
        std::atomic<int32_t> next{0};
        for (int t = 0; t < nthreads && e == cudaSuccess; ++t)
            e = cudaStreamCreateWithFlags(&streams[t], cudaStreamNonBlocking);
        // the inputs may still be in flight on the caller's stream
        cudaEvent_t ready = nullptr;
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ready, s);
        for (int t = 0; t < nthreads && e == cudaSuccess; ++t)
            e = cudaStreamWaitEvent(streams[t], ready, 0);
        st = cuda_status(e);
        if (st == GJ_OK) {
            std::vector<std::thread> pool;
            for (int t = 0; t < nthreads; ++t) {
                pool.emplace_back([&, t]() {
                    cudaSetDevice(dev);
                    gj_config tc = jc;
                    tc.stream = (void *)streams[t];
                    for (;;) {
                        const int32_t i = next.fetch_add(1);
                        if (i >= njobs || tst[t] != GJ_OK)
                            break;
                        const int32_t j = by_size[i];
                        tc.k = ks[j];
                        hs[j] = gj_index_build_ex(jobs[j].points, jobs[j].n, jobs[j].d, jobs[j].eps, &tc);
                        if (!hs[j])
                            tst[t] = gj_last_status();
                    }
                    if (cudaStreamSynchronize(streams[t]) != cudaSuccess && tst[t] == GJ_OK)
                        tst[t] = GJ_ERR_CUDA;
                });
            }
            for (auto &th : pool)
                th.join();
            for (int t = 0; t < nthreads; ++t)
                if (tst[t] != GJ_OK)
                    st = tst[t];
        }
        // from here on every job's memory is used and released in the order of
        // the batch's stream
        for (int32_t j = 0; j < njobs; ++j)
            if (hs[j])
                hs[j]->stream = s;
        if (ready)
            cudaEventDestroy(ready);
        for (auto sm : streams)
            if (sm)
                cudaStreamDestroy(sm);
    }
    for (int32_t j = 0; j < njobs && st == GJ_OK; ++j) {
        b->k_job.push_back(hs[j]->info.k);
        G_total += hs[j]->G;
        I_total += hs[j]->nitems;
        b->candidates += hs[j]->info.candidate_pairs;
    }
    std::vector<int64_t> A_j(njobs, 0);
    if (st == GJ_OK) {
        for (int32_t j = 0; j < njobs; ++j) {
            A_j[j] = hs[j]->G > 0 ? hs[j]->nadj : 0;
            A_total += A_j[j];
        }
        st = cuda_status(e);
    }
    b->G_total = G_total;
    b->nitems = I_total;
    const size_t rows = (size_t)b->npad + 512;

    // 2. combined arrays
    uint64_t *k0 = nullptr, *k1 = nullptr;
    uint32_t *v0 = nullptr, *v1 = nullptr, *counts = nullptr;
    if (st == GJ_OK) {
        e = cudaMalloc(&b->X, (size_t)d_max * b->npad * sizeof(double));
        if (e == cudaSuccess) e = cudaMemsetAsync(b->X, 0, (size_t)d_max * b->npad * sizeof(double), s);
        if (e == cudaSuccess) e = cudaMalloc(&b->orig, (size_t)b->npad * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMalloc(&b->cell_start, (size_t)(G_total + 1) * sizeof(int64_t));
        if (e == cudaSuccess) e = cudaMalloc(&b->adj_start, (size_t)(G_total + 1) * sizeof(int64_t));
        if (e == cudaSuccess) e = cudaMalloc(&b->adj, (size_t)std::max<int64_t>(A_total, 1) * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMalloc(&b->items, (size_t)std::max<int64_t>(I_total, 1) * sizeof(Item));
        if (e == cudaSuccess) e = cudaMalloc(&b->order, (size_t)std::max<int64_t>(I_total, 1) * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMalloc(&b->XA, rows * Kp * 2);
        if (e == cudaSuccess) e = cudaMalloc(&b->XB, rows * Kp * 2);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->XA, 0, rows * Kp * 2, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->XB, 0, rows * Kp * 2, s);
        if (e == cudaSuccess) e = cudaMallocHost(&b->jobs_host, (size_t)njobs * sizeof(TcJob));
        if (e == cudaSuccess) e = cudaMalloc(&b->jobs_dev, (size_t)njobs * sizeof(TcJob));
        if (e == cudaSuccess) e = cudaMalloc(&b->jpos, (size_t)njobs * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMallocHost(&b->jpos_host, (size_t)njobs * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMalloc(&b->ctl, sizeof(JoinCtl));
        if (e == cudaSuccess) e = cudaMallocHost(&b->ctl_host, sizeof(JoinCtl));
        st = cuda_status(e);
    }
    int64_t P = 0, C = 0, A = 0, I = 0;
    for (int32_t j = 0; j < njobs && st == GJ_OK; ++j) {
        gj_index *h = hs[j];
        const int64_t n = h->info.n;
        b->n_job.push_back((uint64_t)n);
        if (n > 0) {
            e = cudaMemcpy2DAsync(b->X + P, (size_t)b->npad * sizeof(double), h->X, (size_t)h->npad * sizeof(double),
                                  (size_t)n * sizeof(double), (size_t)h->info.d, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(b->orig + P, h->orig, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        }
        if (e == cudaSuccess && h->G > 0) {
            note_launch();
            k_shift_i64<<<(int)blocks(h->G, 256), 256, 0, s>>>(h->cell_start, h->G, P, b->cell_start + C);
            note_launch();
            k_shift_i64<<<(int)blocks(h->G, 256), 256, 0, s>>>(h->adj_start, h->G, A, b->adj_start + C);
            if (A_j[j] > 0) {
                note_launch();
                k_shift_u32<<<(int)blocks(A_j[j], 256), 256, 0, s>>>(h->adj, A_j[j], (uint32_t)C, b->adj + A);
            }
            if (h->nitems > 0) {
                note_launch();
                k_shift_items<<<(int)blocks(h->nitems, 256), 256, 0, s>>>(h->items, h->nitems, (uint32_t)C,
                                                                          (uint32_t)P, (uint32_t)j, b->items + I);
            }
            e = cudaGetLastError();
        }
        // filter operands with the common K, this job's centre and scale
        TcJob &J = b->jobs_host[j];
        J.e2 = h->e2;
        J.ew = h->ew;
        J.u = h->u;
        J.d = h->info.d;
        J.pad = 0;
        J.out = nullptr;
        J.cap = 0;
        if (e == cudaSuccess && h->tc_ready) {
            e = tc_pack_into(h->X, n, h->npad, h->info.d, Kp, h->tc_sigma, h->tc_centre, P, b->XA, b->XB, s);
            J.Tbits = tc_threshold_bits(h->info.eps, h->tc_sigma, h->tc_R0, h->info.d, Kp);
        } else {
            J.Tbits = 0;   // an empty job: nothing survives
        }
        st = cuda_status(e);
        P += n;
        C += h->G;
        A += A_j[j];
        I += h->nitems;
    }
    if (st == GJ_OK) {
        note_launch();
        k_set_one_i64<<<1, 1, 0, s>>>(b->cell_start + G_total, n_total);
        note_launch();
        k_set_one_i64<<<1, 1, 0, s>>>(b->adj_start + G_total, A_total);
        e = cudaGetLastError();
        st = cuda_status(e);
    }
    for (auto h : hs)
        gj_free(h);

    // 3. one queue of all work items by descending load
    if (st == GJ_OK && I_total > 0) {
        const int64_t ccap = radix_counts_needed(I_total);
        e = cudaMalloc(&k0, I_total * sizeof(uint64_t));
        if (e == cudaSuccess) e = cudaMalloc(&k1, I_total * sizeof(uint64_t));
        if (e == cudaSuccess) e = cudaMalloc(&v0, I_total * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMalloc(&v1, I_total * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMalloc(&counts, ccap * sizeof(uint32_t));
        if (e == cudaSuccess) {
            note_launch();
            k_item_loads<<<(int)blocks(I_total, 256), 256, 0, s>>>(b->items, I_total, b->cell_start, b->adj_start,
                                                                   b->adj, k0, v0);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = radix_sort_pairs(k0, v0, k1, v1, I_total, 0, 32, counts, ccap, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->order, v0, I_total * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        st = cuda_status(e);
    }
    cudaFree(k0);
    cudaFree(k1);
    cudaFree(v0);
    cudaFree(v1);
    cudaFree(counts);
    if (st != GJ_OK) {
        gj_batch_free(b);
        gj::set_last_status(st);
        return nullptr;
    }
    gj::set_last_status(GJ_OK);
    return b;
}

JoinLaunch batch_launch(const gj_batch *b)
{
    JoinLaunch L{};
    L.ix.X = b->X;
    L.ix.orig = b->orig;
    L.ix.cell_start = b->cell_start;
    L.ix.adj_start = b->adj_start;
    L.ix.adj = b->adj;
    L.ix.items = b->items;
    L.ix.n = b->n_total;
    L.ix.npad = b->npad;
    L.ix.d = b->d_max;
    L.ix.u = -1;
    L.queue = b->order;
    L.qlimit = (uint32_t)b->nitems;
    L.ctl = b->ctl;
    L.out = nullptr;   // pairs go to the jobs' own buffers
    return L;
}

// One count-only launch of the whole batch that also sums, per job, the SM
// cycles its work items took (the autotuner's trial).
int timed_trial(gj_batch *b, std::vector<unsigned long long> &cyc)
{
    cyc.assign((size_t)b->njobs, 0ull);
    if (b->nitems == 0)
        return GJ_OK;
    cudaStream_t s = b->stream;
    unsigned long long *dc = nullptr;
    for (int32_t j = 0; j < b->njobs; ++j) {
        b->jobs_host[j].out = nullptr;
        b->jobs_host[j].cap = 0;
    }
    cudaError_t e = cudaMalloc(&dc, (size_t)b->njobs * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(dc, 0, (size_t)b->njobs * sizeof(unsigned long long), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->jobs_dev, b->jobs_host, (size_t)b->njobs * sizeof(TcJob), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->jpos, 0, (size_t)b->njobs * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ctl, 0, sizeof(JoinCtl), s);
    if (e == cudaSuccess) e = tc_jobs_launch_attr(b->Kp);
    if (e == cudaSuccess) {
        note_launch();
        e = launch_join_tc_jobs(batch_launch(b), b->XA, b->XB, b->Kp, b->jobs_dev, b->jpos, b->sms, s, dc);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cyc.data(), dc, (size_t)b->njobs * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->ctl_host, b->ctl, sizeof(JoinCtl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(dc);
    if (e != cudaSuccess)
        return cuda_status(e);
    if (b->ctl_host->err & kErrTimeout)
        return GJ_ERR_TIMEOUT;
    return b->ctl_host->err ? GJ_ERR_CUDA : GJ_OK;
}

// Picks of earlier tuned builds, per list of job shapes.
std::mutex g_tune_mu;
std::map<std::vector<uint64_t>, std::vector<int32_t>> g_tuned;

std::vector<uint64_t> shape_key(const gj_job *jobs, int32_t njobs, const gj_config &cfg, int device)
{
    std::vector<uint64_t> key;
    key.reserve((size_t)njobs * 3 + 2);
    key.push_back((uint64_t)device);
    key.push_back((uint64_t)(cfg.flags & (GJ_REORDER | GJ_SORTIDU | GJ_SHORTC)));
    for (int32_t j = 0; j < njobs; ++j) {
        uint64_t eb;
        memcpy(&eb, &jobs[j].eps, sizeof(eb));
        key.push_back((uint64_t)jobs[j].n);
        key.push_back(((uint64_t)(uint32_t)jobs[j].d << 32) | (uint32_t)jobs[j].k);
        key.push_back(eb);
    }
    return key;
}

}  // namespace

extern "C" {

gj_batch *gj_batch_build(const gj_job *jobs, int32_t njobs, const gj_config *cfg_in)
{
    gj_config cfg;
    if (cfg_in)
        cfg = *cfg_in;
    else
        gj_config_init(&cfg);
    if (!jobs || njobs < 1) {
        gj::set_last_status(GJ_ERR_INVALID_ARG);
        return nullptr;
    }
    std::vector<int32_t> ks((size_t)njobs);
    bool tune = false;
    for (int32_t j = 0; j < njobs; ++j) {
        ks[j] = jobs[j].k;
        tune = tune || ((cfg.flags & GJ_AUTOTUNE) && jobs[j].k == 0 && jobs[j].d >= 1);
    }
    if (!tune)
        return build_batch(jobs, njobs, cfg, ks.data());
    int dev = cfg.device;
    if (dev < 0)
        cudaGetDevice(&dev);
    const std::vector<uint64_t> key = shape_key(jobs, njobs, cfg, dev);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end())
            return build_batch(jobs, njobs, cfg, it->second.data());
    }
    // trials: every untuned job at k = 1, 2, 3 (capped at its d)
    std::vector<std::vector<unsigned long long>> cyc;
    std::vector<std::vector<int32_t>> used;
    gj_batch *last = nullptr;
    for (int kc = 1; kc <= 3; ++kc) {
        std::vector<int32_t> kt(ks);
        bool differs = kc == 1;
        for (int32_t j = 0; j < njobs; ++j)
            if (jobs[j].k == 0) {
                kt[j] = std::min<int32_t>(kc, jobs[j].d);
                differs = differs || kt[j] == kc;
            }
        if (!differs)
            break;
        gj_batch_free(last);
        last = build_batch(jobs, njobs, cfg, kt.data());
        if (!last)
            return nullptr;
        std::vector<unsigned long long> c;
        const int st = timed_trial(last, c);
        if (st != GJ_OK) {
            gj_batch_free(last);
            gj::set_last_status(st);
            return nullptr;
        }
        cyc.push_back(c);
        used.push_back(last->k_job);
    }
    std::vector<int32_t> pick(ks);
    for (int32_t j = 0; j < njobs; ++j) {
        if (jobs[j].k != 0)
            continue;
        size_t bt = 0;
        for (size_t t = 1; t < cyc.size(); ++t)
            if (cyc[t][j] < cyc[bt][j])
                bt = t;
        pick[j] = used[bt][j];
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = pick;
    }
    if (last && last->k_job == pick) {
        gj::set_last_status(GJ_OK);
        return last;
    }
    gj_batch_free(last);
    return build_batch(jobs, njobs, cfg, pick.data());
}

int gj_batch_get_k(const gj_batch *b, int32_t *k_per_job)
{
    if (!b || !k_per_job)
        return GJ_ERR_INVALID_ARG;
    for (int32_t j = 0; j < b->njobs; ++j)
        k_per_job[j] = b->k_job[(size_t)j];
    return GJ_OK;
}

int gj_batch_self_join(gj_batch *b, gj_pair *const *outs, const uint64_t *caps, uint64_t *counts)
{
    if (!b || !counts)
        return GJ_ERR_INVALID_ARG;
    if (cudaSetDevice(b->device) != cudaSuccess)
        return GJ_ERR_CUDA;
    for (int32_t j = 0; j < b->njobs; ++j) {
        gj_pair *o = outs ? outs[j] : nullptr;
        const uint64_t c = caps ? caps[j] : 0;
        if (!o && c > 0)
            return GJ_ERR_INVALID_ARG;
        if (o && !device_memory_of(o, b->device))
            return GJ_ERR_INVALID_ARG;   // not device memory of the batch's device
        b->jobs_host[j].out = c ? o : nullptr;
        b->jobs_host[j].cap = c;
    }
    cudaStream_t s = b->stream;
    cudaError_t e = cudaSuccess;
    if (!b->graph_ready) {
        const JoinLaunch L = batch_launch(b);
        cudaGraph_t g = nullptr;
        e = tc_jobs_launch_attr(b->Kp);
        if (e == cudaSuccess)
            e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaMemcpyAsync(b->jobs_dev, b->jobs_host, (size_t)b->njobs * sizeof(TcJob), cudaMemcpyHostToDevice, s);
            cudaMemsetAsync(b->jpos, 0, (size_t)b->njobs * sizeof(unsigned long long), s);
            cudaMemsetAsync(b->ctl, 0, sizeof(JoinCtl), s);
            if (b->nitems > 0)
                launch_join_tc_jobs(L, b->XA, b->XB, b->Kp, b->jobs_dev, b->jpos, b->sms, s);
            cudaMemcpyAsync(b->jpos_host, b->jpos, (size_t)b->njobs * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(b->ctl_host, b->ctl, sizeof(JoinCtl), cudaMemcpyDeviceToHost, s);
            e = cudaStreamEndCapture(s, &g);
        }
        if (e == cudaSuccess)
            e = cudaGraphInstantiate(&b->graph, g, 0);
        if (g)
            cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cuda_status(e);
        }
        b->graph_ready = true;
    }
    e = cudaGraphLaunch(b->graph, s);
    if (b->nitems > 0)
        note_launch();   // the graph's join kernel
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return cuda_status(e);
    if (b->ctl_host->err & kErrTimeout)
        return GJ_ERR_TIMEOUT;
    if (b->ctl_host->err)
        return GJ_ERR_CUDA;
    bool over = false;
    for (int32_t j = 0; j < b->njobs; ++j) {
        counts[j] = b->jpos_host[j];
        if (counts[j] > (caps ? caps[j] : 0) && outs && outs[j])
            over = true;
    }
    return over ? GJ_ERR_CAPACITY : GJ_OK;
}

int gj_batch_get_info(const gj_batch *b, int64_t *work_items, int64_t *total_points, uint64_t *candidate_pairs)
{
    if (!b)
        return GJ_ERR_INVALID_ARG;
    if (candidate_pairs)
        *candidate_pairs = b->candidates;
    if (work_items)
        *work_items = b->nitems;
    if (total_points)
        *total_points = b->n_total;
    return GJ_OK;
}

}  // extern "C"
