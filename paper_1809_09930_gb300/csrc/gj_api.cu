// gj_api.cu -- the C ABI (include/gj.h) and the batch loop of Alg. 1.
//
// gj_self_join follows Alg. 1's batch loop with the batching scheme of
// Sec. 3.2.2: a sampled count-only pass estimates |R|; the batch size b_s and
// the number of batches n_b >= 3 follow from it (b_s = 1e8 pairs when the
// estimate exceeds 3e8); each batch is one launch of the persistent join over
// a contiguous range of the load-ordered queue (the queue is interleaved so
// every range is a cost-stratified sample).  A batch whose results outgrow its
// buffer stops at committed work items and hands resume points to the next
// launch, so the result is exact whatever the estimate.  With a host output
// buffer the results of batch i are copied to the host on a second stream
// while batch i+1 runs (the HtoD / Kernel / DtoH overlap of Fig. 4).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <vector>

#include "gj_internal.cuh"

using namespace gj;

static thread_local int t_last_status = GJ_OK;
static std::atomic<unsigned long long> g_launches{0};

namespace gj {
void set_last_status(int st) { t_last_status = st; }

void pool_keep(int device)
{
    static std::atomic<uint64_t> done{0};
    if (device < 0 || device >= 64 || (done.load() >> device) & 1u)
        return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = (uint64_t)8 << 30;   // freed index memory up to 8 GiB stays with the pool
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done.fetch_or((uint64_t)1 << device);
}
gj_pair *device_view(gj_pair *p)
{
    if (!p)
        return nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)
        return p;
    return nullptr;
}
bool device_memory_of(const void *p, int device)
{
    cudaPointerAttributes a{};
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice && a.device == device) || a.type == cudaMemoryTypeManaged;
}
bool foreign_device(const void *p, int device)
{
    cudaPointerAttributes a{};
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device != device;
}
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
unsigned long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace gj

namespace {

// GJ_DEBUG=1 in the environment prints every CUDA failure the library maps
// to a status code (call site and CUDA's error string) to stderr.
bool debug_on()
{
    static const bool on = getenv("GJ_DEBUG") && getenv("GJ_DEBUG")[0] == '1';
    return on;
}

int cuda_status_at(cudaError_t e, const char *where)
{
    if (e == cudaSuccess)
        return GJ_OK;
    if (debug_on())
        fprintf(stderr, "gj: %s failed: %s (%d)\n", where, cudaGetErrorString(e), (int)e);
    if (e == cudaErrorMemoryAllocation)
        return GJ_ERR_OOM;
    return GJ_ERR_CUDA;
}
#define cuda_status(e) cuda_status_at((e), __func__)

__global__ void k_gather_queue(const uint32_t *__restrict__ order, int part, int nparts, int64_t nq,
                               int64_t nb, uint32_t *__restrict__ q)
{
    // Partition item of load rank r goes to batch r % nb at offset r / nb;
    // batch b occupies [b*qn + min(b, rem), ...) with qn = nq / nb,
    // rem = nq % nb.  Every batch range is then a stratified sample of the
    // descending-load order, itself in descending load.
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= nq)
        return;
    const int64_t qn = nq / nb, rem = nq % nb;
    const int64_t b = r % nb;
    q[b * qn + (b < rem ? b : rem) + r / nb] = order[(int64_t)part + r * nparts];
}

__global__ void k_stride_queue(const uint32_t *__restrict__ q, int64_t nq, int64_t stride, uint32_t *__restrict__ out,
                               int64_t nout)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < nout)
        out[t] = q[t * stride];
}

double now_ms()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

namespace gj {

// Launch state of the staged join whose sizes are fixed per handle (the grid
// and the work items are): allocated by the first staged join and kept until
// gj_free, so later joins allocate no pinned memory and create no events.
struct StagedState {
    JoinCtl *ctl = nullptr;
    JoinCtl *hctl_up = nullptr, *hctl_dn = nullptr;   // pinned
    Deferred *def[2] = {nullptr, nullptr};
    uint32_t dcap = 0;                                 // entries of each deferred list
    uint32_t *queue = nullptr, *qtmp = nullptr, *sample = nullptr;   // one entry per work item
    unsigned long long *span = nullptr, *hspan = nullptr;   // per-SM spans (device, pinned host)
    cudaEvent_t ev_k0 = nullptr, ev_k1 = nullptr, ev_ctl = nullptr, ev_drained[2] = {nullptr, nullptr};
    ~StagedState()
    {
        cudaFree(ctl);
        cudaFreeHost(hctl_up);
        cudaFreeHost(hctl_dn);
        cudaFree(def[0]);
        cudaFree(def[1]);
        cudaFree(queue);
        cudaFree(qtmp);
        cudaFree(sample);
        cudaFree(span);
        cudaFreeHost(hspan);
        if (ev_k0) cudaEventDestroy(ev_k0);
        if (ev_k1) cudaEventDestroy(ev_k1);
        if (ev_ctl) cudaEventDestroy(ev_ctl);
        for (auto &e : ev_drained)
            if (e) cudaEventDestroy(e);
    }
};

}  // namespace gj

namespace {

// One staged join's buffers: the handle's StagedState, borrowed, and the
// buffers whose sizes depend on the call (staging, result batches), taken from
// the stream-ordered pool and returned when the join ends.
struct JoinBuffers {
    JoinCtl *ctl = nullptr;
    JoinCtl *hctl_up = nullptr, *hctl_dn = nullptr;
    Deferred *def[2] = {nullptr, nullptr};
    uint32_t *queue = nullptr, *qtmp = nullptr, *sample = nullptr;
    unsigned long long *span = nullptr, *hspan = nullptr;
    cudaEvent_t ev_k0 = nullptr, ev_k1 = nullptr, ev_ctl = nullptr, ev_drained[2] = {nullptr, nullptr};
    gj_pair *staging = nullptr;
    gj_pair *dbuf[2] = {nullptr, nullptr};
    cudaStream_t s = nullptr, drain = nullptr;
    ~JoinBuffers()
    {
        // (a result batch may still be draining after an error)
        if (drain)
            cudaStreamSynchronize(drain);
        dev_free(staging, s);
        dev_free(dbuf[0], s);
        dev_free(dbuf[1], s);
    }
};

// The handle's staged-join state, made on first use; B borrows it.
cudaError_t staged_state(gj_index *h, int grid, JoinBuffers &B)
{
    if (!h->ss) {
        StagedState *t = new (std::nothrow) StagedState();
        if (!t)
            return cudaErrorMemoryAllocation;
        const size_t ni = (size_t)std::max<int64_t>(h->nitems, 1);
        t->dcap = (uint32_t)grid * 8u;   // a CTA defers at most the items in its pipeline
        cudaError_t e = cudaMalloc(&t->ctl, sizeof(JoinCtl));
        if (e == cudaSuccess) e = cudaMallocHost(&t->hctl_up, sizeof(JoinCtl));
        if (e == cudaSuccess) e = cudaMallocHost(&t->hctl_dn, sizeof(JoinCtl));
        if (e == cudaSuccess) e = cudaMalloc(&t->span, 2 * kSmSlots * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMallocHost(&t->hspan, 2 * kSmSlots * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMalloc(&t->def[0], (size_t)t->dcap * sizeof(Deferred));
        if (e == cudaSuccess) e = cudaMalloc(&t->def[1], (size_t)t->dcap * sizeof(Deferred));
        if (e == cudaSuccess) e = cudaMalloc(&t->queue, ni * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMalloc(&t->qtmp, ni * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMalloc(&t->sample, ni * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaEventCreate(&t->ev_k0);
        if (e == cudaSuccess) e = cudaEventCreate(&t->ev_k1);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t->ev_ctl, cudaEventBlockingSync);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t->ev_drained[0], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t->ev_drained[1], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            delete t;
            return e;
        }
        h->ss = t;
    }
    const StagedState &t = *h->ss;
    B.ctl = t.ctl;
    B.hctl_up = t.hctl_up;
    B.hctl_dn = t.hctl_dn;
    B.def[0] = t.def[0];
    B.def[1] = t.def[1];
    B.queue = t.queue;
    B.qtmp = t.qtmp;
    B.sample = t.sample;
    B.span = t.span;
    B.hspan = t.hspan;
    B.ev_k0 = t.ev_k0;
    B.ev_k1 = t.ev_k1;
    B.ev_ctl = t.ev_ctl;
    B.ev_drained[0] = t.ev_drained[0];
    B.ev_drained[1] = t.ev_drained[1];
    B.s = h->stream;
    return cudaSuccess;
}

IndexView view_of(const gj_index *h)
{
    IndexView v{};
    v.X = h->X;
    v.orig = h->orig;
    v.cell_start = h->cell_start;
    v.adj_start = h->adj_start;
    v.adj = h->adj;
    v.items = h->items;
    v.n = h->info.n;
    v.npad = h->npad;
    v.d = h->info.d;
    v.u = h->u;
    v.e2 = h->e2;
    v.ew = h->ew;
    v.ct = h->plain_ct;
    v.qb = h->qb;
    return v;
}

// Busy time of one launch: each SM's occupied span (earliest CTA start to
// latest CTA exit) averaged over the SMs that ran CTAs, in ms.  Co-resident
// CTAs that finish early leave their SM's span unchanged, so the figure never
// credits the survivors' speed-up to the whole SM.
double mean_sm_span_ms(const unsigned long long *span)
{
    double sum = 0.0;
    int used = 0;
    for (int i = 0; i < kSmSlots; ++i) {
        const unsigned long long t1 = span[kSmSlots + i];
        if (t1 == 0)
            continue;
        const unsigned long long t0 = ~span[i];
        if (t1 > t0)
            sum += (double)(t1 - t0);
        ++used;
    }
    return used ? sum / used * 1e-6 : 0.0;
}

// One launch of the persistent join; reads back the control block and the
// per-SM spans (their mean is added to *span_ms).
int run_launch(gj_index *h, JoinBuffers &B, JoinLaunch L, int grid, JoinCtl init, JoinCtl *result,
               double *kernel_ms, double *span_ms)
{
    cudaStream_t s = h->stream;
    *B.hctl_up = init;
    cudaError_t e = cudaMemcpyAsync(B.ctl, B.hctl_up, sizeof(JoinCtl), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(B.span, 0, 2 * kSmSlots * sizeof(unsigned long long), s);
    if (e != cudaSuccess)
        return cuda_status(e);
    L.ctl = B.ctl;
    L.sm_span = B.span;
    cudaEventRecord(B.ev_k0, s);
    e = h->tc_ready ? launch_join_tc(h, L, grid, s, false) : launch_join_plain(L, grid, s);
    if (e != cudaSuccess)
        return cuda_status(e);
    cudaEventRecord(B.ev_k1, s);
    e = cudaMemcpyAsync(B.hctl_dn, B.ctl, sizeof(JoinCtl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B.hspan, B.span, 2 * kSmSlots * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess)
        return cuda_status(e);
    cudaEventRecord(B.ev_ctl, s);
    e = cudaEventSynchronize(B.ev_ctl);
    if (e != cudaSuccess)
        return cuda_status(e);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, B.ev_k0, B.ev_k1);
    *kernel_ms += ms;
    *span_ms += mean_sm_span_ms(B.hspan);
    *result = *B.hctl_dn;
    if (result->err & (kErrStaging | kErrDeferred)) {
        if (debug_on())
            fprintf(stderr, "gj: join kernel reported error bits 0x%x\n", result->err);
        return GJ_ERR_CUDA;
    }
    if (result->err & kErrTimeout)
        return GJ_ERR_TIMEOUT;
    return GJ_OK;
}

void free_direct_state(gj_index *h)
{
    cudaFree(h->jd_ctl);
    cudaFreeHost(h->jd_hctl);
    cudaFree(h->jd_queue);
    cudaFree(h->jd_span);
    cudaFreeHost(h->jd_hspan);
    if (h->jd_ev0)
        cudaEventDestroy(h->jd_ev0);
    if (h->jd_ev1)
        cudaEventDestroy(h->jd_ev1);
    h->jd_ctl = h->jd_hctl = nullptr;
    h->jd_queue = nullptr;
    h->jd_span = h->jd_hspan = nullptr;
    h->jd_ev0 = h->jd_ev1 = nullptr;
    h->jd_ready = false;
}

// The tensor-core join's direct form: one launch over the part's work items
// that writes pairs straight into `out` (device-addressable, cap pairs; pairs
// past cap are counted, not written) or, with out == nullptr, only counts.
// No estimate, batches, staging or resume: the output either holds R or the
// call reports GJ_ERR_CAPACITY with |R|.  The launch state lives on the handle.
int join_tc_direct(gj_index *h, int part, int nparts, int64_t nq, int grid, gj_pair *out, uint64_t cap,
                   uint64_t *total)
{
    cudaStream_t s = h->stream;
    cudaError_t e = cudaSuccess;
    if (!h->jd_ready) {
        e = cudaMalloc(&h->jd_ctl, sizeof(JoinCtl));
        if (e == cudaSuccess) e = cudaMallocHost(&h->jd_hctl, sizeof(JoinCtl));
        if (e == cudaSuccess) e = cudaMalloc(&h->jd_queue, (size_t)std::max<int64_t>(h->nitems, 1) * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMalloc(&h->jd_span, 2 * kSmSlots * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMallocHost(&h->jd_hspan, 2 * kSmSlots * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaEventCreate(&h->jd_ev0);
        if (e == cudaSuccess) e = cudaEventCreate(&h->jd_ev1);
        if (e != cudaSuccess) {
            free_direct_state(h);
            return cuda_status(e);
        }
        h->jd_ready = true;
    }
    note_launch();
    k_gather_queue<<<(int)((nq + 255) / 256), 256, 0, s>>>(h->order, part, nparts, nq, 1, h->jd_queue);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(h->jd_ctl, 0, sizeof(JoinCtl), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->jd_span, 0, 2 * kSmSlots * sizeof(unsigned long long), s);
    if (e != cudaSuccess)
        return cuda_status(e);
    JoinLaunch L{};
    L.ix = view_of(h);
    L.queue = h->jd_queue;
    L.qlimit = (uint32_t)nq;
    L.ctl = h->jd_ctl;
    L.sm_span = h->jd_span;
    L.out = out;
    L.cap = out ? cap : 0;
    cudaEventRecord(h->jd_ev0, s);
    e = launch_join_tc(h, L, grid, s, true);
    if (e != cudaSuccess)
        return cuda_status(e);
    cudaEventRecord(h->jd_ev1, s);
    e = cudaMemcpyAsync(h->jd_hctl, h->jd_ctl, sizeof(JoinCtl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->jd_hspan, h->jd_span, 2 * kSmSlots * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return cuda_status(e);
    const JoinCtl res = *h->jd_hctl;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->jd_ev0, h->jd_ev1);
    *total = out ? res.pos : res.counted;
    h->last.pairs = *total;
    h->last.launches = 1;
    h->last.join_ms = ms;
    h->last.busy_ms = mean_sm_span_ms(h->jd_hspan);
    h->last.tc_survivors = res.survivors;
    h->last.evaluated = res.evaluated;
    h->last.dims = res.dims;
    h->last.batches_planned = 1;
    if (res.err & kErrTimeout)
        return GJ_ERR_TIMEOUT;
    if (res.err)
        return GJ_ERR_CUDA;
    return GJ_OK;
}

int join_impl(gj_index *h, int part, int nparts, gj_pair *pairs_out, uint64_t cap, uint64_t *count)
{
    if (!h || !count || nparts < 1 || part < 0 || part >= nparts || (!pairs_out && cap > 0))
        return GJ_ERR_INVALID_ARG;
    const double t_start = now_ms();
    *count = 0;
    memset(&h->last, 0, sizeof(h->last));
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess)
        return cuda_status(e);
    if (pairs_out && foreign_device(pairs_out, h->device))
        return GJ_ERR_INVALID_ARG;   // another device's memory
    cudaStream_t s = h->stream;
    const int64_t nitems = h->nitems;
    const int64_t nq = nitems > part ? (nitems - part + nparts - 1) / nparts : 0;
    if (nq == 0) {
        h->last.total_ms = now_ms() - t_start;
        return GJ_OK;
    }
    const int per_sm = h->tc_ready ? 1 : plain_ctas_per_sm(h->info.d, h->plain_ct, h->qb);
    if (per_sm < 1)
        return GJ_ERR_UNSUPPORTED;
    const int grid = h->sms * per_sm;
    // pairs per CTA staging area: plain >= 4 tiles of output; tensor-core: two halves
    const uint32_t stg_cap = 1u << 16;
    const size_t stg_per_cta = h->tc_ready ? tc_staging_pairs_per_cta() : (size_t)stg_cap;
    // The kernels write device memory only.  Host output (pageable or
    // pinned) reaches the host by copies: through the result batches of
    // Sec. 3.2.2, or, for a tensor-core index, from one device buffer of cap
    // pairs filled by the direct form.
    gj_pair *const direct = device_view(pairs_out);
    const bool dev_out = direct != nullptr;
    const bool count_only_call = (cap == 0);

    if (h->tc_ready && (dev_out || count_only_call)) {
        uint64_t total = 0;
        const int st = join_tc_direct(h, part, nparts, nq, grid, count_only_call ? nullptr : direct, cap, &total);
        *count = total;
        h->last.total_ms = now_ms() - t_start;
        if (st != GJ_OK)
            return st;
        return total > cap ? GJ_ERR_CAPACITY : GJ_OK;
    }
    if (h->tc_ready && !(h->cfg.flags & GJ_HOST_BATCHED)) {
        // host output: the direct form into a device buffer of cap pairs (from
        // the stream-ordered pool), then one copy of the pairs written; with no
        // room for the buffer, the result batches below
        gj_pair *dbuf = nullptr;
        if (dev_alloc(&dbuf, (size_t)cap * sizeof(gj_pair), h->stream) == cudaSuccess) {
            uint64_t total = 0;
            int st = join_tc_direct(h, part, nparts, nq, grid, dbuf, cap, &total);
            if (st == GJ_OK) {
                const uint64_t ncopy = std::min<uint64_t>(total, cap);
                cudaError_t e = ncopy ? cudaMemcpyAsync(pairs_out, dbuf, ncopy * sizeof(gj_pair),
                                                        cudaMemcpyDeviceToHost, h->stream)
                                      : cudaSuccess;
                if (e == cudaSuccess)
                    e = cudaStreamSynchronize(h->stream);
                if (e != cudaSuccess)
                    st = cuda_status(e);
            }
            dev_free(dbuf, h->stream);
            *count = total;
            h->last.total_ms = now_ms() - t_start;
            if (st != GJ_OK)
                return st;
            return total > cap ? GJ_ERR_CAPACITY : GJ_OK;
        }
        cudaGetLastError();
    }

    JoinBuffers B;
#define TRYC(x)                                                     \
    do {                                                            \
        cudaError_t _e = (x);                                       \
        if (_e != cudaSuccess)                                      \
            return cuda_status_at(_e, #x);                          \
    } while (0)
    TRYC(staged_state(h, grid, B));
    const uint32_t dcap = h->ss->dcap;

    JoinLaunch L{};
    L.ix = view_of(h);
    L.dout_cap = dcap;
    L.stg_cap = stg_cap;
    double kms = 0.0;
    uint32_t launches = 0;
    unsigned long long evaluated = 0, dims = 0, survivors = 0;
    double busy_ms = 0.0;

    // ---- 1. sampled estimate of |R| (count-only over every S-th item), Sec. 3.2.2
    note_launch();
    k_gather_queue<<<(int)((nq + 255) / 256), 256, 0, s>>>(h->order, part, nparts, nq, 1, B.qtmp);
    TRYC(cudaGetLastError());
    uint64_t estimate = 0;
    const bool want_batches = !count_only_call && !dev_out;
    if (want_batches && !h->drain_stream)
        TRYC(cudaStreamCreateWithFlags(&h->drain_stream, cudaStreamNonBlocking));
    B.drain = want_batches ? h->drain_stream : nullptr;
    const int64_t S = std::max<int64_t>(1, std::min<int64_t>(100, nq / std::max(1, grid)));
    if (want_batches && h->cfg.batch_pairs == 0 && S >= 8) {
        const int64_t ns = (nq + S - 1) / S;   // <= nq / 8 + 1: fits the state's sample array
        note_launch();
        k_stride_queue<<<(int)((ns + 255) / 256), 256, 0, s>>>(B.qtmp, nq, S, B.sample, ns);
        TRYC(cudaGetLastError());
        JoinLaunch Ls = L;
        Ls.queue = B.sample;
        Ls.qlimit = (uint32_t)ns;
        Ls.out = nullptr;
        Ls.staging = nullptr;
        Ls.din = nullptr;
        Ls.n_din = 0;
        Ls.dout = B.def[0];
        JoinCtl init{};
        init.fail_base = ~0ull;
        JoinCtl res{};
        double est_ms = 0.0, est_span = 0.0;
        int st0 = run_launch(h, B, Ls, grid, init, &res, &est_ms, &est_span);
        if (st0 != GJ_OK)
            return st0;
        estimate = (uint64_t)((double)res.counted * (double)nq / (double)ns);
        h->last.estimate_ms = est_ms;
    }

    // ---- 2. batch size and count (Sec. 3.2.2: n_b >= 3; b_s = 1e8 above 3e8)
    uint64_t bs;
    int64_t nb;
    if (h->cfg.batch_pairs) {
        bs = h->cfg.batch_pairs;
        nb = std::max<int64_t>(3, (int64_t)((estimate + bs - 1) / bs));
    } else if (estimate > 300000000ull) {
        bs = 100000000ull;
        nb = (int64_t)((estimate + bs - 1) / bs);
    } else {
        nb = 3;
        bs = std::max<uint64_t>((uint64_t)((double)estimate / 3.0 * 1.25), (uint64_t)1 << 20);
    }
    if (!want_batches)
        nb = 1;
    nb = std::max<int64_t>(1, std::min<int64_t>(nb, nq));
    h->last.estimate = estimate;
    h->last.batches_planned = (uint32_t)nb;
    h->last.batch_pairs = want_batches ? bs : 0;

    // the dequeue order: nb interleaved ranges of the load order
    note_launch();
    k_gather_queue<<<(int)((nq + 255) / 256), 256, 0, s>>>(h->order, part, nparts, nq, nb, B.queue);
    TRYC(cudaGetLastError());
    const int64_t qn = nq / nb, rem = nq % nb;
    auto batch_end = [&](int64_t b) { return (b + 1) * qn + std::min<int64_t>(b + 1, rem); };

    if (want_batches) {
        TRYC(dev_alloc(&B.dbuf[0], bs * sizeof(gj_pair), s));
        TRYC(dev_alloc(&B.dbuf[1], bs * sizeof(gj_pair), s));
    }
    if (!count_only_call)
        TRYC(dev_alloc(&B.staging, (size_t)grid * stg_per_cta * sizeof(gj_pair), s));

    // ---- 3. batch loop
    uint64_t written = 0, total = 0;
    uint32_t head = 0, n_din = 0;
    int cur = 0;
    bool counting = count_only_call;
    int64_t batch = 0;
    int st = GJ_OK;
    bool drained_pending[2] = {false, false};
    for (int guard = 0; guard < 1000000; ++guard) {
        const uint32_t qlimit = (uint32_t)std::min<int64_t>(nq, batch_end(batch));
        if (head >= (uint32_t)nq && n_din == 0)
            break;
        JoinLaunch Lb = L;
        Lb.queue = B.queue;
        Lb.qlimit = qlimit;
        Lb.din = B.def[cur];
        Lb.n_din = n_din;
        Lb.dout = B.def[cur ^ 1];
        uint64_t lcap = 0;
        gj_pair *lout = nullptr;
        if (!counting) {
            if (dev_out) {
                lout = direct + written;
                lcap = cap - written;
            } else {
                lout = B.dbuf[launches & 1];
                lcap = bs;
                if (drained_pending[launches & 1])
                    TRYC(cudaStreamWaitEvent(s, B.ev_drained[launches & 1], 0));
            }
            if (lcap == 0)
                counting = true;
        }
        Lb.out = counting ? nullptr : lout;
        Lb.cap = counting ? 0 : lcap;
        Lb.staging = counting ? nullptr : B.staging;
        JoinCtl init{};
        init.fail_base = ~0ull;
        init.head = head;
        JoinCtl res{};
        st = run_launch(h, B, Lb, grid, init, &res, &kms, &busy_ms);
        if (st != GJ_OK)
            break;
        ++launches;
        evaluated += res.evaluated;
        dims += res.dims;
        survivors += res.survivors;
        if (counting) {
            total += res.counted;
        } else {
            uint64_t valid = res.full ? std::min<unsigned long long>(res.pos, res.fail_base) : res.pos;
            total += valid;
            if (!dev_out && valid) {
                const int slot = (launches - 1) & 1;
                uint64_t room = cap > written ? cap - written : 0;
                uint64_t ncopy = std::min<uint64_t>(valid, room);
                if (ncopy) {
                    TRYC(cudaEventRecord(B.ev_ctl, s));
                    TRYC(cudaStreamWaitEvent(h->drain_stream, B.ev_ctl, 0));
                    TRYC(cudaMemcpyAsync(pairs_out + written, B.dbuf[slot], ncopy * sizeof(gj_pair),
                                         cudaMemcpyDeviceToHost, h->drain_stream));
                    TRYC(cudaEventRecord(B.ev_drained[slot], h->drain_stream));
                    drained_pending[slot] = true;
                }
                written += ncopy;
                if (ncopy < valid)   // user buffer full: the rest is only counted
                    counting = true;
            } else if (dev_out) {
                written += valid;
                if (res.full)        // user buffer full: the rest is only counted
                    counting = true;
            }
        }
        n_din = std::min<uint32_t>(res.dout_n, dcap);
        cur ^= 1;
        head = std::min<uint32_t>(res.head, qlimit);
        if (head >= qlimit && batch + 1 < nb)
            ++batch;
    }
    if (st == GJ_OK && h->drain_stream)
        TRYC(cudaStreamSynchronize(h->drain_stream));
    TRYC(cudaStreamSynchronize(s));
#undef TRYC
    *count = total;
    h->last.pairs = total;
    h->last.launches = launches;
    h->last.join_ms = kms;
    h->last.busy_ms = busy_ms;
    h->last.total_ms = now_ms() - t_start;
    h->last.tc_survivors = survivors;
    h->last.evaluated = evaluated;
    h->last.dims = dims;
    if (st != GJ_OK)
        return st;
    if (!count_only_call && total > cap)
        return GJ_ERR_CAPACITY;
    if (count_only_call && total > 0)
        return GJ_ERR_CAPACITY;
    return GJ_OK;
}

}  // namespace

extern "C" {

void gj_config_init(gj_config *cfg)
{
    if (!cfg)
        return;
    memset(cfg, 0, sizeof(*cfg));
    cfg->k = 0;
    cfg->flags = GJ_DEFAULT_FLAGS;
    cfg->stream = nullptr;
    cfg->batch_pairs = 0;
    cfg->device = -1;
}

gj_index *gj_index_build_ex(const double *points, int64_t n, int32_t d, double eps, const gj_config *cfg_in)
{
    gj_config cfg;
    if (cfg_in)
        cfg = *cfg_in;
    else
        gj_config_init(&cfg);
    if (n < 0 || d < 1 || !(eps > 0.0) || !isfinite(eps) || (n > 0 && !points) || cfg.k < 0) {
        t_last_status = GJ_ERR_INVALID_ARG;
        return nullptr;
    }
    if (n >= ((int64_t)1 << 32) || d > GJ_MAX_DIMS) {
        t_last_status = GJ_ERR_TOO_LARGE;
        return nullptr;
    }
    if (cfg.k > std::min(d, MAXK) || cfg.query_block < 0 || (cfg.query_block > 0 && cfg.query_block < 8) ||
        cfg.query_block > QB || (cfg.tile != 0 && cfg.tile != 32 && cfg.tile != 64)) {
        t_last_status = GJ_ERR_INVALID_ARG;
        return nullptr;
    }
    if ((cfg.flags & GJ_AUTOTUNE) && cfg.k == 0) {
        // timed trials pick the settings; the winning trial's index is returned
        gj_index *best = nullptr;
        gj_tune_result r;
        const int st = autotune_impl(points, n, d, eps, &cfg, &r, &best);
        t_last_status = st;
        return st == GJ_OK ? best : nullptr;
    }
    int dev = cfg.device;
    cudaError_t e;
    if (dev < 0) {
        e = cudaGetDevice(&dev);
    } else {
        e = cudaSetDevice(dev);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        t_last_status = GJ_ERR_UNSUPPORTED;
        return nullptr;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess || prop.major != 10 || prop.minor != 3) {
        t_last_status = GJ_ERR_UNSUPPORTED;
        return nullptr;
    }
    gj_index *h = new (std::nothrow) gj_index();
    if (!h) {
        t_last_status = GJ_ERR_OOM;
        return nullptr;
    }
    h->device = dev;
    pool_keep(dev);
    h->cfg = cfg;
    h->sms = prop.multiProcessorCount;
    h->info.n = n;
    h->info.d = d;
    h->info.eps = eps;
    h->info.flags = cfg.flags;
    h->e2 = eps * eps;
    h->ew = eps * (1.0 + ldexp(1.0, -40));
    int st = GJ_OK;
    double *P = nullptr;
    unsigned int *flag = nullptr;
    unsigned int hflag = 0;
    if (cfg.stream) {
        h->stream = (cudaStream_t)cfg.stream;
        h->own_stream = false;
    } else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        h->own_stream = true;
        if (e != cudaSuccess) {
            st = cuda_status(e);
            goto fail;
        }
    }
    // (the drain stream of host-output joins is made by the first such join)
    e = dev_alloc(&P, std::max<size_t>((size_t)n * d, 1) * sizeof(double), h->stream);
    if (e == cudaSuccess)
        e = dev_alloc(&flag, sizeof(unsigned int), h->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(flag, 0, sizeof(unsigned int), h->stream);
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync(P, points, (size_t)n * d * sizeof(double), cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess)
        e = launch_check_finite(P, n * (int64_t)d, flag, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&hflag, flag, sizeof(unsigned int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        st = cuda_status(e);
        goto fail;
    }
    if (hflag) {
        st = GJ_ERR_NONFINITE;
        goto fail;
    }
    st = build_index(h, P, n, d, eps, cfg.k, cfg.flags, h->stream);
    if (st != GJ_OK)
        goto fail;
    dev_free(P, h->stream);
    dev_free(flag, h->stream);
    t_last_status = GJ_OK;
    return h;
fail:
    dev_free(P, h->stream);
    dev_free(flag, h->stream);
    gj_free(h);
    cudaGetLastError();
    t_last_status = st;
    return nullptr;
}

gj_index *gj_index_build(const double *points, int64_t n, int32_t d, double eps, int32_t k)
{
    gj_config cfg;
    gj_config_init(&cfg);
    cfg.k = k;
    return gj_index_build_ex(points, n, d, eps, &cfg);
}

int gj_self_join(gj_index *h, gj_pair *pairs_out, uint64_t cap, uint64_t *count)
{
    int st = join_impl(h, 0, 1, pairs_out, cap, count);
    if (st == GJ_ERR_CAPACITY && cap == 0 && !pairs_out)
        return GJ_OK;   // count-only query
    return st;
}

int gj_self_join_part(gj_index *h, int32_t part, int32_t nparts, gj_pair *pairs_out, uint64_t cap,
                      uint64_t *count)
{
    int st = join_impl(h, part, nparts, pairs_out, cap, count);
    if (st == GJ_ERR_CAPACITY && cap == 0 && !pairs_out)
        return GJ_OK;
    return st;
}

int gj_index_get_info(const gj_index *h, gj_index_info_t *info)
{
    if (!h || !info)
        return GJ_ERR_INVALID_ARG;
    *info = h->info;
    return GJ_OK;
}

int gj_last_join_stats(const gj_index *h, gj_join_stats *st)
{
    if (!h || !st)
        return GJ_ERR_INVALID_ARG;
    *st = h->last;
    return GJ_OK;
}

void gj_free(gj_index *h)
{
    if (!h)
        return;
    cudaSetDevice(h->device);
    // index memory is returned to the pool in stream order: after the work
    // already queued on the handle's stream, without waiting here
    const cudaStream_t s = h->stream;
    dev_free(h->X, s);
    dev_free(h->orig, s);
    dev_free(h->cell_start, s);
    dev_free(h->cell_id, s);
    dev_free(h->adj_start, s);
    dev_free(h->adj, s);
    dev_free(h->items, s);
    dev_free(h->order, s);
    dev_free(h->XA, s);
    dev_free(h->XB, s);
    dev_free(h->tc_centre, s);
    dev_free(h->XR, s);
    dev_free(h->perm_dev, s);
    if (h->jd_ready || h->ss) {
        cudaStreamSynchronize(s);
        if (h->jd_ready)
            free_direct_state(h);
        delete h->ss;
        h->ss = nullptr;
    }
    if (h->drain_stream)
        cudaStreamDestroy(h->drain_stream);
    if (h->own_stream && h->stream)
        cudaStreamDestroy(h->stream);
    delete h;
}

int gj_last_status(void) { return t_last_status; }

const char *gj_status_string(int status)
{
    switch (status) {
    case GJ_OK: return "ok";
    case GJ_ERR_INVALID_ARG: return "invalid argument";
    case GJ_ERR_NONFINITE: return "a coordinate is NaN or infinite";
    case GJ_ERR_OOM: return "out of device or pinned host memory";
    case GJ_ERR_CUDA: return "CUDA error";
    case GJ_ERR_CAPACITY: return "result larger than the output capacity";
    case GJ_ERR_TIMEOUT: return "a bounded device wait ran out";
    case GJ_ERR_UNSUPPORTED: return "no usable GPU (needs compute capability 10.3)";
    case GJ_ERR_TOO_LARGE: return "input too large (n >= 2^32 or d > GJ_MAX_DIMS)";
    default: return "unknown status";
    }
}

const char *gj_version(void) { return "0.1.0"; }

unsigned long long gj_kernel_launches(void) { return launches_so_far(); }

int gj_probe_fp64_tflops(int device, double *tflops)
{
    if (!tflops)
        return GJ_ERR_INVALID_ARG;
    int dev = device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess)
        return GJ_ERR_UNSUPPORTED;
    if (cudaSetDevice(dev) != cudaSuccess)
        return GJ_ERR_UNSUPPORTED;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return GJ_ERR_CUDA;
    const int grid = prop.multiProcessorCount * 8, iters = 1 << 14;
    double *out = nullptr;
    cudaStream_t s;
    cudaEvent_t a, b;
    if (cudaMalloc(&out, grid * sizeof(double)) != cudaSuccess)
        return GJ_ERR_OOM;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    launch_fp64_probe(out, iters, grid, s);   // warm-up
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(a, s);
        launch_fp64_probe(out, iters, grid, s);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        best = std::min(best, ms);
    }
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamDestroy(s);
    cudaFree(out);
    if (e != cudaSuccess)
        return GJ_ERR_CUDA;
    *tflops = 2.0 * 8.0 * iters * (double)grid * 256.0 / (best * 1e-3) / 1e12;
    return GJ_OK;
}

}  // extern "C"
