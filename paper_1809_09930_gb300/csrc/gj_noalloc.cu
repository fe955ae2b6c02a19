// gj_noalloc.cu -- a self-join entry point that allocates no memory.
//
// gj_self_join (gj_api.cu) allocates its launch state with cudaMalloc on
// every call: the control block, the dequeue order of the work items, the
// deferred lists and the per-CTA staging areas.  Some callers cannot let a
// library do that: a service whose device memory is reserved up front by a
// caching allocator (a cudaMalloc from outside the pool can fail or fragment
// it), or a latency-bound loop that must never enter the driver's allocator.
// gj_self_join_noalloc serves them.  It runs the plain FP64 join with pairs
// written straight into the caller's device buffer, and keeps its own scratch
// -- the control block and the work-item order -- in one file-scope
// __device__ array of fixed size, which every GPU that loads the library holds
// until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "gj_internal.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)4 << 20;   // 4 MiB
constexpr size_t kCtlBytes = 256;                    // control block, padded
constexpr uint64_t kMaxItems = (kScratchBytes - kCtlBytes) / sizeof(uint32_t);
constexpr int kMaxDevices = 64;

static_assert(sizeof(gj::JoinCtl) <= kCtlBytes, "control block does not fit its slot");

// The scratch.  In host code this name is only a host-side stand-in for the
// device array, never a device address: host code takes the address with
// cudaGetSymbolAddress (below) and passes that pointer to kernels.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
struct ScratchAt {
    unsigned long long ctx;   // unique id of the context the address belongs to
    void *addr;
};
ScratchAt g_scratch_at[kMaxDevices] = {};

// Unique id of the calling thread's current context (0 when unknown).  A
// device reset destroys the context the cached address belongs to, and the
// next context on that device gets a new id.
unsigned long long current_context_id()
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        cudaGetLastError();
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of the scratch on `dev` (the current device), looked up with
// cudaGetSymbolAddress once per device and context: the first call on a
// device, and the first after that device's context was reset, does this
// set-up.  (With no context id available it is looked up on every call.)
int scratch_address(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices)
        return GJ_ERR_UNSUPPORTED;
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lk(g_mu);
    ScratchAt &at = g_scratch_at[dev];
    if (!at.addr || ctx == 0 || at.ctx != ctx) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return GJ_ERR_CUDA;
        }
        at.addr = p;
        at.ctx = ctx;
    }
    *out = static_cast<unsigned char *>(at.addr);
    return GJ_OK;
}

__global__ void k_noalloc_queue(const uint32_t *__restrict__ order, int part, int nparts, int64_t nq,
                                uint32_t *__restrict__ q)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < nq)
        q[t] = order[(int64_t)part + t * nparts];
}

}  // namespace

extern "C" int gj_self_join_noalloc(const gj_index *h, int32_t part, int32_t nparts, gj_pair *pairs_out,
                                    uint64_t cap, uint64_t *count)
{
    using namespace gj;
    if (!h || !count || nparts < 1 || part < 0 || part >= nparts || (!pairs_out && cap > 0))
        return GJ_ERR_INVALID_ARG;
    if (h->tc_ready)
        return GJ_ERR_INVALID_ARG;   // built with GJ_TC_FILTER: use gj_self_join
    *count = 0;
    if (cudaSetDevice(h->device) != cudaSuccess) {
        cudaGetLastError();
        return GJ_ERR_CUDA;
    }
    if (pairs_out && !device_memory_of(pairs_out, h->device))
        return GJ_ERR_INVALID_ARG;   // the output must be device memory of the handle's device
    const int64_t nitems = h->nitems;
    const int64_t nq = nitems > part ? (nitems - part + nparts - 1) / nparts : 0;
    if ((uint64_t)nq > kMaxItems)
        return GJ_ERR_TOO_LARGE;
    unsigned char *scratch = nullptr;
    int st = scratch_address(h->device, &scratch);
    if (st != GJ_OK)
        return st;
    if (nq == 0)
        return GJ_OK;
    const int per_sm = plain_ctas_per_sm(h->info.d, h->plain_ct, h->qb);
    if (per_sm < 1)
        return GJ_ERR_UNSUPPORTED;
    cudaStream_t s = h->stream;
    JoinCtl *ctl = reinterpret_cast<JoinCtl *>(scratch);
    uint32_t *queue = reinterpret_cast<uint32_t *>(scratch + kCtlBytes);

    // every call shares the scratch and finds the last call's contents: clear
    // the control block (counters, queue head) before the launch
    cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(JoinCtl), s);
    if (e == cudaSuccess) {
        note_launch();
        k_noalloc_queue<<<(int)((nq + 255) / 256), 256, 0, s>>>(h->order, part, nparts, nq, queue);
        e = cudaGetLastError();
    }
    JoinLaunch L{};
    L.ix.X = h->X;
    L.ix.orig = h->orig;
    L.ix.cell_start = h->cell_start;
    L.ix.adj_start = h->adj_start;
    L.ix.adj = h->adj;
    L.ix.items = h->items;
    L.ix.n = h->info.n;
    L.ix.npad = h->npad;
    L.ix.d = h->info.d;
    L.ix.ct = h->plain_ct;
    L.ix.qb = h->qb;
    L.ix.u = h->u;
    L.ix.e2 = h->e2;
    L.ix.ew = h->ew;
    L.queue = queue;
    L.qlimit = (uint32_t)nq;
    L.ctl = ctl;
    L.out = cap ? pairs_out : nullptr;
    L.cap = cap;
    if (e == cudaSuccess)
        e = launch_join_plain_direct(L, h->sms * per_sm, s);
    JoinCtl res;
    memset(&res, 0, sizeof(res));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&res, ctl, sizeof(JoinCtl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GJ_ERR_CUDA;
    }
    if (res.err & kErrTimeout)
        return GJ_ERR_TIMEOUT;
    if (res.err)
        return GJ_ERR_CUDA;
    const uint64_t total = cap ? res.pos : res.counted;
    *count = total;
    if (cap && total > cap)
        return GJ_ERR_CAPACITY;
    if (!pairs_out && cap == 0)
        return GJ_OK;   // count-only
    return total > cap ? GJ_ERR_CAPACITY : GJ_OK;
}
