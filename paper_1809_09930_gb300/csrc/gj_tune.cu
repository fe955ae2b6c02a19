// gj_tune.cu -- the autotuner of the single-join form: k, query block,
// candidate tile and result batch size by timed trials.
//
// The paper fixes k from a comparison of candidate counts against the cost of
// the index search (Sec. 4.1) and b_s by a rule (Sec. 3.2.2).  Here each
// candidate setting is built and timed instead:
//   * a trial builds the index with the setting (host wall time, device
//     synchronous) and runs a count-only join over one part of an entity
//     partition of the load-ordered work items (Sec. 6.2: block r goes to part
//     r mod N_b, so a part is a load-stratified sample).  The part's join time
//     is the kernel's busy time -- each SM's occupied span (earliest CTA start
//     to latest CTA exit) averaged over the SMs, i.e. the part's work spread
//     evenly, without the tail a small sample has -- scaled by N_b.  N_b comes
//     from a first, finely sampled trial of the builder's own choice, so that
//     a trial's join takes about 40 ms (at most 32 parts);
//   * k sweeps 1..min(d, 8) (1..3 for the tensor-core form) with the default
//     tiles and stops once the cost has grown past twice the best for two
//     consecutive k; then the tiles are tried at the best k;
//   * the least build + join time wins (a later setting must be 2 % faster,
//     so near-ties keep the smaller k and the default tiles); its index is kept when the caller
//     wants it (gj_index_build_ex with GJ_AUTOTUNE);
//   * b_s comes from the winner's |R| estimate, a timed device-to-host copy
//     and the measured per-launch overhead (see pick_batch_pairs).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "gj_internal.cuh"

namespace gj {
namespace {

double wall_ms()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Trial {
    gj_config cfg;
    double build_ms = 0, join_ms = 0;
    uint64_t est_pairs = 0;
    double cost() const { return build_ms + join_ms; }
};

constexpr double kTrialTargetMs = 40.0;   // sampled join time a trial aims for
constexpr int kMaxParts = 32;

// Parts of the trial's entity partition: np_req when given, else as many as
// leave at least two work items per resident CTA in the timed part (at most
// kMaxParts); never so many that the part has fewer items than CTAs.
int trial_parts(const gj_index *h, int np_req)
{
    const int per_sm = h->tc_ready ? 1 : std::max(1, plain_ctas_per_sm(h->info.d, h->plain_ct, h->qb));
    const int64_t ctas = (int64_t)h->sms * per_sm;
    const int64_t cap = std::max<int64_t>(1, std::min<int64_t>(kMaxParts, h->nitems / (2 * ctas)));
    return (int)(np_req > 0 ? std::min<int64_t>(np_req, cap) : cap);
}

// One timed trial.  On success *h_out holds the trial's index.
int run_trial(const double *P, int64_t n, int d, double eps, int np_req, Trial *t, gj_index **h_out)
{
    *h_out = nullptr;
    gj_config c = t->cfg;
    c.flags &= ~(GJ_AUTOTUNE | GJ_TUNE_FORM);
    const double t0 = wall_ms();
    gj_index *h = gj_index_build_ex(P, n, d, eps, &c);
    if (!h)
        return gj_last_status();
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        gj_free(h);
        return e == cudaErrorMemoryAllocation ? GJ_ERR_OOM : GJ_ERR_CUDA;
    }
    t->build_ms = wall_ms() - t0;
    const int np = trial_parts(h, np_req);
    const int part = np / 2;
    uint64_t cnt = 0;
    double best = INFINITY;
    // the first launch of a kernel in a process includes loading it: a short
    // trial runs twice and keeps the faster
    for (int rep = 0; rep < 2; ++rep) {
        int st = gj_self_join_part(h, part, np, nullptr, 0, &cnt);
        if (st != GJ_OK) {
            gj_free(h);
            return st;
        }
        best = std::min(best, np > 1 ? h->last.busy_ms : h->last.join_ms);
        if (h->last.join_ms > 20.0)
            break;
    }
    t->join_ms = best * np;
    t->est_pairs = cnt * (uint64_t)np;
    *h_out = h;
    return GJ_OK;
}

// b_s for host output.  With J the join time, C the device-to-host copy time
// of |R| and o the fixed cost of one batch (launch + control round trip), n_b
// batches take about max(J, C) + min(J, C)/n_b + n_b*o when each batch's
// drain overlaps the next batch's join; n_b >= 3 (Sec. 3.2.2) and two batch
// buffers stay within an eighth of the free device memory.
int pick_batch_pairs(int device, cudaStream_t s, uint64_t est_pairs, double join_ms, uint64_t *bs_out)
{
    *bs_out = 0;
    if (est_pairs == 0)
        return GJ_OK;
    const size_t probe = (size_t)std::min<uint64_t>(est_pairs * sizeof(gj_pair), (uint64_t)64 << 20);
    const size_t bytes = std::max<size_t>(probe, 1 << 20);
    void *dbuf = nullptr, *hbuf = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaMalloc(&dbuf, bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&hbuf, bytes);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double bw = 0.0, o_ms = INFINITY;
    if (e == cudaSuccess) e = cudaMemsetAsync(dbuf, 0, bytes, s);
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hbuf, dbuf, bytes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms > 0.f)
            bw = std::max(bw, (double)bytes / ms);   // bytes per ms
    }
    for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
        const double t0 = wall_ms();
        e = cudaMemcpyAsync(hbuf, dbuf, 64, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        o_ms = std::min(o_ms, wall_ms() - t0);
    }
    size_t free_b = 0, total_b = 0;
    if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(dbuf);
    cudaFreeHost(hbuf);
    if (e != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? GJ_ERR_OOM : GJ_ERR_CUDA;
    // a batch also launches the join and reads its control block back
    o_ms = 2.0 * o_ms + 0.02;
    const double C = bw > 0 ? (double)est_pairs * sizeof(gj_pair) / bw : 0.0;
    const double J = join_ms;
    const double hi = std::max(J, C), lo = std::min(J, C);
    const uint64_t max_bs = std::max<uint64_t>((uint64_t)(free_b / 16 / sizeof(gj_pair)), (uint64_t)1 << 20);
    const int64_t nb_min = std::max<int64_t>(3, (int64_t)((est_pairs + max_bs - 1) / max_bs));
    int64_t best_nb = nb_min;
    double best_t = INFINITY;
    for (int64_t nb = nb_min; nb <= std::max<int64_t>(nb_min, 4096); nb = nb < 64 ? nb + 1 : nb + nb / 8) {
        const double tt = hi + lo / (double)nb + (double)nb * o_ms;
        if (tt < best_t) {
            best_t = tt;
            best_nb = nb;
        }
    }
    // a margin for the estimate: a batch that fills early only adds a resume launch
    *bs_out = std::max<uint64_t>((uint64_t)ceil((double)est_pairs * 1.1 / (double)best_nb), (uint64_t)1 << 16);
    return GJ_OK;
}

}  // namespace

int autotune_impl(const double *points, int64_t n, int d, double eps, const gj_config *cfg_in, gj_tune_result *out,
                  gj_index **best_out)
{
    if (best_out)
        *best_out = nullptr;
    if (!out)
        return GJ_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    gj_config base;
    if (cfg_in)
        base = *cfg_in;
    else
        gj_config_init(&base);
    if (n < 0 || d < 1 || !(eps > 0.0) || !isfinite(eps) || (n > 0 && !points))
        return GJ_ERR_INVALID_ARG;
    if (n >= ((int64_t)1 << 32) || d > GJ_MAX_DIMS)
        return GJ_ERR_TOO_LARGE;
    base.flags &= ~GJ_AUTOTUNE;

    // the input is copied to the device once; every trial builds from the copy
    const double *P = points;
    double *Pdev = nullptr;
    int device = base.device;
    cudaError_t e = device < 0 ? cudaGetDevice(&device) : cudaSetDevice(device);
    if (e != cudaSuccess)
        return GJ_ERR_UNSUPPORTED;
    base.device = device;
    // host memory or another device's memory is copied to this device first
    const bool on_dev = n > 0 && device_memory_of(points, device);
    if (n > 0 && !on_dev) {
        e = cudaMalloc(&Pdev, (size_t)n * d * sizeof(double));
        if (e == cudaSuccess)
            e = cudaMemcpy(Pdev, points, (size_t)n * d * sizeof(double), cudaMemcpyDefault);
        if (e != cudaSuccess) {
            cudaFree(Pdev);
            return e == cudaErrorMemoryAllocation ? GJ_ERR_OOM : GJ_ERR_CUDA;
        }
        P = Pdev;
    }

    std::vector<bool> forms;   // true = tensor-core filter
    const bool tc_ok = ((d + 4 + 15) / 16) * 16 <= 128;
    if (base.flags & GJ_TUNE_FORM) {
        forms.push_back(false);
        if (tc_ok)
            forms.push_back(true);
    } else {
        forms.push_back((base.flags & GJ_TC_FILTER) && tc_ok);
    }

    Trial best;
    bool have = false;
    gj_index *best_h = nullptr;
    int trials = 0, st = GJ_OK;
    // calibration: the builder's own choice, sampled finely, sizes the sample
    // of every trial so that its join takes about kTrialTargetMs
    int np_req = kMaxParts;
    {
        Trial t;
        t.cfg = base;
        t.cfg.flags &= ~GJ_TUNE_FORM;
        if (!forms[0])
            t.cfg.flags &= ~GJ_TC_FILTER;
        t.cfg.k = 0;
        gj_index *h = nullptr;
        st = run_trial(P, n, d, eps, kMaxParts, &t, &h);
        ++trials;
        gj_free(h);
        if (st == GJ_OK)
            np_req = (int)std::max(1.0, std::min((double)kMaxParts, floor(t.join_ms / kTrialTargetMs)));
    }
    auto consider = [&](Trial &t) -> int {
        gj_index *h = nullptr;
        const int s2 = run_trial(P, n, d, eps, np_req, &t, &h);
        ++trials;
        if (s2 != GJ_OK)
            return s2;
        // a later setting must win by 2 %: ties go to the earlier (smaller k, default tiles)
        if (!have || t.cost() < 0.98 * best.cost()) {
            best = t;
            have = true;
            gj_free(best_h);
            best_h = h;
        } else {
            gj_free(h);
        }
        return GJ_OK;
    };

    for (size_t f = 0; f < forms.size() && st == GJ_OK; ++f) {
        const bool tc = forms[f];
        const int kmax = std::min(std::min(d, MAXK), tc ? 3 : MAXK);
        double form_best = INFINITY;
        int form_best_k = 1, worse = 0;
        for (int k = 1; k <= kmax && st == GJ_OK; ++k) {
            Trial t;
            t.cfg = base;
            t.cfg.flags = tc ? (base.flags | GJ_TC_FILTER) : (base.flags & ~GJ_TC_FILTER);
            t.cfg.flags &= ~GJ_TUNE_FORM;
            t.cfg.k = k;
            t.cfg.query_block = 0;
            t.cfg.tile = 0;
            st = consider(t);
            if (st != GJ_OK)
                break;
            if (t.cost() < form_best) {
                form_best = t.cost();
                form_best_k = k;
                worse = 0;
            } else if (t.cost() > 2.0 * form_best && ++worse >= 2) {
                break;
            }
        }
        if (st != GJ_OK)
            break;
        // tiles at the best k of this form
        const int dflt_ct = d <= 32 ? 64 : 32;
        for (int qb : {0, 64}) {   // 0: the default blocks (120 points plain; 128-aligned tensor-core)
            for (int ct : {64, 32}) {
                if (tc && ct != 64)
                    continue;
                if (qb == 0 && (tc || ct == dflt_ct))
                    continue;   // the default, timed in the sweep
                Trial t;
                t.cfg = base;
                t.cfg.flags = tc ? (base.flags | GJ_TC_FILTER) : (base.flags & ~GJ_TC_FILTER);
                t.cfg.flags &= ~GJ_TUNE_FORM;
                t.cfg.k = form_best_k;
                t.cfg.query_block = qb;
                t.cfg.tile = tc ? 0 : ct;
                st = consider(t);
                if (st != GJ_OK)
                    break;
            }
            if (st != GJ_OK)
                break;
        }
    }
    cudaFree(Pdev);
    if (st != GJ_OK || !have) {
        gj_free(best_h);
        return st != GJ_OK ? st : GJ_ERR_INVALID_ARG;
    }
    uint64_t bs = 0;
    st = pick_batch_pairs(device, best_h->stream, best.est_pairs, best.join_ms, &bs);
    if (st != GJ_OK) {
        gj_free(best_h);
        return st;
    }
    out->k = best_h->info.k;
    out->flags = best.cfg.flags;
    out->query_block = best.cfg.query_block;   // 0 = the default blocks
    out->tile = best_h->tc_ready ? 0 : (best.cfg.tile ? best.cfg.tile : (d <= 32 ? 64 : 32));
    out->batch_pairs = bs;
    out->est_pairs = best.est_pairs;
    out->build_ms = best.build_ms;
    out->join_ms = best.join_ms;
    out->trials = trials;
    if (best_out) {
        best_h->cfg.batch_pairs = bs;
        best_h->cfg.k = best_h->info.k;
        *best_out = best_h;
    } else {
        gj_free(best_h);
    }
    return GJ_OK;
}

}  // namespace gj

extern "C" int gj_autotune(const double *points, int64_t n, int32_t d, double eps, const gj_config *cfg,
                           gj_tune_result *out)
{
    return gj::autotune_impl(points, n, d, eps, cfg, out, nullptr);
}
