// rime_batched.cu -- rime_chi2_batched: chi^2 of many sky models (the
// proposals of one sampler iteration) against one observation.
//
// FP32: one persistent launch (k_batched_f32, rime_fused.cu) over work items
// (t, channel group, antenna unit, group of sets), each the fused predict +
// chi^2 of its sets' sources for the unit's baselines, then one fixed-order
// sum per set.
// FP64, and arrays the small-array kernel takes: one launch per set.
//
// The schedule (set order and source offsets) reaches the device as kernel
// arguments, so a captured CUDA graph carries it and replays stand alone.
// The launch configuration (channels and sets per work item, blocks per SM,
// set order) is chosen by timing each candidate on a sample of the work (the
// first timesteps of every set) on the first call for a given number of sets
// and sources, unless a call fixes it.
#include "rime_internal.cuh"

#include <algorithm>
#include <climits>
#include <cstring>
#include <numeric>
#include <vector>

using namespace rime;

namespace {

#define CKB(c, call, what)                                         \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail_ctx(c, e_, what);  \
    } while (0)

// 1000 ints per launch keeps the kernel's arguments under 4 KB.
constexpr int kChunkInts = 1000;
struct IntChunk {
    int n;
    int v[kChunkInts];
};

__global__ void k_put_ints(int *dst, const IntChunk c) {
    for (int i = threadIdx.x; i < c.n; i += blockDim.x) dst[i] = c.v[i];
}

cudaError_t put_ints(int *dst, const int *src, size_t n, cudaStream_t st) {
    for (size_t i = 0; i < n; i += kChunkInts) {
        IntChunk ch;
        ch.n = (int)std::min<size_t>(kChunkInts, n - i);
        std::memcpy(ch.v, src + i, sizeof(int) * ch.n);
        k_put_ints<<<1, 256, 0, st>>>(dst + i, ch);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

constexpr int kCpi[] = {1, 2, 4};
constexpr int kGsets[] = {1, 4, 16};

struct Sched {
    int nsets;
    int max_set;          // sources of the largest set
    int per_set;          // partials per set
    const int *order[2];  // device: by size, by index
    const int *offsets;   // device
};

BatchParams batch_params(rime_ctx *c, const Sched &S, const rime_batch_config &cfg, int ntime_items) {
    BatchParams B{};
    B.cpi = cfg.channels_per_item;
    B.nkc = (c->dims.nchan + B.cpi - 1) / B.cpi;
    B.nsets = S.nsets;
    B.gsets = cfg.sets_per_item;
    B.ngroups = (S.nsets + B.gsets - 1) / B.gsets;
    B.nitems = (long long)ntime_items * B.nkc * c->nunits * B.ngroups;
    B.per_set = S.per_set;
    B.order = S.order[cfg.order];
    B.offsets = S.offsets;
    B.counter = c->d_bcounter;
    B.partials = c->d_bpart;
    B.max_set = S.max_set;
    return B;
}

cudaError_t run_batched(rime_ctx *c, const Sched &S, const rime_batch_config &cfg, int ntime_items) {
    cudaError_t e = cudaMemsetAsync(c->d_bcounter, 0, sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return e;
    const BatchParams B = batch_params(c, S, cfg, ntime_items);
    const long long grid = std::min<long long>((long long)c->nsm * cfg.blocks_per_sm, B.nitems);
    return launch_batched_f32(c, B, (int)grid);
}

// Times every candidate on the first timesteps of every set; best first.
rime_status tune(rime_ctx *c, const Sched &S, rime_batch_config &best) {
    const int tt = std::max(1, std::min(c->dims.ntime, c->dims.ntime / 16));
    std::vector<rime_batch_config> cand;
    for (int cpi : kCpi) {
        if (cpi > 1 && cpi > c->dims.nchan) continue;
        for (int gs : kGsets) {
            if (gs > 1 && gs > S.nsets) continue;
            for (int bps = std::min(2, c->bmax_bps); bps >= 1; bps--)
                for (int order = 0; order < 2; order++) {
                    rime_batch_config x{};
                    x.channels_per_item = cpi;
                    x.blocks_per_sm = bps;
                    x.order = order;
                    x.sets_per_item = gs;
                    cand.push_back(x);
                }
        }
    }
    cudaEvent_t e0, e1;
    CKB(c, cudaEventCreate(&e0), "tuning events");
    CKB(c, cudaEventCreate(&e1), "tuning events");
    rime_batch_config rec{};
    int ibest = -1;
    float tbest = 0.f;
    cudaError_t err = cudaSuccess;
    for (size_t i = 0; i < cand.size() && err == cudaSuccess && i < 40; i++) {
        float tmin = 0.f;
        for (int rep = 0; rep < 2 && err == cudaSuccess; rep++) {
            err = cudaEventRecord(e0, c->stream);
            if (err == cudaSuccess) err = run_batched(c, S, cand[i], tt);
            if (err == cudaSuccess) err = cudaEventRecord(e1, c->stream);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            if (rep == 0 || ms < tmin) tmin = ms;
        }
        rec.trial_cfg[i][0] = cand[i].channels_per_item;
        rec.trial_cfg[i][1] = cand[i].blocks_per_sm;
        rec.trial_cfg[i][2] = cand[i].order;
        rec.trial_cfg[i][3] = cand[i].sets_per_item;
        rec.trial_ms[i] = tmin;
        rec.ntrials = (int)i + 1;
        if (ibest < 0 || tmin < tbest) {
            ibest = (int)i;
            tbest = tmin;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail_ctx(c, err, "batched tuning trials");
    rec.channels_per_item = cand[ibest].channels_per_item;
    rec.blocks_per_sm = cand[ibest].blocks_per_sm;
    rec.order = cand[ibest].order;
    rec.sets_per_item = cand[ibest].sets_per_item;
    rec.tuned = 1;
    best = rec;
    return RIME_OK;
}

}  // namespace

extern "C" {

rime_status rime_chi2_batched(rime_ctx *c, int32_t nsets, const int32_t *off, const rime_sources *all,
                              double *chi2_dev) {
    if (!c) return fail_ctx(nullptr, RIME_E_INVALID, "ctx is NULL");
    if (nsets < 0) return fail_ctx(c, RIME_E_INVALID, "nsets must be >= 0");
    if (!all) return fail_ctx(c, RIME_E_INVALID, "sources is NULL");
    if (nsets > 0 && (!off || !chi2_dev)) return fail_ctx(c, RIME_E_INVALID, "src_offsets or chi2_dev is NULL");
    if (!c->has_data) return fail_ctx(c, RIME_E_STATE, "no observed data (rime_set_data)");
    if (nsets > 0) {
        if (off[0] != 0) return fail_ctx(c, RIME_E_INVALID, "src_offsets[0] must be 0");
        for (int j = 0; j < nsets; j++)
            if (off[j + 1] < off[j]) return fail_ctx(c, RIME_E_INVALID, "src_offsets must be non-decreasing");
        if (off[nsets] != all->nsrc)
            return fail_ctx(c, RIME_E_INVALID, "src_offsets[nsets] must equal the number of sources");
    }
    const long long per_set = (long long)c->dims.ntime * c->dims.nchan * c->nunits;
    if (nsets > 0 && per_set > LLONG_MAX / 8 / nsets) return fail_ctx(c, RIME_E_INVALID, "too many sets");
    rime_status st = rime_set_sources(c, all);
    if (st != RIME_OK) return st;
    if (nsets == 0) return RIME_OK;

    // buffers
    Alloc alloc{c};
    if ((size_t)nsets > c->bsched_cap) {
        if (c->d_bsched) cudaFree(c->d_bsched);
        c->d_bsched = nullptr;
        c->bsched_cap = 0;
        CKB(c, alloc((void **)&c->d_bsched, (3 * (size_t)nsets + 1) * sizeof(int)), "allocating the schedule");
        c->bsched_cap = nsets;
    }
    const size_t npart = (size_t)nsets * per_set;
    if (c->dims.precision == RIME_FP32 && npart > c->bpart_cap) {
        if (c->d_bpart) cudaFree(c->d_bpart);
        c->d_bpart = nullptr;
        c->bpart_cap = 0;
        CKB(c, alloc((void **)&c->d_bpart, npart * sizeof(double)), "allocating batched partials");
        c->bpart_cap = npart;
    }
    if (!c->d_bcounter) CKB(c, alloc((void **)&c->d_bcounter, sizeof(unsigned long long)), "allocating a counter");

    // one launch per set: FP64, and small arrays (whose tiled work items would
    // be nearly empty blocks); each set's chi^2 is that of a plain call
    if (c->dims.precision == RIME_FP64 || narrow_applies(c)) {
        for (int j = 0; j < nsets; j++)
            CKB(c, narrow_applies(c) ? launch_narrow(c, MODE_CHI2, nullptr, chi2_dev + j, off[j], off[j + 1])
                                     : launch_fused_f64_range(c, off[j], off[j + 1], chi2_dev + j),
                "batched per-set kernel");
        return RIME_OK;
    }

    // schedule: ranks by size (largest first, ties by index) and by index
    const size_t cap = c->bsched_cap;
    std::vector<int> host(3 * cap + 1, 0);
    std::iota(host.begin(), host.begin() + nsets, 0);
    std::stable_sort(host.begin(), host.begin() + nsets,
                     [&](int a, int b) { return off[a + 1] - off[a] > off[b + 1] - off[b]; });
    std::iota(host.begin() + cap, host.begin() + cap + nsets, 0);
    std::copy(off, off + nsets + 1, host.begin() + 2 * cap);
    CKB(c, put_ints(c->d_bsched, host.data(), nsets, c->stream), "uploading the schedule");
    CKB(c, put_ints(c->d_bsched + cap, host.data() + cap, nsets, c->stream), "uploading the schedule");
    CKB(c, put_ints(c->d_bsched + 2 * cap, host.data() + 2 * cap, (size_t)nsets + 1, c->stream),
        "uploading the schedule");
    const int max_set = off[host[0] + 1] - off[host[0]];   // host[0]: the largest set's index
    Sched S{nsets, max_set, (int)per_set, {c->d_bsched, c->d_bsched + cap}, c->d_bsched + 2 * cap};

    if (c->bmax_bps == 0) {
        c->bmax_bps = std::max(1, batched_blocks_per_sm());
        CKB(c, cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device), "device attributes");
    }
    rime_batch_config cfg{};
    if (c->bcfg_forced) {
        cfg = c->bcfg;
        cfg.blocks_per_sm = std::min(cfg.blocks_per_sm, c->bmax_bps);
    } else {
        const rime_ctx::BatchTune *hit = nullptr;
        for (const auto &e : c->btuned)
            if (e.nsets == nsets && e.nsrc == all->nsrc) hit = &e;
        if (hit) {
            cfg = hit->cfg;
        } else {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            CKB(c, cudaStreamIsCapturing(c->stream, &cs), "capture status");
            if (cs == cudaStreamCaptureStatusNone) {
                st = tune(c, S, cfg);
                if (st != RIME_OK) return st;
                c->btuned.push_back({nsets, all->nsrc, cfg});
            } else {   // no timing inside a capture: the default configuration
                cfg.channels_per_item = 1;
                cfg.blocks_per_sm = std::min(2, c->bmax_bps);
                cfg.order = 0;
                cfg.sets_per_item = 1;
            }
        }
    }
    c->bcfg = cfg;
    CKB(c, run_batched(c, S, cfg, c->dims.ntime), "batched chi2 kernel");
    CKB(c, launch_set_sums(c, nsets, (int)per_set, c->d_bpart, chi2_dev), "batched chi2 sums");
    return RIME_OK;
}

rime_status rime_batched_config(const rime_ctx *c, rime_batch_config *out) {
    if (!c) return fail_ctx(nullptr, RIME_E_INVALID, "ctx is NULL");
    if (!out) return fail_ctx(const_cast<rime_ctx *>(c), RIME_E_INVALID, "out is NULL");
    *out = c->bcfg;
    return RIME_OK;
}

rime_status rime_set_batched_config(rime_ctx *c, const rime_batch_config *cfg) {
    if (!c) return fail_ctx(nullptr, RIME_E_INVALID, "ctx is NULL");
    if (!cfg) {
        c->bcfg_forced = false;
        return RIME_OK;
    }
    const int cpi = cfg->channels_per_item;
    if (cpi != 1 && cpi != 2 && cpi != 4) return fail_ctx(c, RIME_E_INVALID, "channels_per_item must be 1, 2 or 4");
    if (cfg->blocks_per_sm != 1 && cfg->blocks_per_sm != 2)
        return fail_ctx(c, RIME_E_INVALID, "blocks_per_sm must be 1 or 2");
    if (cfg->order != 0 && cfg->order != 1) return fail_ctx(c, RIME_E_INVALID, "order must be 0 or 1");
    if (cfg->sets_per_item < 1 || cfg->sets_per_item > 64)
        return fail_ctx(c, RIME_E_INVALID, "sets_per_item must be 1..64");
    rime_batch_config x{};
    x.channels_per_item = cpi;
    x.blocks_per_sm = cfg->blocks_per_sm;
    x.order = cfg->order;
    x.sets_per_item = cfg->sets_per_item;
    c->bcfg = x;
    c->bcfg_forced = true;
    return RIME_OK;
}

}  // extern "C"
