// rime_stream.cu -- rime_chi2_streamed: chi^2 (eq. 7) of an observation whose
// data and weights stay in host memory, in time chunks (Sec. 4.4).
//
// The paper subdivides a problem that does not fit the GPU along time and
// keeps two solvers, so that the transfer of one chunk's data overlaps the
// computation of the other's; the chunk chi^2 values are then added. Here the
// "solvers" are a ring of up to four device buffers: chunk i's data and
// weights are copied on a copy stream into buffer i mod n while the fused
// kernel reduces earlier chunks. More than two buffers let the copies run
// ahead of the kernels. The chunk kernels alternate between the context's
// stream (even chunks) and a second kernel stream (odd chunks), so that one
// chunk's blocks take the SM slots that the previous chunk's last blocks free
// instead of waiting for that launch to drain; each chunk kernel has its own
// range of block partials and each kernel stream its own last-block counter.
// Events order the streams:
//   copied[b]  (copy stream)    -> the kernel of the chunk in buffer b may start;
//   free[b]    (kernel stream)  -> buffer b may be overwritten (n chunks on);
//   start      (context stream, end of the previous call) -> the buffers are free;
//   upload     (context stream, after its latest upload copy) -> the chunk
//              copies may start: they overlap the kernels that follow the
//              uploads (input checks, delays) but do not queue ahead of them;
//   entry      (context stream, at the call) -> the second kernel stream may
//              start (the chunk kernels need the sky model set before the call);
//   k2         (second kernel stream, its last chunk) -> the chunk sum may start.
// Each chunk's data are checked on arrival; each chunk's kernel writes its
// chi^2 to its own slot, and one thread adds the slots in chunk order, so the
// result does not depend on the chunking schedule's timing.
#include "rime_internal.cuh"

#include <algorithm>

namespace rime {
namespace {

__global__ void k_sum_in_order(int n, const double *in, double *out, const DevStatus *st) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    if (inputs_bad(st)) return;
    double s = 0.0;
    for (int i = 0; i < n; i++) s += in[i];
    *out = s;
}

// Makes `nbuf` chunk buffers of `bytes` each (fewer, but at least two, when
// the ring would take more than half of the free device memory) and room for
// `nchunks` chunk results; creates the copy stream and events on first use.
// Returns the number of buffers to use in `*nuse`.
cudaError_t ensure(rime_ctx *c, size_t bytes, int nbuf, int nchunks, int *nuse) {
    cudaError_t e;
    if (!c->copy_stream) {
        e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        e = cudaStreamCreateWithFlags(&c->kstream2, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        for (cudaEvent_t *ev : {&c->ev_start, &c->ev_entry, &c->ev_k2}) {
            e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
            if (e != cudaSuccess) return e;
        }
        Alloc alloc{c};
        e = alloc((void **)&c->d_stream_counters, 2 * sizeof(unsigned));
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(c->d_stream_counters, 0, 2 * sizeof(unsigned), c->stream);
        if (e != cudaSuccess) return e;
        for (int b = 0; b < rime_ctx::kStreamBufs; b++) {
            e = cudaEventCreateWithFlags(&c->ev_copied[b], cudaEventDisableTiming);
            if (e != cudaSuccess) return e;
            e = cudaEventCreateWithFlags(&c->ev_free[b], cudaEventDisableTiming);
            if (e != cudaSuccess) return e;
        }
    }
    if (bytes > c->sbuf_cap || nbuf > c->sbuf_asked) {
        for (int b = 0; b < rime_ctx::kStreamBufs; b++) {
            if (c->d_sbuf[b]) cudaFree(c->d_sbuf[b]);
            c->d_sbuf[b] = nullptr;
        }
        c->sbuf_cap = 0;
        c->sbuf_n = 0;
        c->sbuf_asked = nbuf;
        size_t free_b = 0, total_b = 0;
        if (nbuf > 2 && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
            nbuf = (int)std::max<size_t>(2, std::min<size_t>(nbuf, free_b / 2 / std::max<size_t>(bytes, 1)));
        Alloc alloc{c};
        for (int b = 0; b < nbuf; b++) {
            e = alloc(&c->d_sbuf[b], bytes);
            if (e != cudaSuccess) return e;
            c->sbuf_n = b + 1;
        }
        c->sbuf_cap = bytes;
    }
    *nuse = std::min(nbuf, c->sbuf_n);
    if ((size_t)nchunks > c->schi_cap) {
        if (c->d_schi) cudaFree(c->d_schi);
        c->d_schi = nullptr;
        c->schi_cap = 0;
        Alloc alloc{c};
        e = alloc((void **)&c->d_schi, (size_t)nchunks * sizeof(double));
        if (e != cudaSuccess) return e;
        c->schi_cap = nchunks;
    }
    return cudaSuccess;
}

}  // namespace
}  // namespace rime

using namespace rime;

#define CKS(c, call, what)                                         \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail_ctx(c, e_, what);  \
    } while (0)

extern "C" {

int32_t rime_stream_chunk_ntime(const rime_ctx *c) {
    if (!c) return 0;
    // about one wave of the fused kernel per chunk (2 blocks on each of the
    // device's SMs): the chunk kernels alternate between two streams, so a
    // launch's last blocks do not hold the next chunk back, and short chunks
    // start the kernels sooner after the first copy (measured on the
    // 64-antenna, 100-timestep, 64-channel chi^2: chunks of 4-6 timesteps
    // 2.53 ms, of 19 timesteps 2.82 ms, against 2.22 ms for the copies alone)
    rime_ctx *m = const_cast<rime_ctx *>(c);   // caches the SM count
    if (m->nsm <= 0 && cudaDeviceGetAttribute(&m->nsm, cudaDevAttrMultiProcessorCount, m->device) != cudaSuccess)
        m->nsm = 152;
    long long per_t = narrow_applies(c) ? narrow_blocks_per_time(m) : (long long)c->dims.nchan * c->nunits;
    long long nt = (2LL * m->nsm + per_t - 1) / std::max(1LL, per_t);
    return (int32_t)std::max(1LL, std::min<long long>(nt, c->dims.ntime));
}

rime_status rime_chi2_streamed(rime_ctx *c, const void *data, const void *weight, int32_t chunk_ntime,
                               double *chi2) {
    if (!c) return fail_ctx(nullptr, RIME_E_INVALID, "ctx is NULL");
    if (!data) return fail_ctx(c, RIME_E_INVALID, "data is NULL");
    if (!chi2) return fail_ctx(c, RIME_E_INVALID, "chi2 is NULL");
    if (!c->sources_set) return fail_ctx(c, RIME_E_STATE, "rime_set_sources has not been called");
    const int ntime = c->dims.ntime;
    const int nt = chunk_ntime > 0 ? std::min<int>(chunk_ntime, ntime) : rime_stream_chunk_ntime(c);
    // the first chunk's copy is the one no kernel hides: a quarter-length
    // first chunk (library-chosen lengths only) starts the kernels sooner
    const int first = chunk_ntime > 0 ? nt : std::max(1, nt / 4);
    const int nchunks = 1 + (ntime - first + nt - 1) / nt;
    const size_t ts = c->tsize();
    const size_t vis_t = (size_t)c->nbl * c->dims.nchan;           // visibilities per timestep
    const size_t dbytes = vis_t * 8 * ts, wbytes = vis_t * ts;      // per timestep
    int nbuf = 0;
    CKS(c, ensure(c, (size_t)nt * std::max(dbytes + wbytes, (size_t)16), std::min(nchunks, rime_ctx::kStreamBufs),
                  nchunks, &nbuf),
        "allocating chunk buffers");
    CKS(c, reset_status_class(c, EC_SDATA), "reset status");
    // the copy stream must not overwrite a buffer that the previous streamed
    // call's kernels still read; it need not wait for the rest of the
    // context's work (uploads of uvw, gains, sources), which the copies overlap
    if (c->stream_used) CKS(c, cudaStreamWaitEvent(c->copy_stream, c->ev_start, 0), "stream wait");
    // nor queue ahead of the context's own uploads (one DMA queue serves
    // both streams' host-to-device copies in the order they become ready)
    if (c->upload_marked) CKS(c, cudaStreamWaitEvent(c->copy_stream, c->ev_upload, 0), "stream wait");
    // device-memory inputs may be written by work queued on the context's
    // stream: then the copies follow that work
    auto on_device = [](const void *p) {
        cudaPointerAttributes a;
        if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();   // clear a sticky "invalid value" from an unknown pointer
            return false;
        }
        return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
    };
    CKS(c, cudaEventRecord(c->ev_entry, c->stream), "event");
    if (on_device(data) || on_device(weight)) CKS(c, cudaStreamWaitEvent(c->copy_stream, c->ev_entry, 0), "stream wait");
    CKS(c, cudaStreamWaitEvent(c->kstream2, c->ev_entry, 0), "stream wait");
    // the chunk kernels' block partials: chunk [t0, t0 + nti) owns blocks
    // [t0 bpt, (t0 + nti) bpt) of the context's partials buffer
    const bool narrow = narrow_applies(c);
    const long long bpt = narrow ? narrow_blocks_per_time(c) : (long long)c->dims.nchan * c->nunits;
    if ((long long)ntime * bpt > (long long)c->partials_cap)
        return fail_ctx(c, RIME_E_INVALID, "internal: block partials exceed their buffer");
    // long FP32 source lists fold into per-block running sums: the second
    // kernel stream's chunks get their own scratch
    const bool seg2 = !narrow && c->dims.precision == RIME_FP32 && (long long)c->nsrc > seg_source_threshold();
    if (seg2) CKS(c, ensure_segsum2(c), "allocating the running sums of long source lists");
    const char *hd = static_cast<const char *>(data);
    const char *hw = static_cast<const char *>(weight);
    for (int i = 0; i < nchunks; i++) {
        const int b = i % nbuf;
        const int t0 = i == 0 ? 0 : first + (i - 1) * nt;
        const int nti = std::min(i == 0 ? first : nt, ntime - t0);
        char *bd = static_cast<char *>(c->d_sbuf[b]);
        char *bw = bd + (size_t)nt * dbytes;
        if (i >= nbuf) CKS(c, cudaStreamWaitEvent(c->copy_stream, c->ev_free[b], 0), "stream wait");
        CKS(c, cudaMemcpyAsync(bd, hd + (size_t)t0 * dbytes, (size_t)nti * dbytes, cudaMemcpyDefault, c->copy_stream),
            "copying a data chunk");
        if (hw)
            CKS(c, cudaMemcpyAsync(bw, hw + (size_t)t0 * wbytes, (size_t)nti * wbytes, cudaMemcpyDefault,
                                   c->copy_stream),
                "copying a weight chunk");
        CKS(c, cudaEventRecord(c->ev_copied[b], c->copy_stream), "event");
        cudaStream_t ks = (i & 1) ? c->kstream2 : c->stream;
        CKS(c, cudaStreamWaitEvent(ks, c->ev_copied[b], 0), "stream wait");
        CKS(c, launch_validate_chunk(c, (long long)nti * vis_t, bd, hw ? bw : nullptr, EC_SDATA,
                                     (long long)t0 * vis_t, ks),
            "checking a chunk");
        // the kernels index data and weights by the global timestep: hand them
        // base addresses t0 rows before the chunk (never dereferenced there)
        FusedParams P{};
        fill_fused_params(c, P, nullptr, c->d_schi + i, nullptr, nullptr);
        P.t_begin = t0;
        P.segsum = seg2 && (i & 1) ? c->d_segsum2 : nullptr;   // the two streams' kernels run side by side
        P.data = reinterpret_cast<const void *>(reinterpret_cast<uintptr_t>(bd) - (uintptr_t)t0 * dbytes);
        P.weight = hw ? reinterpret_cast<const void *>(reinterpret_cast<uintptr_t>(bw) - (uintptr_t)t0 * wbytes)
                      : nullptr;
        P.has_weight = hw != nullptr;
        P.partials = c->d_partials + (long long)t0 * bpt;
        P.counter = c->d_stream_counters + (i & 1);
        cudaError_t e = narrow ? launch_narrow_params(c, MODE_CHI2, P, nti, ks)
                               : launch_tiled_params(c, MODE_CHI2, P, (long long)nti * bpt, ks);
        CKS(c, e, "chunk chi2 kernel");
        CKS(c, cudaEventRecord(c->ev_free[b], ks), "event");
    }
    CKS(c, cudaEventRecord(c->ev_k2, c->kstream2), "event");
    CKS(c, cudaStreamWaitEvent(c->stream, c->ev_k2, 0), "stream wait");
    k_sum_in_order<<<1, 32, 0, c->stream>>>(nchunks, c->d_schi, &c->d_status->chi2, c->d_status);
    CKS(c, cudaGetLastError(), "chunk sum");
    CKS(c, cudaEventRecord(c->ev_start, c->stream), "event");   // the buffers' last readers
    c->stream_used = true;
    rime_status s = sync_status_ctx(c);
    // streamed data errors belong to this call only
    cudaError_t e = reset_status_class(c, EC_SDATA);
    if (s != RIME_OK) return s;
    CKS(c, e, "reset status");
    *chi2 = c->h_status->chi2;
    return RIME_OK;
}

}  // extern "C"
