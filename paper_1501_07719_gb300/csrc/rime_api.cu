// rime_api.cu -- the C ABI declared in include/rime.h.
//
// Host-side argument checks happen before any CUDA call, so that invalid
// sizes and pointers are reported without touching the GPU. Value checks of
// uploaded arrays run on the GPU (rime_prep.cu) and are reported by the next
// call that waits for the stream.
#include "rime_internal.cuh"

#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace rime {
void build_units(int na, int precision, std::vector<Unit> &units, std::vector<Tile> &tiles);
}

using namespace rime;

namespace rime {
size_t alloc_cap() {
    const char *s = std::getenv("RIME_TEST_MAX_BYTES");
    return s ? (size_t)std::strtoull(s, nullptr, 10) : (size_t)-1;
}
}  // namespace rime

namespace {

thread_local std::string g_create_error;

// Upper limits that keep every index of the kernels inside int32 grid sizes
// and the tile offsets inside uint8.
constexpr long long kMaxNa = 4096;
constexpr long long kMaxBlocks = 2147483647LL;

rime_status fail(rime_ctx *c, rime_status s, const std::string &msg) {
    if (c) c->err = msg;
    else g_create_error = msg;
    return s;
}

rime_status cuda_fail(rime_ctx *c, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? RIME_E_OOM : RIME_E_CUDA, m);
}

#define CK(c, call, what)                                   \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

}  // namespace

rime_status rime::fail_ctx(rime_ctx *c, rime_status s, const std::string &msg) { return fail(c, s, msg); }
rime_status rime::cuda_fail_ctx(rime_ctx *c, cudaError_t e, const char *what) { return cuda_fail(c, e, what); }

namespace {

void free_all(rime_ctx *c) {
    void *ptrs[] = {c->d_freq, c->d_chan, c->d_uvw, c->d_uvw_f, c->d_pointing, c->d_data,
                    c->d_weight, c->d_gains_in, c->d_gains, c->d_src_in, c->d_stokes,
                    c->d_gauss, c->d_alpha, c->d_src_extra, c->d_tau, c->d_rho, c->d_units,
                    c->d_tiles, c->d_partials, c->d_counter, c->d_status, c->d_yadj, c->d_gpart,
                    c->d_gunits, c->d_gbl, c->d_bsched, c->d_bpart, c->d_bcounter, c->d_stiles,
                    c->d_spart, c->d_scounter, c->d_sscale, c->d_schi,
                    c->d_chainN, c->d_chain_scratch, c->d_pair, c->d_pair_kind, c->d_chain_part, c->d_segsum,
                    c->d_dgain, c->d_segsum2};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (void *p : c->d_sbuf)
        if (p) cudaFree(p);
    if (c->d_stream_counters) cudaFree(c->d_stream_counters);
    for (cudaEvent_t e : {c->ev_start, c->ev_entry, c->ev_upload, c->ev_k2})
        if (e) cudaEventDestroy(e);
    for (int b = 0; b < rime_ctx::kStreamBufs; b++) {
        if (c->ev_copied[b]) cudaEventDestroy(c->ev_copied[b]);
        if (c->ev_free[b]) cudaEventDestroy(c->ev_free[b]);
    }
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->kstream2) cudaStreamDestroy(c->kstream2);
    if (c->h_status) cudaFreeHost(c->h_status);
}

__global__ void k_reset_status(DevStatus *st, int cls) {
    if (cls < 0) {
        st->chi2 = 0.0;
        st->aux = 0.0;
        for (int i = 0; i < EC_N; i++) {
            st->err[i] = 0;
            st->first_bad[i] = LLONG_MAX;
        }
    } else {
        st->err[cls] = 0;
        st->first_bad[cls] = LLONG_MAX;
    }
}

cudaError_t reset_class(rime_ctx *c, int cls) {
    k_reset_status<<<1, 1, 0, c->stream>>>(c->d_status, cls);
    return cudaGetLastError();
}

}  // namespace

cudaError_t rime::reset_status_class(rime_ctx *c, int cls) { return reset_class(c, cls); }

// Marks the end of the context's latest host-to-device upload on its stream:
// the streamed chi^2 starts its chunk copies after it, so that they neither
// queue ahead of an upload that the chunk kernels need nor wait for the
// kernels queued after it.
cudaError_t rime::mark_upload(rime_ctx *c) {
    if (!c->ev_upload) {
        cudaError_t e = cudaEventCreateWithFlags(&c->ev_upload, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaEventRecord(c->ev_upload, c->stream);
    if (e == cudaSuccess) c->upload_marked = true;
    return e;
}

namespace {

const char *class_name(int cls) {
    switch (cls) {
        case EC_FREQ: return "freq_hz";
        case EC_UVW: return "uvw/pointing";
        case EC_DATA: return "data/weight";
        case EC_GAINS: return "gains";
        case EC_SRC: return "sources";
        case EC_MODE: return "sources (tensor-core mode)";
        case EC_SDATA: return "streamed data/weight";
        default: return "kernel";
    }
}

// Waits for the stream and turns the device status block into a status.
rime_status sync_status(rime_ctx *c) {
    CK(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream),
       "reading the status block");
    CK(c, cudaStreamSynchronize(c->stream), "stream synchronize");
    for (int cls = 0; cls < EC_N; cls++) {
        int e = c->h_status->err[cls];
        if (!e) continue;
        char buf[256];
        long long idx = c->h_status->first_bad[cls];
        if (cls == EC_RUN) {
            CK(c, reset_class(c, EC_RUN), "reset status");
            return fail(c, RIME_E_TIMEOUT, "a kernel gave up a bounded wait (pipeline stalled)");
        }
        if (cls == EC_MODE) {
            if (e & EB_F16)
                std::snprintf(buf, sizeof buf,
                              "the FP16 split mode takes scaled Stokes values of magnitude up to 6e4 "
                              "(first source beyond: %lld); use RIME_TC_SPLIT_BF16, RIME_TC_SPLIT_TF32 or RIME_TC_OFF",
                              idx);
            else
                std::snprintf(buf, sizeof buf,
                              "the split-precision tensor-core mode takes point sources only "
                              "(first Gaussian source: %lld); use RIME_TC_OFF", idx);
            return fail(c, RIME_E_INVALID, buf);
        }
        if (e & EB_NONFINITE) {
            std::snprintf(buf, sizeof buf, "%s: NaN or Inf (first at element %lld)", class_name(cls), idx);
            return fail(c, RIME_E_NONFINITE, buf);
        }
        const char *why = cls == EC_SRC ? "l^2+m^2 >= 1, or not major >= minor >= 0"
                          : (cls == EC_DATA || cls == EC_SDATA) ? "negative weight"
                          : cls == EC_FREQ ? "frequency <= 0" : "value out of range";
        std::snprintf(buf, sizeof buf, "%s: %s (first at element %lld)", class_name(cls), why, idx);
        return fail(c, RIME_E_INVALID, buf);
    }
    return RIME_OK;
}

}  // namespace

rime_status rime::sync_status_ctx(rime_ctx *c) { return sync_status(c); }

namespace {

size_t vis_count(const rime_ctx *c) { return (size_t)c->dims.ntime * c->nbl * c->dims.nchan; }

rime_status upload_data(rime_ctx *c, const void *data, const void *weight) {
    Alloc alloc{c};
    size_t nvis = vis_count(c);
    size_t ts = c->tsize();
    if (data) {
        if (!c->d_data) CK(c, alloc(&c->d_data, nvis * 8 * ts), "allocating data");
        CK(c, cudaMemcpyAsync(c->d_data, data, nvis * 8 * ts, cudaMemcpyDefault, c->stream), "copying data");
        c->has_data = true;
    }
    if (weight) {
        if (!c->d_weight) CK(c, alloc(&c->d_weight, nvis * ts), "allocating weights");
        CK(c, cudaMemcpyAsync(c->d_weight, weight, nvis * ts, cudaMemcpyDefault, c->stream),
           "copying weights");
    }
    c->has_weight = weight != nullptr;
    CK(c, mark_upload(c), "event");
    CK(c, reset_class(c, EC_DATA), "reset status");
    CK(c, launch_validate_data(c), "validating data");
    return RIME_OK;
}

rime_status upload_uvw(rime_ctx *c, const double *uvw, const double *pointing) {
    Alloc alloc{c};
    size_t nta = (size_t)c->dims.ntime * c->dims.na;
    CK(c, cudaMemcpyAsync(c->d_uvw, uvw, nta * 3 * sizeof(double), cudaMemcpyDefault, c->stream),
       "copying uvw");
    if (pointing) {
        if (!c->d_pointing) CK(c, alloc((void **)&c->d_pointing, nta * 2 * sizeof(double)), "allocating pointing");
        CK(c, cudaMemcpyAsync(c->d_pointing, pointing, nta * 2 * sizeof(double), cudaMemcpyDefault, c->stream),
           "copying pointing");
    }
    c->has_pointing = pointing != nullptr;
    CK(c, mark_upload(c), "event");
    CK(c, reset_class(c, EC_UVW), "reset status");
    CK(c, launch_validate_uvw(c), "validating uvw");
    CK(c, launch_prep_delays(c), "delays");
    return RIME_OK;
}

}  // namespace

namespace rime {
void set_global_error(const char *msg) { g_create_error = msg; }
}  // namespace rime

extern "C" {

int64_t rime_nbl(int32_t na) { return na < 2 ? 0 : (int64_t)na * (na - 1) / 2; }

const char *rime_status_string(rime_status s) {
    switch (s) {
        case RIME_OK: return "RIME_OK";
        case RIME_E_INVALID: return "RIME_E_INVALID";
        case RIME_E_STATE: return "RIME_E_STATE";
        case RIME_E_OOM: return "RIME_E_OOM";
        case RIME_E_CUDA: return "RIME_E_CUDA";
        case RIME_E_TIMEOUT: return "RIME_E_TIMEOUT";
        case RIME_E_NONFINITE: return "RIME_E_NONFINITE";
    }
    return "RIME_E_UNKNOWN";
}

const char *rime_last_error(const rime_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

rime_status rime_create(rime_ctx **out, const rime_dims *dims, const double *freq_hz,
                        const double *uvw, const double *pointing, const void *data,
                        const void *weight, void *cuda_stream) {
    g_create_error.clear();
    if (!out) return fail(nullptr, RIME_E_INVALID, "ctx output pointer is NULL");
    *out = nullptr;
    if (!dims) return fail(nullptr, RIME_E_INVALID, "dims is NULL");
    if (dims->na < 2 || dims->na > kMaxNa)
        return fail(nullptr, RIME_E_INVALID, "na must be in [2, 4096]");
    if (dims->ntime < 1 || dims->nchan < 1)
        return fail(nullptr, RIME_E_INVALID, "ntime and nchan must be >= 1");
    if (dims->precision != RIME_FP32 && dims->precision != RIME_FP64)
        return fail(nullptr, RIME_E_INVALID, "precision must be RIME_FP32 or RIME_FP64");
    if (!(dims->ref_freq_hz > 0.0) || !std::isfinite(dims->ref_freq_hz))
        return fail(nullptr, RIME_E_INVALID, "ref_freq_hz must be finite and > 0");
    if (!(dims->beam_c >= 0.0) || !std::isfinite(dims->beam_c))
        return fail(nullptr, RIME_E_INVALID, "beam_c must be finite and >= 0");
    if (!freq_hz) return fail(nullptr, RIME_E_INVALID, "freq_hz is NULL");
    if (!uvw) return fail(nullptr, RIME_E_INVALID, "uvw is NULL");
    std::vector<Unit> units;
    std::vector<Tile> tiles;
    build_units(dims->na, dims->precision, units, tiles);
    long long blocks = (long long)dims->ntime * dims->nchan * (long long)units.size();
    if (blocks > kMaxBlocks) return fail(nullptr, RIME_E_INVALID, "ntime * nchan * antenna units exceeds 2^31-1");

    rime_ctx *c = new rime_ctx();
    c->dims = *dims;
    c->nbl = rime_nbl(dims->na);
    c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    c->nunits = (int)units.size();
    auto bail = [&](rime_status s) {
        g_create_error = c->err;
        free_all(c);
        delete c;
        return s;
    };
#define CKC(call, what)                                            \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return bail(cuda_fail(c, e_, what)); \
    } while (0)
    CKC(cudaGetDevice(&c->device), "cudaGetDevice");
    Alloc alloc{c};
    size_t nchan = dims->nchan, nta = (size_t)dims->ntime * dims->na;
    CKC(alloc((void **)&c->d_freq, nchan * sizeof(double)), "allocating freq");
    CKC(alloc(&c->d_chan, nchan * std::max(sizeof(ChanF), sizeof(ChanD))), "allocating channels");
    CKC(alloc((void **)&c->d_uvw, nta * 3 * sizeof(double)), "allocating uvw");
    if (dims->precision == RIME_FP32) CKC(alloc(&c->d_uvw_f, nta * sizeof(float4)), "allocating uvw");
    CKC(alloc((void **)&c->d_status, sizeof(DevStatus)), "allocating status");
    CKC(cudaMallocHost((void **)&c->h_status, sizeof(DevStatus)), "allocating pinned status");
    CKC(alloc((void **)&c->d_counter, sizeof(unsigned int)), "allocating counter");
    c->partials_cap = (size_t)blocks;
    CKC(alloc((void **)&c->d_partials, c->partials_cap * sizeof(double)), "allocating partials");
    CKC(alloc((void **)&c->d_units, units.size() * sizeof(Unit)), "allocating units");
    CKC(alloc((void **)&c->d_tiles, tiles.size() * sizeof(Tile)), "allocating tiles");
    CKC(cudaMemcpyAsync(c->d_units, units.data(), units.size() * sizeof(Unit), cudaMemcpyHostToDevice, c->stream),
        "copying units");
    CKC(cudaMemcpyAsync(c->d_tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice, c->stream),
        "copying tiles");
    CKC(cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned int), c->stream), "clearing counter");
    CKC(reset_class(c, -1), "reset status");
    CKC(cudaMemcpyAsync(c->d_freq, freq_hz, nchan * sizeof(double), cudaMemcpyDefault, c->stream), "copying freq");
    CKC(launch_prep_channels(c), "channel constants");
    rime_status s = upload_uvw(c, uvw, pointing);
    if (s != RIME_OK) return bail(s);
    if (data || weight) {
        s = upload_data(c, data, weight);
        if (s != RIME_OK) return bail(s);
    }
    s = sync_status(c);
    if (s != RIME_OK) return bail(s);
#undef CKC
    *out = c;
    return RIME_OK;
}

rime_status rime_set_uvw(rime_ctx *c, const double *uvw, const double *pointing) {
    if (!c) return fail(nullptr, RIME_E_INVALID, "ctx is NULL");
    if (!uvw) return fail(c, RIME_E_INVALID, "uvw is NULL");
    return upload_uvw(c, uvw, pointing);
}

rime_status rime_set_data(rime_ctx *c, const void *data, const void *weight) {
    if (!c) return fail(nullptr, RIME_E_INVALID, "ctx is NULL");
    if (!data) return fail(c, RIME_E_INVALID, "data is NULL");
    return upload_data(c, data, weight);
}

rime_status rime_set_gains(rime_ctx *c, const double *gains) {
    if (!c) return fail(nullptr, RIME_E_INVALID, "ctx is NULL");
    if (!gains) {
        c->has_gains = false;
        CK(c, reset_class(c, EC_GAINS), "reset status");
        return RIME_OK;
    }
    Alloc alloc{c};
    size_t n = (size_t)c->dims.ntime * c->dims.na * c->dims.nchan * 8;
    if (!c->d_gains_in) CK(c, alloc((void **)&c->d_gains_in, n * sizeof(double)), "allocating gains");
    if (!c->d_gains) CK(c, alloc(&c->d_gains, n * c->tsize()), "allocating gains");
    CK(c, cudaMemcpyAsync(c->d_gains_in, gains, n * sizeof(double), cudaMemcpyDefault, c->stream),
       "copying gains");
    CK(c, mark_upload(c), "event");
    CK(c, reset_class(c, EC_GAINS), "reset status");
    CK(c, launch_convert_gains(c), "converting gains");
    c->has_gains = true;
    return RIME_OK;
}

rime_status rime_set_sources(rime_ctx *c, const rime_sources *src) {
    if (!c) return fail(nullptr, RIME_E_INVALID, "ctx is NULL");
    if (!src) return fail(c, RIME_E_INVALID, "sources is NULL");
    if (src->nsrc < 0) return fail(c, RIME_E_INVALID, "nsrc must be >= 0");
    if (src->time_varying != 0 && src->time_varying != 1)
        return fail(c, RIME_E_INVALID, "time_varying must be 0 or 1");
    if (src->nsrc > 0 && (!src->lm || !src->stokes || !src->alpha))
        return fail(c, RIME_E_INVALID, "lm, stokes and alpha must not be NULL when nsrc > 0");
    size_t n = (size_t)src->nsrc;
    size_t rows = src->time_varying ? (size_t)c->dims.ntime : 1;
    size_t nd = (size_t)c->dims.ntime * n * c->dims.na;
    if (nd > (size_t)LLONG_MAX / 16) return fail(c, RIME_E_INVALID, "nsrc too large");
    if (n > c->src_cap || rows != c->src_stokes_rows) {
        void *old[] = {c->d_src_in, c->d_stokes, c->d_gauss, c->d_alpha, c->d_src_extra, c->d_tau, c->d_rho,
                       c->d_gpart};
        for (void *p : old)
            if (p) cudaFree(p);
        c->d_src_in = nullptr;
        c->d_stokes = c->d_gauss = c->d_alpha = c->d_src_extra = c->d_tau = c->d_rho = nullptr;
        c->d_gpart = nullptr;
        c->gpart_cap = 0;
        c->src_cap = 0;
        c->sources_set = false;
        size_t cap = std::max<size_t>(n, 1);
        size_t ts = c->tsize();
        size_t ndc = (size_t)c->dims.ntime * cap * c->dims.na;
        Alloc alloc{c};
        CK(c, alloc((void **)&c->d_src_in, rime_ctx::src_in_doubles(rows, cap) * sizeof(double)), "allocating sources");
        CK(c, alloc(&c->d_stokes, rows * cap * 4 * ts), "allocating sources");
        CK(c, alloc(&c->d_gauss, cap * 4 * ts), "allocating sources");
        CK(c, alloc(&c->d_alpha, cap * ts), "allocating sources");
        CK(c, alloc(&c->d_src_extra, cap * 8 * ts), "allocating sources");
        CK(c, alloc(&c->d_tau, ndc * 8), "allocating delays");
        CK(c, alloc(&c->d_rho, ndc * ts), "allocating delays");
        c->src_cap = cap;
        c->src_stokes_rows = rows;
    }
    c->nsrc = src->nsrc;
    c->time_varying = src->time_varying;
    c->has_shape = src->shape != nullptr;
    c->has_kind = src->shape != nullptr && src->kind != nullptr;
    if (n > 0) {
        CK(c, cudaMemcpyAsync(c->src_lm(), src->lm, n * 2 * sizeof(double), cudaMemcpyDefault, c->stream),
           "copying lm");
        CK(c, cudaMemcpyAsync(c->src_stokes(), src->stokes, rows * n * 4 * sizeof(double), cudaMemcpyDefault,
                              c->stream), "copying stokes");
        CK(c, cudaMemcpyAsync(c->src_alpha(), src->alpha, n * sizeof(double), cudaMemcpyDefault, c->stream),
           "copying alpha");
        if (src->shape)
            CK(c, cudaMemcpyAsync(c->src_shape(), src->shape, n * 3 * sizeof(double), cudaMemcpyDefault,
                                  c->stream), "copying shape");
        if (c->has_kind)
            CK(c, cudaMemcpyAsync(c->src_kind(), src->kind, n * sizeof(int32_t), cudaMemcpyDefault, c->stream),
               "copying kind");
    }
    if (n > 0) CK(c, mark_upload(c), "event");
    CK(c, reset_class(c, EC_SRC), "reset status");
    CK(c, reset_class(c, EC_MODE), "reset status");
    c->sources_set = true;
    CK(c, launch_prep_sources(c), "source factors");
    return RIME_OK;
}

rime_status rime_predict(rime_ctx *c, void *vis_out) {
    if (!c) return fail(nullptr, RIME_E_INVALID, "ctx is NULL");
    if (!vis_out) return fail(c, RIME_E_INVALID, "vis_out is NULL");
    if (!c->sources_set) return fail(c, RIME_E_STATE, "rime_set_sources has not been called");
    if (c->tc_mode != RIME_TC_OFF) CK(c, launch_split(c, true, vis_out, nullptr), "tensor-core predict kernel");
    else CK(c, launch_fused_auto(c, vis_out, nullptr, false), "predict kernel");
    return RIME_OK;
}

rime_status rime_chi2_async(rime_ctx *c, double *chi2_dev) {
    if (!c) return fail(nullptr, RIME_E_INVALID, "ctx is NULL");
    if (!chi2_dev) return fail(c, RIME_E_INVALID, "chi2_dev is NULL");
    if (!c->sources_set) return fail(c, RIME_E_STATE, "rime_set_sources has not been called");
    if (!c->has_data) return fail(c, RIME_E_STATE, "no observed data (rime_set_data)");
    if (c->tc_mode != RIME_TC_OFF) CK(c, launch_split(c, false, nullptr, chi2_dev), "tensor-core chi2 kernel");
    else CK(c, launch_fused_auto(c, nullptr, chi2_dev, true), "chi2 kernel");
    return RIME_OK;
}

rime_status rime_set_tensor_mode(rime_ctx *c, int32_t mode) {
    if (!c) return fail(nullptr, RIME_E_INVALID, "ctx is NULL");
    if (mode != RIME_TC_OFF && mode != RIME_TC_SPLIT_BF16 && mode != RIME_TC_SPLIT_TF32 && mode != RIME_TC_SPLIT_F16)
        return fail(c, RIME_E_INVALID,
                    "mode must be RIME_TC_OFF, RIME_TC_SPLIT_BF16, RIME_TC_SPLIT_TF32 or RIME_TC_SPLIT_F16");
    if (mode != RIME_TC_OFF && c->dims.precision != RIME_FP32)
        return fail(c, RIME_E_INVALID, "the tensor-core modes need an RIME_FP32 context");
    c->tc_mode = mode;
    CK(c, reset_class(c, EC_MODE), "reset status");
    return RIME_OK;
}

rime_status rime_set_beam(rime_ctx *c, int32_t model, double beam_c) {
    if (!c) return fail(nullptr, RIME_E_INVALID, "ctx is NULL");
    if (model != RIME_BEAM_COS3 && model != RIME_BEAM_JINC)
        return fail(c, RIME_E_INVALID, "model must be RIME_BEAM_COS3 or RIME_BEAM_JINC");
    if (!(beam_c >= 0.0) || !std::isfinite(beam_c)) return fail(c, RIME_E_INVALID, "beam_c must be finite and >= 0");
    c->beam_model = model;
    c->dims.beam_c = beam_c;
    CK(c, launch_prep_channels(c), "channel constants");
    return RIME_OK;
}

rime_status rime_set_wait_limit(rime_ctx *c, uint64_t ns) {
    if (!c) return RIME_E_INVALID;
    c->wait_ns = (unsigned long long)ns;
    return RIME_OK;
}

rime_status rime_set_kernel(rime_ctx *c, int32_t kernel) {
    if (!c) return fail(nullptr, RIME_E_INVALID, "ctx is NULL");
    if (kernel != RIME_KERNEL_AUTO && kernel != RIME_KERNEL_TILED && kernel != RIME_KERNEL_NARROW)
        return fail(c, RIME_E_INVALID, "kernel must be RIME_KERNEL_AUTO, RIME_KERNEL_TILED or RIME_KERNEL_NARROW");
    if (kernel == RIME_KERNEL_NARROW && c->dims.na > NARROW_MAX_NA)
        return fail(c, RIME_E_INVALID, "RIME_KERNEL_NARROW takes arrays of at most 45 antennas");
    c->kernel = kernel;
    return RIME_OK;
}

rime_status rime_chi2(rime_ctx *c, double *chi2) {
    if (!c) return fail(nullptr, RIME_E_INVALID, "ctx is NULL");
    if (!chi2) return fail(c, RIME_E_INVALID, "chi2 is NULL");
    rime_status s = rime_chi2_async(c, &c->d_status->chi2);
    if (s != RIME_OK) return s;
    s = sync_status(c);
    if (s != RIME_OK) return s;
    *chi2 = c->h_status->chi2;
    return RIME_OK;
}

rime_status rime_chi2_grad(rime_ctx *c, double *chi2, double *grad_src, void *grad_gains) {
    if (!c) return fail(nullptr, RIME_E_INVALID, "ctx is NULL");
    if (!chi2) return fail(c, RIME_E_INVALID, "chi2 is NULL");
    if (!c->sources_set) return fail(c, RIME_E_STATE, "rime_set_sources has not been called");
    if (!c->has_data) return fail(c, RIME_E_STATE, "no observed data (rime_set_data)");
    if (c->time_varying)
        return fail(c, RIME_E_INVALID, "the gradient needs static brightness (time_varying = 0)");
    if (c->nsrc > 0 && !grad_src) return fail(c, RIME_E_INVALID, "grad_src is NULL");
    Alloc alloc{c};
    if (!c->d_yadj) CK(c, alloc(&c->d_yadj, vis_count(c) * 4 * 2 * c->tsize()), "allocating the adjoint buffer");
    double *gg = static_cast<double *>(grad_gains);
    // the gains gradient: the forward kernel stores each visibility's two
    // terms, a second kernel sums them per antenna in a fixed order
    if (gg && !c->d_dgain)
        CK(c, alloc(&c->d_dgain, vis_count(c) * 16 * c->tsize()), "allocating the gains-gradient terms");
    void *dg = gg ? c->d_dgain : nullptr;
    if (narrow_applies(c))
        CK(c, launch_narrow(c, MODE_GRAD, nullptr, &c->d_status->chi2, 0, c->nsrc, c->d_yadj, dg),
           "gradient forward kernel");
    else
        CK(c, launch_fused_mode(c, MODE_GRAD, nullptr, &c->d_status->chi2, c->d_yadj, dg), "gradient forward kernel");
    if (gg) CK(c, launch_gains_grad(c, gg), "gains gradient kernel");
    CK(c, launch_grad_src(c, grad_src), "source gradient kernels");
    rime_status s = sync_status(c);
    if (s != RIME_OK) return s;
    *chi2 = c->h_status->chi2;
    return RIME_OK;
}

rime_status rime_ln_norm(rime_ctx *c, double *ln_norm) {
    if (!c) return fail(nullptr, RIME_E_INVALID, "ctx is NULL");
    if (!ln_norm) return fail(c, RIME_E_INVALID, "ln_norm is NULL");
    CK(c, launch_ln_norm(c), "ln-norm kernel");
    rime_status s = sync_status(c);
    if (s != RIME_OK) return s;
    *ln_norm = c->h_status->aux;
    return RIME_OK;
}

rime_status rime_sync(rime_ctx *c) {
    if (!c) return fail(nullptr, RIME_E_INVALID, "ctx is NULL");
    return sync_status(c);
}

void rime_destroy(rime_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

}  // extern "C"
