// rime_noalloc.cu -- rime_chi2_noalloc: the fused chi^2 without any device
// memory allocation, for callers that cannot call cudaMalloc.
//
// Every intermediate the fused chi^2 needs (channel constants, converted
// gains, per-source constants, per-(t, s, a) delays, the work-unit table,
// the per-block partial sums, the completion counter and the status block)
// is carved out of one file-scope device array of fixed size. Host code only
// ever passes the array's device address, obtained once per device with
// cudaGetSymbolAddress; the kernels are the same ones the context-based
// entry points launch.
#include "rime_internal.cuh"

#include <climits>
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <mutex>

using namespace rime;

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;   // 32 MiB
constexpr int kMaxNaNoAlloc = 256;                    // bounds the unit table below
// at 256 antennas: 16 units (FP32) or 36 (FP64), at most 256 thread tiles each
constexpr int kMaxUnits = 40;
constexpr int kMaxTiles = kMaxUnits * 256;

// The scratch shared by every call in this process on a given device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 256;
void *g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

// Device address of g_scratch on the current device (looked up once per device).
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

__global__ void k_noalloc_reset(DevStatus *st, unsigned int *counter) {
    st->chi2 = 0.0;
    st->aux = 0.0;
    for (int i = 0; i < EC_N; i++) {
        st->err[i] = 0;
        st->first_bad[i] = LLONG_MAX;
    }
    *counter = 0u;
}

// Bump layout over the scratch array, 256-byte aligned regions.
struct Layout {
    size_t off = 0;
    size_t take(size_t bytes) {
        size_t at = off;
        off += (bytes + 255) & ~size_t(255);
        return at;
    }
};

rime_status fail(rime_status s, const char *msg) {
    set_global_error(msg);
    return s;
}

const char *class_name(int cls) {
    switch (cls) {
        case EC_FREQ: return "freq_hz";
        case EC_UVW: return "uvw/pointing";
        case EC_DATA: return "data/weight";
        case EC_GAINS: return "gains";
        case EC_SRC: return "sources";
        default: return "kernel";
    }
}

}  // namespace

extern "C" rime_status rime_chi2_noalloc(const rime_dims *dims, const double *freq_hz, const double *uvw,
                                         const double *pointing, const void *data, const void *weight,
                                         const double *gains, const rime_sources *src, double *chi2_dev,
                                         void *cuda_stream) {
    // ---- host-side checks, before any CUDA call ----
    if (!dims) return fail(RIME_E_INVALID, "dims is NULL");
    if (dims->na < 2 || dims->na > kMaxNaNoAlloc)
        return fail(RIME_E_INVALID, "rime_chi2_noalloc: na must be in [2, 256]");
    if (dims->ntime < 1 || dims->nchan < 1) return fail(RIME_E_INVALID, "ntime and nchan must be >= 1");
    if (dims->precision != RIME_FP32 && dims->precision != RIME_FP64)
        return fail(RIME_E_INVALID, "precision must be RIME_FP32 or RIME_FP64");
    if (!(dims->ref_freq_hz > 0.0) || !std::isfinite(dims->ref_freq_hz))
        return fail(RIME_E_INVALID, "ref_freq_hz must be finite and > 0");
    if (!(dims->beam_c >= 0.0) || !std::isfinite(dims->beam_c))
        return fail(RIME_E_INVALID, "beam_c must be finite and >= 0");
    if (!freq_hz || !uvw || !data || !src || !chi2_dev)
        return fail(RIME_E_INVALID, "freq_hz, uvw, data, src and chi2_dev must not be NULL");
    if (src->nsrc < 0 || (src->time_varying != 0 && src->time_varying != 1))
        return fail(RIME_E_INVALID, "nsrc must be >= 0 and time_varying 0 or 1");
    if (src->nsrc > 0 && (!src->lm || !src->stokes || !src->alpha))
        return fail(RIME_E_INVALID, "lm, stokes and alpha must not be NULL when nsrc > 0");

    // every argument array must be device memory of the current device (or
    // managed memory): the kernels read them as they are
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(RIME_E_CUDA, "rime_chi2_noalloc: no current device");
    const void *ptrs[] = {freq_hz, uvw, pointing, data, weight, gains, src->lm, src->stokes, src->alpha,
                          src->shape, src->kind, chi2_dev};
    const char *names[] = {"freq_hz", "uvw", "pointing", "data", "weight", "gains", "lm", "stokes", "alpha",
                           "shape", "kind", "chi2_dev"};
    for (int i = 0; i < 12; i++) {
        if (!ptrs[i]) continue;
        if (i >= 6 && i <= 10 && src->nsrc == 0) continue;   // source arrays are not read
        if (i == 10 && !src->shape) continue;                // kind is read only with a shape
        cudaPointerAttributes a;
        const bool known = cudaPointerGetAttributes(&a, ptrs[i]) == cudaSuccess;
        if (!known) cudaGetLastError();   // clear the error of an unregistered host pointer
        const bool ok = known && (a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == dev));
        if (!ok) {
            char buf[160];
            std::snprintf(buf, sizeof buf, "rime_chi2_noalloc: %s is not device memory of the current device", names[i]);
            return fail(RIME_E_INVALID, buf);
        }
    }

    Unit units[kMaxUnits];
    Tile tiles[kMaxTiles];   // 40 KB on the caller's stack
    int ntiles = 0;
    int nunits = build_units_fixed(dims->na, dims->precision, units, kMaxUnits, tiles, kMaxTiles, &ntiles);
    if (nunits <= 0) return fail(RIME_E_INVALID, "rime_chi2_noalloc: work-unit table does not fit");

    rime_ctx c;   // a view over the caller's arrays and the scratch; owns nothing
    c.view = true;
    c.device = dev;
    c.dims = *dims;
    c.nbl = rime_nbl(dims->na);
    c.stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    c.nunits = nunits;
    const size_t ts = c.tsize();
    const size_t nsrc = (size_t)src->nsrc, cap = nsrc > 0 ? nsrc : 1;
    const size_t rows = src->time_varying ? (size_t)dims->ntime : 1;
    const size_t nta = (size_t)dims->ntime * dims->na;
    const size_t blocks = (size_t)dims->ntime * dims->nchan * (size_t)nunits;

    Layout L;
    size_t o_status = L.take(sizeof(DevStatus));
    size_t o_counter = L.take(sizeof(unsigned int));
    size_t o_chan = L.take((size_t)dims->nchan * sizeof(ChanF) * 2);
    size_t o_uvwf = L.take(dims->precision == RIME_FP32 ? nta * sizeof(float4) : 0);
    size_t o_gains = L.take(gains ? nta * dims->nchan * 8 * ts : 0);
    size_t o_srcin = L.take(rime_ctx::src_in_doubles(rows, cap) * sizeof(double));
    size_t o_stokes = L.take(rows * cap * 4 * ts);
    size_t o_gauss = L.take(cap * 4 * ts);
    size_t o_alpha = L.take(cap * ts);
    size_t o_tau = L.take(nta * cap * 8);
    size_t o_rho = L.take(nta * cap * ts);
    size_t o_units = L.take((size_t)nunits * sizeof(Unit));
    size_t o_tiles = L.take((size_t)ntiles * sizeof(Tile));
    size_t o_part = L.take(blocks * sizeof(double));
    // long FP32 source lists: the running sums of the persistent kernel's
    // blocks, as many blocks as the rest of the array holds (at most two per SM)
    size_t o_seg = 0, nseg = 0;
    if (dims->precision == RIME_FP32 && (long long)nsrc > seg_source_threshold()) {
        int nsm = 0;
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 152;
        const size_t per = seg_scratch_per_block();
        const size_t room = L.off < kScratchBytes ? (kScratchBytes - L.off) / per : 0;
        nseg = std::min((size_t)2 * nsm, room);
        if (nseg == 0) nseg = 1;   // reported below as too large
        o_seg = L.take(nseg * per);
    }
    if (L.off > kScratchBytes) {
        char buf[200];
        std::snprintf(buf, sizeof buf,
                      "rime_chi2_noalloc: this problem needs %zu bytes of scratch; the fixed scratch "
                      "holds %zu bytes (use the context API for larger problems)",
                      L.off, kScratchBytes);
        return fail(RIME_E_INVALID, buf);
    }

    void *base_v = nullptr;
    cudaError_t e = scratch_address(&base_v);
    if (e != cudaSuccess) return fail(RIME_E_CUDA, cudaGetErrorString(e));
    unsigned char *base = static_cast<unsigned char *>(base_v);

    c.d_status = reinterpret_cast<DevStatus *>(base + o_status);
    c.d_counter = reinterpret_cast<unsigned int *>(base + o_counter);
    c.d_chan = base + o_chan;
    c.d_uvw_f = dims->precision == RIME_FP32 ? base + o_uvwf : nullptr;
    c.d_freq = const_cast<double *>(freq_hz);
    c.d_uvw = const_cast<double *>(uvw);
    c.d_pointing = const_cast<double *>(pointing);
    c.has_pointing = pointing != nullptr;
    c.d_data = const_cast<void *>(data);
    c.has_data = true;
    c.d_weight = const_cast<void *>(weight);
    c.has_weight = weight != nullptr;
    c.d_gains_in = const_cast<double *>(gains);
    c.d_gains = gains ? base + o_gains : nullptr;
    c.has_gains = gains != nullptr;
    c.src_cap = cap;
    c.src_stokes_rows = rows;
    c.d_src_in = reinterpret_cast<double *>(base + o_srcin);
    c.d_stokes = base + o_stokes;
    c.d_gauss = base + o_gauss;
    c.d_alpha = base + o_alpha;
    c.d_tau = base + o_tau;
    c.d_rho = base + o_rho;
    c.d_units = reinterpret_cast<Unit *>(base + o_units);
    c.d_tiles = reinterpret_cast<Tile *>(base + o_tiles);
    c.d_partials = reinterpret_cast<double *>(base + o_part);
    c.partials_cap = blocks;
    if (nseg) {
        c.d_segsum = reinterpret_cast<float *>(base + o_seg);
        c.segsum_blocks = nseg;
    }
    c.nsrc = (int)nsrc;
    c.time_varying = src->time_varying;
    c.has_shape = src->shape != nullptr;
    c.has_kind = src->shape != nullptr && src->kind != nullptr;
    c.sources_set = true;

#define CKN(call)                                                     \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return fail(RIME_E_CUDA, cudaGetErrorString(e_)); \
    } while (0)
    k_noalloc_reset<<<1, 1, 0, c.stream>>>(c.d_status, c.d_counter);
    CKN(cudaGetLastError());
    CKN(cudaMemcpyAsync(c.d_units, units, (size_t)nunits * sizeof(Unit), cudaMemcpyHostToDevice, c.stream));
    CKN(cudaMemcpyAsync(c.d_tiles, tiles, (size_t)ntiles * sizeof(Tile), cudaMemcpyHostToDevice, c.stream));
    if (nsrc > 0) {
        CKN(cudaMemcpyAsync(c.src_lm(), src->lm, nsrc * 2 * sizeof(double), cudaMemcpyDefault, c.stream));
        CKN(cudaMemcpyAsync(c.src_stokes(), src->stokes, rows * nsrc * 4 * sizeof(double), cudaMemcpyDefault,
                            c.stream));
        CKN(cudaMemcpyAsync(c.src_alpha(), src->alpha, nsrc * sizeof(double), cudaMemcpyDefault, c.stream));
        if (src->shape)
            CKN(cudaMemcpyAsync(c.src_shape(), src->shape, nsrc * 3 * sizeof(double), cudaMemcpyDefault,
                                c.stream));
        if (c.has_kind)
            CKN(cudaMemcpyAsync(c.src_kind(), src->kind, nsrc * sizeof(int32_t), cudaMemcpyDefault, c.stream));
    }
    CKN(launch_prep_channels(&c));
    CKN(launch_validate_uvw(&c));
    CKN(launch_validate_data(&c));
    if (gains) CKN(launch_convert_gains(&c));
    CKN(launch_prep_sources(&c));
    CKN(launch_fused_auto(&c, nullptr, chi2_dev, true));

    // Wait and report the input checks; the status lives in the scratch too.
    DevStatus st;
    CKN(cudaMemcpyAsync(&st, c.d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, c.stream));
    CKN(cudaStreamSynchronize(c.stream));
#undef CKN
    for (int cls = 0; cls < EC_N; cls++) {
        if (!st.err[cls]) continue;
        char buf[200];
        bool nonfinite = st.err[cls] & EB_NONFINITE;
        std::snprintf(buf, sizeof buf, "%s: %s (first at element %lld)", class_name(cls),
                      nonfinite ? "NaN or Inf" : "value out of range", st.first_bad[cls]);
        return fail(nonfinite ? RIME_E_NONFINITE : RIME_E_INVALID, buf);
    }
    return RIME_OK;
}
