// rime_internal.cuh -- types shared by the librime translation units.
//
// Data kept on the device by a context (all sizes from rime_dims):
//   observation   uvw [ntime][na][3] f64, pointing [ntime][na][2] f64,
//                 data [ntime][nbl][nchan][4] complex, weight [ntime][nbl][nchan]
//   gains         [ntime][na][nchan][4] complex in the compute precision
//   channels      per-channel constants of eqs. 2-4 (ChanF / ChanD)
//   sources       stokes [ntime|1][nsrc] x4, Gaussian quadratic form [nsrc] x4,
//                 spectral index [nsrc]
//   delays        per (t, s, a): the geometric delay tau = (u l + v m + w (n-1)) / c
//                 (double-float pair in FP32 mode, double in FP64 mode) and the
//                 beam radius rho = |l_s - dl_ta|; [ntime][nsrc][na]
//   scratch       one FP64 partial chi^2 per thread block, a completion
//                 counter and a small status block
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rime.h"

namespace rime {

constexpr double kCLight = 299792458.0;
constexpr double kInvCLight = 1.0 / kCLight;
constexpr double kPi = 3.141592653589793;
constexpr double kLn2 = 0.6931471805599453;
// pi^2 / (4 ln 2): the FWHM Gaussian's Fourier-transform constant
constexpr double kGaussK = kPi * kPi / (4.0 * kLn2);
constexpr double kLog2e = 1.4426950408889634;

// Error classes: one status word per input class, cleared when that input
// is set again.
// EC_RUN: a kernel gave up a bounded wait (reported once, then cleared);
// EC_MODE: the sources do not suit the tensor-core mode (Gaussian sources).
enum ErrClass {
    EC_FREQ = 0, EC_UVW = 1, EC_DATA = 2, EC_GAINS = 3, EC_SRC = 4, EC_RUN = 5, EC_MODE = 6,
    EC_SDATA = 7,   // data / weights of a streamed chi^2 (checked per chunk, cleared per call)
    EC_N = 8
};
enum ErrBits : int {
    EB_NONFINITE = 1,
    EB_RANGE = 2,       // value outside its domain (l^2+m^2 >= 1, w < 0, nu <= 0, axes)
    EB_TIMEOUT = 4,     // a bounded wait inside a kernel gave up
    EB_F16 = 8,         // EC_MODE: a scaled Stokes value beyond the FP16 split mode's range
};

// Status block in device memory, copied to the host in one transfer.
struct DevStatus {
    double chi2;              // result of the fused reduction
    double aux;               // second scalar (ln-norm)
    int err[EC_N];            // ErrBits per class
    long long first_bad[EC_N];
};

// A unit of work for one thread block: antenna rows [r0, r0+nr) against
// columns [c0, c0+nc) (diag = 1: the same antennas, pairs p < q only). Its
// thread tiles are tiles[tile0 .. tile0+nbody) ("body" tiles, thread tid <
// nbody) followed by nhead "head" tiles that start at the first warp boundary
// after the body tiles (FP32 kernel only).
struct Unit {
    int32_t r0, c0, nr, nc;
    int32_t tile0, nbody, nhead, diag;
};
// A thread tile, antennas relative to the unit's r0 / c0.
//  FP32 body tile: row antenna p, column antennas q .. q+7.
//  FP32 head tile: pairs inside the 8-antenna block starting at p (= q):
//                  with x_i = p + ((fold + i) mod 8), the seven pairs
//                  (x_0, x_1..x_4) and (x_4, x_5..x_7); folds 0..3 cover the
//                  block's 28 pairs once (round-robin by cyclic distance).
//  FP64 tile:      row antennas p, p+1 against columns q, q+1.
struct Tile {
    uint8_t p, q, fold, pad;
};

// Per-channel constants, single precision path.
struct ChanF {
    float nu_hi, nu_lo;   // nu as a double-float pair (Hz)
    float hlr;            // 0.5 log2(nu / nu_ref): sqrt of the spectral factor is 2^(alpha hlr)
    float cnu;            // beam_c * nu[GHz]
    float nu2;            // nu^2 (Hz^2), for the Gaussian exponent
    int beam;             // rime_beam model of eq. 4's E (argument cnu * rho)
    float pad[2];
};
// Per-channel constants, double precision path.
struct ChanD {
    double nu, hlr, cnu, nu2;
    int beam, pad;        // rime_beam model of eq. 4's E (argument cnu * rho)
};

struct rime_ctx_impl;  // forward

// Kernel parameter block for the fused predict / chi^2 kernels.
struct FusedParams {
    int na, ntime, nchan, nsrc;
    long long nbl;
    int stokes_tstride;        // nsrc*4 if time varying, else 0 (elements)
    int nchp;                  // channel groups per timestep
    int nunits;
    int has_gains, has_weight, has_pointing;
    const Unit *units;
    const Tile *tiles;
    const void *chan;          // ChanF* or ChanD*
    const double *uvw;         // [ntime][na][3]
    const float4 *uvw_f;       // [ntime][na] (u, v, w, 0), FP32 path
    const void *stokes;        // float4* or double4-like (4 x T)
    const void *gauss;         // 4 x T per source: A, B, C (exponent form), flag
    const void *alpha;         // T per source
    const void *tau;           // float2 / double per (t, s, a)
    const void *rho;           // float / double per (t, s, a)
    const void *gains;         // complex T [ntime][na][nchan][4]
    const void *data;          // complex T [ntime][nbl][nchan][4]
    const void *weight;        // T [ntime][nbl][nchan]
    void *vis_out;             // complex T [ntime][nbl][nchan][4]
    double *partials;          // [gridDim] FP64 partial chi^2
    unsigned int *counter;     // completion counter (reset by the last block)
    double *result;            // where the last block stores chi^2
    const DevStatus *status;   // kernels skip their work if any err word is set
    // gradient mode only
    void *yout;                // complex T [ntime][nbl][nchan][4]: Stokes-projected adjoint Y_X
    void *dgain;               // T [2][ntime][nbl][nchan][8] or null: per visibility the terms of the
                               // gains gradient, d chi^2 / dG_p (plane 0) and d chi^2 / dG_q (plane 1),
                               // 4 complex each
    int src0, src1;            // the source range [src0, src1) of this launch (default: all)
    int t_begin;               // first timestep of the launch (the grid covers a time range)
    float *segsum;             // FP32 tile kernel, long source lists: per-block running sums
};

// Batched chi^2: the schedule of a persistent launch. Work item i is
// (t, channel group, unit) = i / ngroups and the group of sets i % ngroups.
struct BatchParams {
    long long nitems;          // (timesteps covered * nkc * nunits) * ngroups
    int nsets, gsets, ngroups; // sets; sets per item; ceil(nsets / gsets)
    int per_set;               // partials per set: ntime * nchan * nunits
    int nkc, cpi;              // channel groups, channels per group
    const int *order;          // set of each rank
    const int *offsets;        // [nsets + 1] source offsets
    unsigned long long *counter;   // next work item (zeroed before the launch)
    double *partials;          // [nsets][ntime][nchan][nunits]
    int max_set;               // sources of the largest set (host side: scratch for long lists)
};

// Kernel modes of the fused predict / chi^2 kernels.
enum FusedMode { MODE_PREDICT = 0, MODE_CHI2 = 1, MODE_GRAD = 2 };

// Checks on the status block that every kernel makes before working.
__device__ __forceinline__ bool inputs_bad(const DevStatus *st) {
    int e = 0;
#pragma unroll
    for (int i = 0; i < EC_RUN; i++) e |= st->err[i];
    return (e | st->err[EC_MODE] | st->err[EC_SDATA]) != 0;
}

}  // namespace rime

// The opaque context of the public ABI.
struct rime_ctx {
    rime_dims dims;
    long long nbl = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    std::string err;

    // observation
    double *d_freq = nullptr;
    void *d_chan = nullptr;
    double *d_uvw = nullptr;
    void *d_uvw_f = nullptr;          // float4 copy for the FP32 path
    double *d_pointing = nullptr;
    void *d_data = nullptr;
    void *d_weight = nullptr;
    bool has_data = false, has_weight = false, has_pointing = false;
    // gains
    double *d_gains_in = nullptr;     // complex128 staging
    void *d_gains = nullptr;          // compute precision
    bool has_gains = false;
    // sources
    int nsrc = 0, time_varying = 0;
    bool sources_set = false;
    size_t src_cap = 0;               // sources the buffers below can hold
    size_t src_stokes_rows = 0;       // 1 or ntime
    // copy of the FP64 parameters (lm, stokes, alpha, shape, kind), then the
    // per-source geometry the delays need (l, m, n - 1, |lm|)
    double *d_src_in = nullptr;
    static size_t src_in_doubles(size_t rows, size_t cap) { return (2 + 4 * rows + 1 + 3 + 1 + 4) * cap; }
    double *src_lm() const { return d_src_in; }
    double *src_stokes() const { return d_src_in + 2 * src_cap; }
    double *src_alpha() const { return d_src_in + 2 * src_cap + 4 * src_cap * src_stokes_rows; }
    double *src_shape() const { return src_alpha() + src_cap; }
    int32_t *src_kind() const { return reinterpret_cast<int32_t *>(src_shape() + 3 * src_cap); }
    double *src_geo() const { return src_shape() + 4 * src_cap; }
    bool has_kind = false;            // a kind array was given (disks may be present)
    bool has_shape = false;
    void *d_stokes = nullptr, *d_gauss = nullptr, *d_alpha = nullptr;
    void *d_src_extra = nullptr;      // per source: l, m, l/n, m/n, major, minor, sin pa, cos pa
    // gradient scratch (allocated by the first rime_chi2_grad)
    void *d_yadj = nullptr;           // Y_X per visibility
    void *d_dgain = nullptr;          // per visibility the two terms of the gains gradient (16 T)
    double *d_gpart = nullptr;        // per (t, k, unit) partial source gradients
    size_t gpart_cap = 0;
    rime::Unit *d_gunits = nullptr;   // gradient work units and their baseline lists
    uint16_t *d_gbl = nullptr;
    int ngunits = 0;
    void *d_tau = nullptr, *d_rho = nullptr;
    // work decomposition
    rime::Unit *d_units = nullptr;
    rime::Tile *d_tiles = nullptr;
    int nunits = 0;
    // scratch
    double *d_partials = nullptr;
    size_t partials_cap = 0;
    unsigned int *d_counter = nullptr;
    rime::DevStatus *d_status = nullptr;
    rime::DevStatus *h_status = nullptr;   // pinned
    // batched chi^2 (allocated by the first rime_chi2_batched)
    int *d_bsched = nullptr;          // [order by size (cap) | set order (cap) | offsets (cap + 1)]
    size_t bsched_cap = 0;            // sets
    double *d_bpart = nullptr;        // per (set, t, k, unit) partials
    size_t bpart_cap = 0;
    unsigned long long *d_bcounter = nullptr;
    rime_batch_config bcfg{};         // configuration of the last FP32 batched call
    bool bcfg_forced = false;
    struct BatchTune {
        int nsets, nsrc;
        rime_batch_config cfg;
    };
    std::vector<BatchTune> btuned;    // tuned configurations by (nsets, total sources)
    int bmax_bps = 0;                 // resident batched blocks per SM (0: not queried yet)
    int nsm = 0;
    unsigned long long wait_ns = 0;   // limit of the kernels' bounded waits (0: about two seconds)
    float *d_segsum = nullptr;        // FP32 tile kernel: running sums of long source lists, per block
    float *d_segsum2 = nullptr;       // the same for the streamed chi^2's second kernel stream
    size_t segsum_blocks = 0;         // blocks each holds
    bool view = false;                // a view over caller memory (rime_chi2_noalloc): allocates nothing
    // tensor-core split-precision mode (FP32 contexts)
    int tc_mode = 0;                  // rime_tc_mode
    int kernel = 0;                   // rime_kernel
    int beam_model = 0;               // rime_beam
    // chains (rime_chains.cu): per-chain residuals N_c = D - V_c
    int chains_n = 0, chains_move = 0;       // chains; sources moved per chain by the last proposal
    void *d_chainN = nullptr;                // [chains][ntime][nbl][nchan][4] complex
    void *d_chain_scratch = nullptr;         // one chain's visibilities
    double *d_pair = nullptr;                // staged proposal sky model (FP64 parameters)
    size_t pair_cap = 0;                     // sources it holds
    int32_t *d_pair_kind = nullptr;
    double *d_chain_part = nullptr;          // [chains][ntime][blocks]: proposal chi^2 partials
    // streamed chi^2 (rime_stream.cu): a copy stream, a ring of chunk buffers
    static constexpr int kStreamBufs = 8;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_start = nullptr, ev_copied[kStreamBufs] = {}, ev_free[kStreamBufs] = {};
    bool stream_used = false;                // ev_start marks the previous streamed call's end
    cudaEvent_t ev_entry = nullptr;          // the context's stream at a call with device inputs
    cudaEvent_t ev_upload = nullptr;         // the context's stream after its latest upload copy
    cudaStream_t kstream2 = nullptr;         // odd chunks' kernels (even ones: the context's stream)
    cudaEvent_t ev_k2 = nullptr;             // kstream2's last chunk kernel
    unsigned *d_stream_counters = nullptr;   // last-block counters of the two kernel streams
    bool upload_marked = false;
    void *d_sbuf[kStreamBufs] = {};          // chunk data, then chunk weights
    size_t sbuf_cap = 0;                     // bytes of each buffer
    int sbuf_n = 0;                          // buffers allocated
    int sbuf_asked = 0;                      // buffers asked for when they were (memory may allow fewer)
    double *d_schi = nullptr;                // chi^2 of each chunk
    size_t schi_cap = 0;
    int2 *d_stiles = nullptr;         // its tiles (p0, q0)
    int nstiles = 0;
    double *d_spart = nullptr;        // one partial chi^2 per block
    size_t spart_cap = 0;
    unsigned *d_scounter = nullptr;
    void *d_sscale = nullptr;         // per (t, k, source) Stokes scale factors
    size_t sscale_cap = 0;

    size_t tsize() const { return dims.precision == RIME_FP64 ? 8 : 4; }
};

namespace rime {
// launchers (rime_prep.cu)
cudaError_t launch_prep_channels(rime_ctx *c);
cudaError_t launch_validate_uvw(rime_ctx *c);
cudaError_t launch_validate_data(rime_ctx *c);
cudaError_t launch_convert_gains(rime_ctx *c);
cudaError_t launch_prep_sources(rime_ctx *c);
cudaError_t launch_prep_delays(rime_ctx *c);
cudaError_t launch_ln_norm(rime_ctx *c);
// checks nvis visibilities' data / weights (either may be NULL) and flags class
// cls with the index i0 + i of the first bad one
cudaError_t launch_validate_chunk(rime_ctx *c, long long nvis, const void *data, const void *weight, int cls,
                                  long long i0, cudaStream_t stream = nullptr);
// rime_grad.cu
cudaError_t launch_grad_src(rime_ctx *c, double *grad_src);
// the gains gradient from the per-visibility terms: a fixed-order sum per (t, antenna, channel)
cudaError_t launch_gains_grad(rime_ctx *c, double *grad_gains);
// launchers (rime_fused.cu)
cudaError_t launch_fused(rime_ctx *c, void *vis_out, double *result, bool chi2);
cudaError_t launch_fused_mode(rime_ctx *c, int mode, void *vis_out, double *result, void *yout,
                              void *dgain);
int fused_blocks(const rime_ctx *c);
int build_units_fixed(int na, int precision, Unit *units, int max_units, Tile *tiles, int max_tiles,
                      int *ntiles);
cudaError_t launch_batched_f32(rime_ctx *c, const BatchParams &B, int grid);
int batched_blocks_per_sm();
cudaError_t launch_set_sums(rime_ctx *c, int nsets, int per_set, const double *partials, double *chi2);
cudaError_t launch_fused_f64_range(rime_ctx *c, int src0, int src1, double *result);
// FP32 source lists longer than this run the persistent kernel with per-block
// running sums of this many bytes per block (rime_fused.cu)
long long seg_source_threshold();
cudaError_t ensure_segsum(rime_ctx *c);
// a second scratch of the same size, for launches that may run beside those
// using the first (the streamed chi^2's second kernel stream)
cudaError_t ensure_segsum2(rime_ctx *c);
size_t seg_scratch_per_block();
void fill_fused_params(const rime_ctx *c, FusedParams &P, void *vis_out, double *result, void *yout,
                       void *dgain);
// launches the tiled fused kernel of `mode` with prepared parameters over `blocks` blocks
// (stream: nullptr = the context's stream)
cudaError_t launch_tiled_params(rime_ctx *c, int mode, const FusedParams &P, long long blocks,
                                cudaStream_t stream = nullptr);
// rime_narrow.cu: the small-array kernel (one thread per baseline and channel)
constexpr int NARROW_MAX_NA = 45;      // it takes arrays of up to this many antennas (990 baselines)
constexpr int NARROW_AUTO_NA_F32 = 32; // RIME_KERNEL_AUTO picks it up to here in FP32 (FP64: 45)
bool narrow_applies(const rime_ctx *c);
cudaError_t launch_narrow(rime_ctx *c, int mode, void *vis_out, double *result, int src0, int src1,
                          void *yout = nullptr, void *dgain = nullptr);
// the same with prepared parameters over timesteps [P.t_begin, P.t_begin + nt)
cudaError_t launch_narrow_params(rime_ctx *c, int mode, const FusedParams &P, int nt,
                                 cudaStream_t stream = nullptr);
// blocks of one timestep of the small-array kernel (launches cover whole timesteps)
long long narrow_blocks_per_time(rime_ctx *c);
// predict (chi2 = false) or chi^2 over all sources with the kernel that suits the array
cudaError_t launch_fused_auto(rime_ctx *c, void *vis_out, double *result, bool chi2);
// rime_split.cu
cudaError_t launch_split(rime_ctx *c, bool write, void *vis_out, double *result);
// rime_api.cu: clears one error class of the status block (stream-ordered)
cudaError_t reset_status_class(rime_ctx *c, int cls);
cudaError_t mark_upload(rime_ctx *c);
// sets the message rime_last_error(NULL) returns (rime_api.cu)
void set_global_error(const char *msg);
// error reporting and the allocation cap shared by the entry points (rime_api.cu)
rime_status fail_ctx(rime_ctx *c, rime_status s, const std::string &msg);
rime_status cuda_fail_ctx(rime_ctx *c, cudaError_t e, const char *what);
// waits for the context's stream and turns the device status block into a status
rime_status sync_status_ctx(rime_ctx *c);
size_t alloc_cap();

// Device allocations of one context call; RIME_TEST_MAX_BYTES caps their sum,
// so that the out-of-memory path can be exercised.
struct Alloc {
    rime_ctx *c;
    size_t total = 0, cap = alloc_cap();
    cudaError_t operator()(void **p, size_t bytes) {
        if (bytes == 0) bytes = 16;
        if (total + bytes > cap) return cudaErrorMemoryAllocation;
        total += bytes;
        return cudaMalloc(p, bytes);
    }
};
}  // namespace rime
