/*
 * rime.h -- C ABI of librime: GPU RIME predict fused with a weighted chi^2
 * (Montblanc, arXiv 1501.07719), for NVIDIA GB300 (sm_103a).
 *
 * The library evaluates, for every timestep t, baseline (p, q) and channel k,
 *
 *   V_tpqk = G_tpk ( sum_s E_tpsk K_tpsk B_sk K_tqsk^H E_tqsk^H ) G_tqk^H   (eq. 1)
 *   B_sk   = (nu_k / nu_ref)^alpha_s [[I+Q, U+iV], [U-iV, I-Q]] * g_spqk    (eq. 2)
 *   K_tpsk = exp(2 pi i (u l + v m + w (n - 1)) nu_k / c)                  (eq. 3)
 *   E_tpsk = cos^3(C nu_k[GHz] |l_s - dl_tp|), zero past the first null      (eq. 4)
 *
 * with g the Gaussian shape factor (1 for point sources; the Fourier
 * transform of a unit-flux elliptical Gaussian of FWHM axes (major, minor) and
 * position angle pa from +m towards +l, at the baseline (u_p-u_q, v_p-v_q)/lambda)
 * and reduces it, in the same kernel, to
 *
 *   chi^2 = sum_{t,pq,k} w_tpqk sum_c |V_tpqk,c - D_tpqk,c|^2              (eq. 7)
 *
 * Conventions used by every entry point:
 *  - Baselines are the pairs p < q in row-major upper-triangle order:
 *    bl(p, q) = p*na - p*(p+1)/2 + (q - p - 1); nbl = na*(na-1)/2 (Sec. 2.2:
 *    autocorrelations are discarded).
 *  - Correlations: the 2x2 matrix in row-major order (00, 01, 10, 11).
 *  - Complex numbers are interleaved (re, im). "complex" below means complex64
 *    (2 x float) in RIME_FP32 mode and complex128 (2 x double) in RIME_FP64.
 *  - Array order is time slowest, channel (then correlation) fastest, as in
 *    Sec. 4.1: vis/data [ntime][nbl][nchan][4], weight [ntime][nbl][nchan].
 *  - Source parameters, uvw, frequencies, pointing and gains are always
 *    double precision, whatever the compute precision.
 *  - Input pointers may be host (pageable or pinned) or device pointers; the
 *    library copies what it needs into buffers it owns and the caller keeps
 *    ownership of its arrays. Output pointers are device pointers unless
 *    stated otherwise.
 *  - All work is ordered on the CUDA stream given to rime_create. Only the
 *    calls that return a host value (rime_create, rime_chi2, rime_chi2_grad,
 *    rime_sync) wait for the stream.
 *  - Every call returns a status and never aborts. On error the outputs are
 *    left untouched and rime_last_error() describes the cause.
 *  - Input values are checked on the GPU as they are uploaded (NaN/Inf,
 *    l^2+m^2 >= 1, major < minor or negative axes, negative weights,
 *    frequencies <= 0). A failed check makes every later kernel skip its
 *    work; the status is returned by the next call that waits for the stream
 *    (rime_chi2, rime_chi2_grad, rime_sync), until the offending input is set
 *    again with valid values.
 *  - A context is not thread safe; use one context per host thread.
 */
#ifndef RIME_H
#define RIME_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rime_ctx rime_ctx;

typedef enum {
    RIME_OK = 0,
    RIME_E_INVALID = 1,   /* bad argument: size, pointer or value out of range */
    RIME_E_STATE = 2,     /* call out of order (e.g. rime_chi2 before rime_set_sources) */
    RIME_E_OOM = 3,       /* a device allocation failed */
    RIME_E_CUDA = 4,      /* a CUDA runtime call or kernel launch failed */
    RIME_E_TIMEOUT = 5,   /* a bounded wait inside a kernel gave up */
    RIME_E_NONFINITE = 6  /* NaN or Inf in an input array */
} rime_status;

typedef enum {
    RIME_FP32 = 0,        /* FP32 arithmetic; phase reduced exactly in double-float; FP64 chi^2 sums */
    RIME_FP64 = 1         /* FP64 throughout */
} rime_precision;

/* Problem dimensions (Table 1) and the two model constants. */
typedef struct {
    int32_t na;           /* antennas, >= 2 */
    int32_t ntime;        /* timesteps, >= 1 */
    int32_t nchan;        /* channels, >= 1 */
    int32_t precision;    /* rime_precision */
    double ref_freq_hz;   /* nu_ref of eq. 2 (> 0); 1.4e9 in the paper's sample code */
    double beam_c;        /* C of eq. 4 in rad^-1 GHz^-1 (>= 0); 65 for WSRT */
} rime_dims;

/* A sky model (Table 2: lm, brightness, gaussian shapes), structure of
 * arrays, double precision (kind: int32), host or device pointers. */
typedef struct {
    int32_t nsrc;         /* >= 0 */
    int32_t time_varying; /* 0: stokes [nsrc][4]; 1: stokes [ntime][nsrc][4] (Table 2) */
    const double *lm;     /* [nsrc][2] direction cosines (l, m), l^2 + m^2 < 1 */
    const double *stokes; /* Stokes (I, Q, U, V) in Jy at nu_ref */
    const double *alpha;  /* [nsrc] spectral index (eq. 2) */
    const double *shape;  /* [nsrc][3] (major, minor, pa) in rad, major >= minor >= 0,
                             pa from +m towards +l; (0, 0, *) is a point source.
                             NULL: all sources are points. */
    const int32_t *kind;  /* [nsrc] morphology of a source with a shape, or NULL (all 0):
                             0 Gaussian, major / minor its FWHM:
                               g = exp(-pi^2 (major^2 u_maj^2 + minor^2 u_min^2) / (4 ln 2));
                             1 exponential disk (the Sersic profile of index 1 that
                               Sec. 1 names), major / minor its scale lengths:
                               g = (1 + 4 pi^2 (major^2 u_maj^2 + minor^2 u_min^2))^(-3/2);
                             with (u_maj, u_min) = (u sin pa + v cos pa, u cos pa - v sin pa)
                             the baseline (u_p - u_q, v_p - v_q) / lambda. Another value
                             is RIME_E_INVALID (reported by the next waiting call). */
} rime_sources;

/* Number of baselines na*(na-1)/2 (Sec. 2.2). */
int64_t rime_nbl(int32_t na);

/* Human-readable name of a status code. Never NULL. */
const char *rime_status_string(rime_status s);

/* Creates a context: validates dims, allocates the device buffers the
 * problem needs and uploads the observation (Table 2 inputs from the
 * measurement set). Waits for the stream.
 *   ctx       out: the new context (NULL on failure)
 *   dims      problem dimensions and model constants
 *   freq_hz   [nchan] channel frequencies, > 0
 *   uvw       [ntime][na][3] antenna coordinates in metres
 *   pointing  [ntime][na][2] pointing errors (dl, dm) in rad, or NULL (none)
 *   data      [ntime][nbl][nchan][4] complex observed visibilities, or NULL
 *             (rime_predict still works; rime_chi2 needs data)
 *   weight    [ntime][nbl][nchan] float (FP32) / double (FP64), >= 0, or NULL
 *             (unit weights)
 *   cuda_stream  cudaStream_t to order all work on (NULL: legacy default stream)
 * Errors: RIME_E_INVALID (sizes, NULL required pointers, invalid values in
 * freq/uvw/data/weight), RIME_E_NONFINITE, RIME_E_OOM, RIME_E_CUDA. */
rime_status rime_create(rime_ctx **ctx, const rime_dims *dims, const double *freq_hz,
                        const double *uvw, const double *pointing, const void *data,
                        const void *weight, void *cuda_stream);

/* Replaces uvw [ntime][na][3] and pointing [ntime][na][2] (NULL: none). */
rime_status rime_set_uvw(rime_ctx *ctx, const double *uvw, const double *pointing);

/* Replaces the observed data and weights (same layouts as rime_create;
 * weight NULL: unit weights). */
rime_status rime_set_data(rime_ctx *ctx, const void *data, const void *weight);

/* Sets the direction-independent gains G_tpk of eq. 1:
 * [ntime][na][nchan][4] complex128 (the 2x2 Jones matrix, row-major), or NULL
 * for identity gains (the default). */
rime_status rime_set_gains(rime_ctx *ctx, const double *gains);

/* Sets the sky model (Table 2) and precomputes the per-source and
 * per-(time, source, antenna) factors of eqs. 2-4 on the GPU. Does not wait. */
rime_status rime_set_sources(rime_ctx *ctx, const rime_sources *src);

/* Model visibilities V (eq. 1) for every (t, bl, k): writes
 * vis_out [ntime][nbl][nchan][4] complex (device pointer, caller-owned).
 * Algorithms 1-2 with the per-antenna factors kept on chip. Does not wait. */
rime_status rime_predict(rime_ctx *ctx, void *vis_out);

/* chi^2 of eq. 7 (without the ln-weight term), fused with the predict: the
 * visibilities are never written to memory. Waits for the stream and stores
 * the value in *chi2 (host pointer). Requires data. */
rime_status rime_chi2(rime_ctx *ctx, double *chi2);

/* As rime_chi2 but leaves the result in device memory (*chi2_dev, one
 * double) and does not wait; suitable for CUDA graph capture. */
rime_status rime_chi2_async(rime_ctx *ctx, double *chi2_dev);

/* chi^2 (eq. 7) and its gradient: the adjoint of eqs. 1-7 with respect to
 * every source parameter and every gain, recomputing K and E (eqs. 3-4)
 * rather than storing them. Waits for the stream.
 *   chi2        host pointer, receives chi^2 (the same value rime_chi2 gives)
 *   grad_src    device [nsrc][10] double: d chi^2 / d(l, m, I, Q, U, V, alpha,
 *               major, minor, pa) (the shape derivatives are 0 for points)
 *   grad_gains  device [ntime][na][nchan][4] complex128, or NULL: the complex
 *               gradient d chi^2/dRe G + i d chi^2/dIm G of each Jones entry
 *               (with identity gains when none are set)
 * Needs static brightness (time_varying = 0), else RIME_E_INVALID. Uses a
 * device buffer of one complex Y_X per visibility and correlation, one
 * partial per (t, channel, antenna unit, source) and, when grad_gains is
 * given, the 8 complex gains-gradient terms of each visibility (16 values of
 * the context's precision), all allocated on first use. Every sum runs in a
 * fixed order: repeated calls give bit-identical results. */
rime_status rime_chi2_grad(rime_ctx *ctx, double *chi2, double *grad_src, void *grad_gains);

/* sum over visibilities of ln(2 pi / w) (the second term of eq. 7), so that
 * -2 ln L = chi^2 + rime_ln_norm. Waits for the stream. */
rime_status rime_ln_norm(rime_ctx *ctx, double *ln_norm);

/* Waits for all work on the context's stream and returns any deferred
 * status (failed input checks, kernel errors). */
rime_status rime_sync(rime_ctx *ctx);

/* Tensor-core modes of an RIME_FP32 context (rime_set_tensor_mode). */
typedef enum {
    RIME_TC_OFF = 0,          /* direct FP32 source sum (default) */
    RIME_TC_SPLIT_BF16 = 1,   /* tcgen05 products of BF16 hi + lo operand pairs, FP32 accumulation */
    RIME_TC_SPLIT_TF32 = 2,   /* the same with TF32 hi + lo pairs (more accurate, half the rate) */
    RIME_TC_SPLIT_F16 = 3     /* FP16 hi + lo pairs: TF32's significand at the BF16 rate; scaled
                                 Stokes values must stay below 6e4 in magnitude */
} rime_tc_mode;

/* Selects how rime_predict, rime_chi2 and rime_chi2_async evaluate the source
 * sum of an RIME_FP32 context. With point sources the sum over s of
 * A_ps X_s conj(A_qs), A = E K per antenna (eqs. 3-4), is a complex matrix
 * product A diag(X) A^H for each (t, k) and Stokes X (the source sum of
 * Algorithm 2 for all baselines at once); the split modes run it on the
 * tensor cores with each operand split into a rounded high part and a
 * rounded remainder (three products, FP32 accumulation). The phase nu tau is
 * reduced exactly before its sine and cosine are taken with the SFU (the
 * FP64 value of the reduced argument to within one FP32 unit of 1/2, see
 * rime_phase_turns), and the chi^2 is summed in FP64. Errors against the FP64
 * result on 256 antennas, 128 channels and 4096 point sources (|V| ~ 1e2 Jy,
 * residuals at a 0.01 Jy noise level; 192 sampled visibilities, chi^2 on one
 * timestep and two channels): BF16 5.8e-6 of the largest visibility and
 * 7.7e-4 of chi^2 (above an FP32 bound of 1e-4); TF32 8.6e-7 and 3.0e-5
 * (within it); FP16 8.7e-7 and 1.7e-5 (within it, at the BF16 rate). The
 * FP16 split needs every scaled Stokes value (the source's Stokes vector
 * times (nu / nu_ref)^alpha, and E^2 without pointing errors) below 6e4 in
 * magnitude: otherwise the next waiting call returns RIME_E_INVALID and
 * leaves its outputs untouched.
 * The split modes take point sources only: a sky model with a Gaussian
 * source makes the next waiting call return RIME_E_INVALID. rime_chi2_grad
 * and rime_chi2_batched always use the direct FP32 path.
 *   mode  a rime_tc_mode; RIME_E_INVALID for an RIME_FP64 context. */
rime_status rime_set_tensor_mode(rime_ctx *ctx, int32_t mode);

/* The split modes' tile plan for na antennas (host only, no GPU needed).
 * The paper has no counterpart: it is the work decomposition of the
 * tensor-core form of Algorithm 2's source sum (rime_set_tensor_mode).
 * Antennas fall into groups of 32 (the last one ragged); one CTA of the split
 * kernel computes, for one (t, k), the products of up to four row groups
 * (128 rows) against one column group. S_X is Hermitian (S_X[q, p] =
 * conj S_X[p, q] for real X), so each unordered pair of distinct groups is
 * computed in exactly one tile, in either orientation, and each group's own
 * baselines in one tile whose rows include the column group itself.
 *   na    antennas, 2 .. 4096
 *   out   [cap][5] int32: the column group, then four row groups (-1: empty)
 *   cap   tiles out can hold (0: only count them)
 * Returns the number of tiles (256 antennas: 9), or -1 for na out of range,
 * cap < 0, or out NULL with cap > 0. */
int32_t rime_split_tiles(int32_t na, int32_t *out, int32_t cap);

/* chi^2 (eq. 7, without the ln-weight term) of an observation whose data
 * and weights stay in host memory, streamed to the GPU in chunks of
 * chunk_ntime timesteps (the time subdivision of Sec. 4.4): while the fused
 * kernel reduces earlier chunks (alternating between the context's stream
 * and a second kernel stream), the next ones are copied on a copy stream
 * into a ring of up to eight device buffers, and the chunk values are added
 * in chunk order. The copies start after the context's latest upload
 * (rime_set_uvw / _gains / _sources / _data) has been copied. Device memory
 * for the data is the ring (at most half of the free memory, at least two
 * chunks), not the observation: an observation larger than the GPU fits.
 * The context's uvw, gains and sources
 * cover the whole observation; its own data buffer is not used (the context
 * may be created with data = NULL). The tensor-core modes do not apply.
 *   data         [ntime][nbl][nchan][4] complex, host memory (pinned memory
 *                lets the copies overlap the kernels; pageable works, without
 *                overlap) or device memory
 *   weight       [ntime][nbl][nchan] real, or NULL (unit weights)
 *   chunk_ntime  timesteps per chunk; <= 0: rime_stream_chunk_ntime(ctx), with a
 *                first chunk a quarter as long (its copy is not overlapped)
 *   chi2         out: host pointer
 * Waits for the result. Each chunk's data and weights are checked on the GPU
 * as they arrive: NaN/Inf gives RIME_E_NONFINITE, a negative weight
 * RIME_E_INVALID (the index in the message is the visibility's in the whole
 * observation); such an error concerns this call only. */
rime_status rime_chi2_streamed(rime_ctx *ctx, const void *data, const void *weight, int32_t chunk_ntime,
                               double *chi2);

/* The chunk length rime_chi2_streamed picks: about one wave of the fused
 * kernel per chunk (2 blocks per SM), at most ntime. 0 for a NULL context. */
int32_t rime_stream_chunk_ntime(const rime_ctx *ctx);

/* Chains: per-chain residuals for a sampler whose proposals move a few
 * sources at a time (the BIRO loop of Sec. 2.3 with Metropolis moves).
 * Chain c keeps N_c = D - V_c in device memory (V_c: the model visibilities
 * of the chain's current sky model; nchains * ntime * nbl * nchan * 4
 * complex values). Because eqs. 1-2 are linear in the Stokes vector, a
 * proposal that gives m sources new values changes the model by the
 * visibilities dV of a 2m-source sky model (the new values, and the current
 * values with the Stokes vector negated), and its chi^2 (eq. 7) is
 * sum w |dV - N_c|^2: the fused predict + chi^2 of 2m sources against N_c.
 * The chains use the direct kernels; they need static brightness. In FP32
 * the residuals gather rounding over many accepted moves (about 1e-7 of the
 * visibilities per move); rime_chains_init starts them afresh. */

/* Starts nchains chains at the context's sky model: N_c = D - V for all c.
 * Needs data and sources; allocates the residuals (RIME_E_OOM if they do not
 * fit). Does not wait. */
rime_status rime_chains_init(rime_ctx *ctx, int32_t nchains);

/* Evaluates one proposal per chain.
 *   nmove     sources moved per chain, >= 1
 *   proposed  nchains * nmove sources: chain c's new values of its moved
 *             sources are sources c*nmove .. c*nmove + nmove - 1
 *   current   the same sources' current values, in the same order (both
 *             give shape and kind, or both omit them)
 *   chi2_dev  device [nchains]: chi^2 of each chain's proposed sky model
 * The staged pairs become the context's sky model (rime_set_sources), which
 * rime_chains_accept then reads. Does not wait. */
rime_status rime_chains_propose(rime_ctx *ctx, int32_t nmove, const rime_sources *proposed,
                                const rime_sources *current, double *chi2_dev);

/* Applies the last proposal of the chains with accept[c] != 0 (host array
 * [nchains]): N_c -= dV_c. The caller records the accepted values as the
 * chains' current ones. Does not wait. */
rime_status rime_chains_accept(rime_ctx *ctx, const int32_t *accept);

/* Primary beam models E(x), x = beam_c * nu[GHz] * rho, rho the distance of
 * the source from the antenna's pointing centre (rime_set_beam). */
typedef enum {
    RIME_BEAM_COS3 = 0,   /* eq. 4 (WSRT): cos^3 x for x < pi/2, zero past the first null (default) */
    RIME_BEAM_JINC = 1    /* the Jinc that Sec. 2.1 names for the VLA: 2 J1(x) / x, the Airy
                             pattern of a uniformly illuminated dish (sidelobes change sign) */
} rime_beam;

/* Selects the beam model and its constant C (rad^-1 GHz^-1: 65 for the WSRT
 * cos^3 beam; pi D / (c * 1e-9 s) ~ 262 for a 25 m dish's Jinc). Applies to
 * every later call of the context (predict, chi^2, gradient, batched,
 * streamed, tensor-core modes). Does not wait.
 *   model   a rime_beam; RIME_E_INVALID otherwise
 *   beam_c  finite, >= 0; RIME_E_INVALID otherwise */
rime_status rime_set_beam(rime_ctx *ctx, int32_t model, double beam_c);

/* Limit of the bounded waits inside the tensor-core modes' kernels (their
 * pipeline of mbarriers between the warps that form the operands, the warp
 * that issues the MMAs and the warps that drain the accumulators): a block
 * whose wait lasts longer gives up, records the timeout, frees its tensor
 * memory once the MMAs it issued have completed, and the next call that waits
 * returns RIME_E_TIMEOUT (once; later calls run normally). For callers that
 * prefer an early error to a long stall, and for tests of that path.
 *   ns  nanoseconds; 0 restores the default of about two seconds
 * Does not wait. RIME_E_INVALID for a NULL context. */
rime_status rime_set_wait_limit(rime_ctx *ctx, uint64_t ns);

/* Direct-sum kernels of rime_predict, rime_chi2 and rime_chi2_async
 * (rime_set_kernel). */
typedef enum {
    RIME_KERNEL_AUTO = 0,     /* NARROW for arrays of up to 32 (FP32) or 45 (FP64) antennas,
                                 else TILED (default) */
    RIME_KERNEL_TILED = 1,    /* a block per (t, channel, antenna unit), several baselines per thread */
    RIME_KERNEL_NARROW = 2    /* a block per (t, group of channels), one or two (baseline,
                                 channel) pairs per thread; arrays of up to 45 antennas */
} rime_kernel;

/* Selects the kernel that evaluates the direct source sum (Algorithms 1-2
 * fused with eqs. 1 and 7) in both precisions; the result is the same sum
 * in another order (equal to rounding). TILED suits large arrays (each
 * staged per-antenna factor serves a whole antenna unit); NARROW suits small
 * ones, whose few baselines per channel would leave a tiled block nearly
 * empty. The gradient and the batched FP32 launch always use the tiled
 * kernel; the tensor-core modes take precedence when set.
 *   kernel  a rime_kernel; RIME_E_INVALID for another value, or for
 *           RIME_KERNEL_NARROW with more than 45 antennas. */
rime_status rime_set_kernel(rime_ctx *ctx, int32_t kernel);

/* Configuration of the batched FP32 launch, and the autotuner's record.
 * A work item of the persistent launch is (timestep, group of
 * channels_per_item channels, antenna unit, group of sets_per_item sets),
 * each set with all of its sources; the grid holds blocks_per_sm blocks per
 * SM. Sets of one item share their data, weights and gains. */
typedef struct {
    int32_t channels_per_item;  /* 1, 2 or 4 */
    int32_t blocks_per_sm;      /* 1 or 2 */
    int32_t order;              /* 0: largest sets first, 1: in set order */
    int32_t sets_per_item;      /* 1 .. 64 (the tuner tries 1, 4, 16) */
    int32_t tuned;              /* out: 1 if chosen by timing trials */
    int32_t ntrials;            /* out: configurations timed, <= 40 */
    int32_t trial_cfg[40][4];   /* out: (channels_per_item, blocks_per_sm, order, sets_per_item) */
    float trial_ms[40];         /* out: each trial's time on the trial sample, ms */
} rime_batch_config;

/* chi^2 (eq. 7) of nsets sky models against the context's observation, data
 * and gains: set j is sources src_offsets[j] .. src_offsets[j+1]-1 of `all`.
 * The paper evaluates one sky model per solve of its BIRO loop (Fig. 3,
 * Sec. 3); this entry point evaluates the many proposals of one sampler
 * iteration in one persistent launch of the tiled FP32 kernel, or in one
 * launch per set (FP64, and arrays that the small-array kernel takes under
 * rime_set_kernel: then the configuration below does not apply).
 *   nsets        >= 0 (0: nothing is computed)
 *   src_offsets  HOST array [nsets + 1], src_offsets[0] = 0, non-decreasing,
 *                src_offsets[nsets] = all->nsrc; empty sets are allowed
 *   all          the concatenated sources, as for rime_set_sources (they
 *                become the context's sources)
 *   chi2_dev     device array [nsets] of double, receives chi^2 of each set
 * Does not wait; suitable for CUDA graph capture once a first call with the
 * same sizes has run outside capture (it allocates the buffers and, in FP32,
 * times the candidate configurations on a sample of the work: the first
 * timesteps, every set). Under capture the schedule is recorded into the
 * graph as kernel arguments and the source arrays are re-read on each
 * replay, so `all` must then be device memory updated in place. Each set's
 * chi^2 is summed in a fixed order that does not depend on the
 * configuration: results are reproducible run to run.
 * Errors in source values are reported by the next call that waits. */
rime_status rime_chi2_batched(rime_ctx *ctx, int32_t nsets, const int32_t *src_offsets,
                              const rime_sources *all, double *chi2_dev);

/* The configuration the last FP32 rime_chi2_batched call used (zeros before
 * the first call). */
rime_status rime_batched_config(const rime_ctx *ctx, rime_batch_config *out);

/* Fixes the configuration of later batched calls (its first four fields;
 * the rest is ignored); NULL returns to timing trials. */
rime_status rime_set_batched_config(rime_ctx *ctx, const rime_batch_config *cfg);

/* chi^2 for callers that cannot allocate device memory. The paper has no
 * counterpart to this call.
 *
 * Who needs it: code that runs where cudaMalloc is not available to a
 * library -- for example inside a host framework whose memory pool has
 * reserved the device, or in a latency-critical loop where cudaMalloc's
 * implicit device synchronisation is not acceptable. Every other entry point
 * allocates device buffers in rime_create / rime_set_*.
 *
 * It evaluates the same fused predict + chi^2 as rime_chi2 for one problem
 * given entirely by the caller, and allocates nothing: all intermediates
 * (channel constants, converted gains, per-source constants, per-(t, s, a)
 * delays, work table, per-block partial sums, completion counter, status)
 * live in one fixed array of 32 MiB declared in the library's device code.
 * Every GPU on which the library's module containing this call is loaded
 * holds that array until the process exits.
 *
 *   dims, freq_hz, uvw, pointing, data, weight: as for rime_create, but all
 *             array pointers must be device pointers (pointing and weight may
 *             be NULL)
 *   gains     [ntime][na][nchan][4] complex128 device array, or NULL (identity)
 *   src       the sky model as for rime_set_sources (device pointers)
 *   chi2_dev  device pointer to one double, receives chi^2
 *   cuda_stream  the stream to order the work on
 * Limits: na <= 256, and the problem's intermediates must fit the 32 MiB
 * array (the 64-antenna, 100-timestep, 64-channel, 200-source FP32 problem
 * needs about 29 MB); larger problems return RIME_E_INVALID with the size
 * needed -- use the context API for those.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture. Every call reuses the same array and overwrites what the previous
 * call left there, so calls that overlap on the GPU (concurrent streams, or
 * several host threads on one device) race: serialise them.
 * Waits for the stream, then reports input checks like rime_chi2; errors are
 * read with rime_last_error(NULL). */
rime_status rime_chi2_noalloc(const rime_dims *dims, const double *freq_hz, const double *uvw,
                              const double *pointing, const void *data, const void *weight,
                              const double *gains, const rime_sources *src, double *chi2_dev,
                              void *cuda_stream);

/* The phase argument of eq. 3 as the FP32 kernels and the tensor-core modes
 * form it, for checking against an FP64 evaluation: for each i,
 * nu tau - round(nu tau) in turns (about [-1/2, 1/2]), with nu and tau split
 * into double-float pairs as the library splits channel frequencies and
 * delays (tau = (u l + v m + w (n - 1)) / c, eq. 3), multiplied exactly and
 * reduced exactly. It equals the FP64 value rounded to FP32 within about
 * 2^-24 + 2^-47 |nu tau| turns.
 *   n       >= 0 pairs
 *   nu_hz   [n] frequencies (Hz), tau_s [n] delays (s): host or device memory
 *   turns   [n] float, host or device memory
 * Uses its own temporary device buffers and the legacy default stream; waits
 * for the result. Errors: RIME_E_INVALID, RIME_E_OOM, RIME_E_CUDA (message
 * from rime_last_error(NULL)). */
rime_status rime_phase_turns(int64_t n, const double *nu_hz, const double *tau_s, float *turns);

/* Arithmetic pipes whose issue rates the roofline fractions of this
 * library's kernels are quoted against (rime_pipe_rate). The paper has no
 * counterpart to this call: it quotes its K40's nominal peaks (Sec. 4.3). */
typedef enum {
    RIME_PIPE_FFMA = 0,   /* FP32 fused multiply-add */
    RIME_PIPE_FFMA2 = 1,  /* FP32 FMA on packed pairs (counted as two) */
    RIME_PIPE_DFMA = 2,   /* FP64 fused multiply-add */
    RIME_PIPE_EX2 = 3     /* the SFU's exp2 approximation */
} rime_pipe;

/* Measures the rate of one pipe on the current device with a kernel of
 * independent register-resident chains over every SM (about 20 ms per
 * launch; uses the legacy default stream and a small temporary buffer).
 *   pipe        a rime_pipe
 *   ops_per_s   out: lane operations per second (one FMA counts one)
 * Errors: RIME_E_INVALID, RIME_E_OOM, RIME_E_CUDA. */
rime_status rime_pipe_rate(int32_t pipe, double *ops_per_s);

/* The message for the last failed call on this context ("" if none). */
const char *rime_last_error(const rime_ctx *ctx);

/* Frees the context and its device buffers. NULL is ignored. */
void rime_destroy(rime_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* RIME_H */
