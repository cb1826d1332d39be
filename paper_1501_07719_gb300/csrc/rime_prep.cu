// rime_prep.cu -- upload-time kernels: input checks and the per-channel,
// per-source and per-(time, source, antenna) factors of eqs. 2-4.
//
// Everything the fused kernel needs in double precision is computed here,
// once per upload, so that the FP32 fused kernel runs no FP64 instruction.
#include "rime_internal.cuh"

#include <algorithm>
#include "rime_fused_common.cuh"

#include <math.h>

namespace rime {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void flag(DevStatus *st, int cls, int bits, long long idx) {
    atomicOr(&st->err[cls], bits);
    atomicMin(&st->first_bad[cls], idx);
}

__device__ __forceinline__ bool finite(double x) { return isfinite(x); }

// Per-channel constants of eqs. 2-4.
__global__ void k_prep_channels(int nchan, const double *freq, double ref_freq, double beam_c, int beam_model,
                                int fp64, void *chan, DevStatus *st) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nchan) return;
    double nu = freq[k];
    if (!finite(nu)) flag(st, EC_FREQ, EB_NONFINITE, k);
    else if (!(nu > 0.0)) flag(st, EC_FREQ, EB_RANGE, k);
    // sqrt of the spectral factor (nu / nu_ref)^alpha is 2^(alpha * hlr)
    double hlr = 0.5 * log2(nu / ref_freq);
    double cnu = beam_c * (nu * 1e-9);
    if (fp64) {
        ChanD c{nu, hlr, cnu, nu * nu, beam_model, 0};
        reinterpret_cast<ChanD *>(chan)[k] = c;
    } else {
        ChanF c;
        c.nu_hi = (float)nu;
        c.nu_lo = (float)(nu - (double)c.nu_hi);
        c.hlr = (float)hlr;
        c.cnu = (float)cnu;
        c.nu2 = (float)(nu * nu);
        c.beam = beam_model;
        c.pad[0] = c.pad[1] = 0.f;
        reinterpret_cast<ChanF *>(chan)[k] = c;
    }
}

// uvw / pointing must be finite; the FP32 path also gets a float4 copy of uvw.
__global__ void k_validate_uvw(long long n_ta, const double *uvw, const double *pointing,
                               float4 *uvw_f, DevStatus *st) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_ta) return;
    double u = uvw[3 * i], v = uvw[3 * i + 1], w = uvw[3 * i + 2];
    bool ok = finite(u) && finite(v) && finite(w);
    if (pointing) ok = ok && finite(pointing[2 * i]) && finite(pointing[2 * i + 1]);
    if (!ok) flag(st, EC_UVW, EB_NONFINITE, i);
    if (uvw_f) uvw_f[i] = make_float4((float)u, (float)v, (float)w, 0.f);
}

template <typename T>
__global__ void k_validate_data(long long nvis, const T *data, const T *weight, DevStatus *st, int cls,
                                long long i0) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nvis) return;
    bool ok = true;
    if (data) {
#pragma unroll
        for (int c = 0; c < 8; c++) ok = ok && isfinite(data[8 * i + c]);
    }
    if (weight) {
        T w = weight[i];
        if (!isfinite(w)) ok = false;
        else if (w < T(0)) flag(st, cls, EB_RANGE, i0 + i);
    }
    if (!ok) flag(st, cls, EB_NONFINITE, i0 + i);
}

// complex128 gains -> compute precision; checks finiteness.
template <typename T>
__global__ void k_convert_gains(long long n, const double *in, T *out, DevStatus *st) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;   // n = number of doubles
    double x = in[i];
    if (!isfinite(x)) flag(st, EC_GAINS, EB_NONFINITE, i / 8);
    out[i] = (T)x;
}

// Per source: checks, the Gaussian exponent's quadratic form, brightness in
// the compute precision.  Shape factor (the Fourier transform of an
// elliptical Gaussian with FWHM axes maj, min at position angle pa):
//   ln g = -K nu^2 / c^2 [maj^2 (du sp + dv cp)^2 + min^2 (du cp - dv sp)^2]
//        = nu^2 (A du^2 + B du dv + C dv^2),   K = pi^2 / (4 ln 2).
// The FP32 path stores A, B, C scaled by log2(e) for an exp2.
template <typename T>
__global__ void k_prep_sources(int nsrc, int stokes_rows, const double *lm, const double *stokes,
                               const double *alpha, const double *shape, const int32_t *kind, T *o_stokes,
                               T *o_gauss, T *o_alpha, T *o_extra, double *o_geo, DevStatus *st) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long nst = (long long)stokes_rows * nsrc;
    if (i < nst) {
        bool ok = true;
#pragma unroll
        for (int c = 0; c < 4; c++) {
            double x = stokes[4 * i + c];
            ok = ok && isfinite(x);
            o_stokes[4 * i + c] = (T)x;
        }
        if (!ok) flag(st, EC_SRC, EB_NONFINITE, i % nsrc);
    }
    if (i >= nsrc) return;
    double l = lm[2 * i], m = lm[2 * i + 1], a = alpha[i];
    {
        // eq. 3's direction cosines: n - 1 = -(l^2+m^2)/(1+n) (no
        // cancellation); |lm| is the beam radius without pointing errors
        const double r2 = l * l + m * m;
        o_geo[4 * i + 0] = l;
        o_geo[4 * i + 1] = m;
        o_geo[4 * i + 2] = -r2 / (1.0 + sqrt(1.0 - r2));
        o_geo[4 * i + 3] = hypot(l, m);
    }
    double maj = 0.0, mn = 0.0, pa = 0.0;
    if (shape) {
        maj = shape[3 * i];
        mn = shape[3 * i + 1];
        pa = shape[3 * i + 2];
    }
    if (!(isfinite(l) && isfinite(m) && isfinite(a) && isfinite(maj) && isfinite(mn) && isfinite(pa)))
        flag(st, EC_SRC, EB_NONFINITE, i);
    else if (!(l * l + m * m < 1.0) || !(mn >= 0.0) || !(maj >= mn))
        flag(st, EC_SRC, EB_RANGE, i);
    const int kd = kind ? kind[i] : 0;
    if (kd != 0 && kd != 1) flag(st, EC_SRC, EB_RANGE, i);
    double sp, cp;
    sincos(pa, &sp, &cp);
    // the shape factor's quadratic form in the baseline (du, dv) in metres,
    // times nu^2 in the kernels: Gaussian exponent -pi^2/(4 ln 2) (... )/c^2
    // (log2 units in FP32, for ex2), disk q = 4 pi^2 (...)/c^2 in g = (1+q)^-3/2
    double k;
    if (kd == 1) {
        k = 4.0 * kPi * kPi / (kCLight * kCLight);
    } else {
        k = -kGaussK / (kCLight * kCLight);
        if (sizeof(T) == 4) k *= kLog2e;
    }
    double A = k * (maj * maj * sp * sp + mn * mn * cp * cp);
    double B = k * 2.0 * sp * cp * (maj * maj - mn * mn);
    double C = k * (maj * maj * cp * cp + mn * mn * sp * sp);
    bool extended = (maj != 0.0 || mn != 0.0);
    o_gauss[4 * i + 0] = (T)A;
    o_gauss[4 * i + 1] = (T)B;
    o_gauss[4 * i + 2] = (T)C;
    // 0 point, 1 Gaussian, 2 exponential disk
    o_gauss[4 * i + 3] = extended ? T(kd == 1 ? 2 : 1) : T(0);
    o_alpha[i] = (T)a;
    if (o_extra) {
        // for the gradient: l, m, l/n, m/n, major, minor, sin pa, cos pa
        double n = sqrt(1.0 - (l * l + m * m));
        T *x = o_extra + 8 * i;
        x[0] = (T)l; x[1] = (T)m; x[2] = (T)(l / n); x[3] = (T)(m / n);
        x[4] = (T)maj; x[5] = (T)mn; x[6] = (T)sp; x[7] = (T)cp;
    }
}

// Per (t, s, a): geometric delay tau = (u l + v m + w (n - 1)) / c in
// seconds (eq. 3 without the frequency) and the beam radius rho = |(l, m) -
// dl_ta| of eq. 4, from the per-source geometry (l, m, n - 1, |lm|) that the
// source kernel writes. A few FP64 operations per entry: the square root and
// division per source are done once there, 1/c is a constant, and the index
// arithmetic is 32-bit unless the table has 2^31 entries or more.
template <bool FP64, typename I>
__device__ __forceinline__ void prep_delay(I i, int nsrc, int na, const double *uvw, const double *pointing,
                                           const double *geo, void *tau_out, void *rho_out) {
    const int a = (int)(i % (I)na);
    const I ts = i / (I)na;
    const int s = (int)(ts % (I)nsrc);
    const I t = ts / (I)nsrc;
    const double *g = geo + 4 * s;   // 8-byte aligned only
    const long long ta = (long long)t * na + a;
    const double *x = uvw + 3 * ta;
    const double tau = fma(x[0], g[0], fma(x[1], g[1], x[2] * g[2])) * kInvCLight;
    double rho = g[3];
    if (pointing) {
        const double dl = g[0] - pointing[2 * ta], dm = g[1] - pointing[2 * ta + 1];
        rho = sqrt(fma(dl, dl, dm * dm));
    }
    if (FP64) {
        reinterpret_cast<double *>(tau_out)[i] = tau;
        reinterpret_cast<double *>(rho_out)[i] = rho;
    } else {
        const float hi = (float)tau;
        const float lo = (float)(tau - (double)hi);
        reinterpret_cast<float2 *>(tau_out)[i] = make_float2(hi, lo);
        reinterpret_cast<float *>(rho_out)[i] = (float)rho;
    }
}
template <bool FP64>
__global__ void k_prep_delays(long long n, int nsrc, int na, const double *uvw, const double *pointing,
                              const double *geo, void *tau_out, void *rho_out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (n <= 0x7fffffffLL) prep_delay<FP64>((int)i, nsrc, na, uvw, pointing, geo, tau_out, rho_out);
    else prep_delay<FP64>(i, nsrc, na, uvw, pointing, geo, tau_out, rho_out);
}

// sum ln(2 pi / w) over all visibilities (single block, fixed order).
template <typename T>
__global__ void k_ln_norm(long long nvis, const T *weight, DevStatus *st) {
    __shared__ double red[32];
    double acc = 0.0;
    for (long long i = threadIdx.x; i < nvis; i += blockDim.x) {
        double w = weight ? (double)weight[i] : 1.0;
        acc += log(2.0 * 3.141592653589793 / w);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) st->aux = v;
    }
}

inline unsigned blocks_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

cudaError_t launch_prep_channels(rime_ctx *c) {
    int n = c->dims.nchan;
    k_prep_channels<<<blocks_for(n), kThreads, 0, c->stream>>>(
        n, c->d_freq, c->dims.ref_freq_hz, c->dims.beam_c, c->beam_model, c->dims.precision == RIME_FP64, c->d_chan,
        c->d_status);
    return cudaGetLastError();
}

cudaError_t launch_validate_uvw(rime_ctx *c) {
    long long n = (long long)c->dims.ntime * c->dims.na;
    float4 *uvw_f = c->dims.precision == RIME_FP64 ? nullptr : reinterpret_cast<float4 *>(c->d_uvw_f);
    k_validate_uvw<<<blocks_for(n), kThreads, 0, c->stream>>>(
        n, c->d_uvw, c->has_pointing ? c->d_pointing : nullptr, uvw_f, c->d_status);
    return cudaGetLastError();
}

cudaError_t launch_validate_data(rime_ctx *c) {
    long long nvis = (long long)c->dims.ntime * c->nbl * c->dims.nchan;
    return launch_validate_chunk(c, nvis, c->has_data ? c->d_data : nullptr, c->has_weight ? c->d_weight : nullptr,
                                 EC_DATA, 0);
}

cudaError_t launch_validate_chunk(rime_ctx *c, long long nvis, const void *data, const void *weight, int cls,
                                  long long i0, cudaStream_t stream) {
    if (nvis == 0) return cudaSuccess;
    if (!stream) stream = c->stream;
    if (c->dims.precision == RIME_FP64)
        k_validate_data<double><<<blocks_for(nvis), kThreads, 0, stream>>>(
            nvis, (const double *)data, (const double *)weight, c->d_status, cls, i0);
    else
        k_validate_data<float><<<blocks_for(nvis), kThreads, 0, stream>>>(
            nvis, (const float *)data, (const float *)weight, c->d_status, cls, i0);
    return cudaGetLastError();
}

cudaError_t launch_convert_gains(rime_ctx *c) {
    long long n = (long long)c->dims.ntime * c->dims.na * c->dims.nchan * 8;
    if (c->dims.precision == RIME_FP64)
        k_convert_gains<double><<<blocks_for(n), kThreads, 0, c->stream>>>(
            n, c->d_gains_in, (double *)c->d_gains, c->d_status);
    else
        k_convert_gains<float><<<blocks_for(n), kThreads, 0, c->stream>>>(
            n, c->d_gains_in, (float *)c->d_gains, c->d_status);
    return cudaGetLastError();
}

cudaError_t launch_prep_sources(rime_ctx *c) {
    int nsrc = c->nsrc;
    if (nsrc == 0) return cudaSuccess;
    int rows = c->time_varying ? c->dims.ntime : 1;
    long long n = (long long)rows * nsrc;
    const double *shape = c->has_shape ? c->src_shape() : nullptr;
    const int32_t *kind = c->has_kind ? c->src_kind() : nullptr;
    if (c->dims.precision == RIME_FP64)
        k_prep_sources<double><<<blocks_for(n), kThreads, 0, c->stream>>>(
            nsrc, rows, c->src_lm(), c->src_stokes(), c->src_alpha(), shape, kind, (double *)c->d_stokes,
            (double *)c->d_gauss, (double *)c->d_alpha, (double *)c->d_src_extra, c->src_geo(), c->d_status);
    else
        k_prep_sources<float><<<blocks_for(n), kThreads, 0, c->stream>>>(
            nsrc, rows, c->src_lm(), c->src_stokes(), c->src_alpha(), shape, kind, (float *)c->d_stokes,
            (float *)c->d_gauss, (float *)c->d_alpha, (float *)c->d_src_extra, c->src_geo(), c->d_status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_prep_delays(c);
}

cudaError_t launch_prep_delays(rime_ctx *c) {
    int nsrc = c->nsrc;
    if (nsrc == 0 || !c->sources_set) return cudaSuccess;
    long long nd = (long long)c->dims.ntime * nsrc * c->dims.na;
    const double *pt = c->has_pointing ? c->d_pointing : nullptr;
    if (c->dims.precision == RIME_FP64)
        k_prep_delays<true><<<blocks_for(nd), kThreads, 0, c->stream>>>(nd, nsrc, c->dims.na, c->d_uvw, pt,
                                                                         c->src_geo(), c->d_tau, c->d_rho);
    else
        k_prep_delays<false><<<blocks_for(nd), kThreads, 0, c->stream>>>(nd, nsrc, c->dims.na, c->d_uvw, pt,
                                                                          c->src_geo(), c->d_tau, c->d_rho);
    return cudaGetLastError();
}

cudaError_t launch_ln_norm(rime_ctx *c) {
    long long nvis = (long long)c->dims.ntime * c->nbl * c->dims.nchan;
    if (c->dims.precision == RIME_FP64)
        k_ln_norm<double><<<1, 1024, 0, c->stream>>>(
            nvis, c->has_weight ? (const double *)c->d_weight : nullptr, c->d_status);
    else
        k_ln_norm<float><<<1, 1024, 0, c->stream>>>(
            nvis, c->has_weight ? (const float *)c->d_weight : nullptr, c->d_status);
    return cudaGetLastError();
}

// The reduced phase of eq. 3 as the FP32 kernels form it, for (nu, tau)
// pairs split into double-float pairs exactly as k_prep_channels and the
// delays kernel split them.
__global__ void k_phase_turns(long long n, const double *nu, const double *tau, float *out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float nh = (float)nu[i], nl = (float)(nu[i] - (double)nh);
        const float th = (float)tau[i], tl = (float)(tau[i] - (double)th);
        out[i] = f32::reduced_turns(make_float2(th, tl), nh, nl);
    }
}

}  // namespace rime

extern "C" rime_status rime_phase_turns(int64_t n, const double *nu_hz, const double *tau_s, float *turns) {
    using namespace rime;
    if (n < 0 || (n > 0 && (!nu_hz || !tau_s || !turns))) {
        set_global_error("rime_phase_turns: n must be >= 0 and the arrays non-NULL");
        return RIME_E_INVALID;
    }
    if (n == 0) return RIME_OK;
    double *d = nullptr;
    const size_t nb = (size_t)n * (2 * sizeof(double) + sizeof(float));
    cudaError_t e = cudaMalloc((void **)&d, nb);
    if (e != cudaSuccess) {
        set_global_error(cudaGetErrorString(e));
        return RIME_E_OOM;
    }
    float *o = reinterpret_cast<float *>(d + 2 * n);
    e = cudaMemcpy(d, nu_hz, (size_t)n * sizeof(double), cudaMemcpyDefault);
    if (e == cudaSuccess) e = cudaMemcpy(d + n, tau_s, (size_t)n * sizeof(double), cudaMemcpyDefault);
    if (e == cudaSuccess) {
        const long long blocks = std::min<long long>((n + 255) / 256, 4096);
        k_phase_turns<<<(unsigned)blocks, 256>>>(n, d, d + n, o);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(turns, o, (size_t)n * sizeof(float), cudaMemcpyDefault);
    cudaFree(d);
    if (e != cudaSuccess) {
        set_global_error(cudaGetErrorString(e));
        return RIME_E_CUDA;
    }
    return RIME_OK;
}
