// rime_narrow.cu -- the fused RIME predict + chi^2 (eqs. 1-7) for small
// arrays: one thread per (baseline, channel) pair.
//
// The tiled kernels of rime_fused.cu give a block one (t, channel, antenna
// unit) and a thread eight baselines; an array of 7 antennas has 21
// baselines, so such a block has 3 threads with work and the launch is a
// long chain of nearly empty blocks. Here a block owns one timestep and a
// group of cg channels, chosen so that cg * nbl fills the block (or, for
// 23..45 antennas, one channel and two pairs per thread):
//
//  * per chunk of sources it stages the per-antenna phase factors K (eq. 3),
//    times the beam E (eq. 4) when there are pointing errors, for the cg
//    channels in shared memory (Algorithm 1); each is reused by the na - 1
//    baselines of its antenna and channel;
//  * without pointing errors every antenna sees the same beam, so E_s^2 and
//    the spectral factor (nu/nu_ref)^alpha of eq. 2 scale the source's Stokes
//    vector once per (channel, source);
//  * each thread accumulates its pair's four Stokes sums sum_s z_s X_s with
//    z = A_p conj(A_q) g (Algorithm 2), the Gaussian exponent evaluated from
//    the pair's own nu^2 (du^2, du dv, dv^2);
//  * the epilogue and the chi^2 reduction are those of the tiled kernels.
//
// Both precisions share the code; the FP32 phase is the double-float
// reduction of the tiled FP32 kernel, the FP64 one is reduced in FP64.
#include "rime_internal.cuh"
#include "rime_dev.cuh"
#include "rime_fused_common.cuh"

#include <algorithm>
#include <type_traits>

namespace rime {
namespace narrow {

constexpr int CG_MAX = 64;   // channels per block at most (bounds the staged factors of tiny arrays)

template <typename T> struct Cfg;
template <> struct Cfg<float> {
    static constexpr int SC = 32;    // sources per chunk
    using T2 = float2;
    using T4 = float4;
    using Chan = ChanF;
};
template <> struct Cfg<double> {
    static constexpr int SC = 16;
    using T2 = double2;
    struct T4 { double x, y, z, w; };
    using Chan = ChanD;
};

// Per-launch shape: channels per block, pairs per thread, threads per
// block, channel groups. Up to 256 baselines: 256 threads, one pair each,
// as many channels as fit; up to 512: one channel, two pairs per thread;
// up to 1024 (45 antennas): 512 threads of two pairs.
struct Shape {
    int cg, m, nt, ngroups;
};

static Shape shape_for(int na, int ntime, int nchan, int nsm) {
    const int nbl = na * (na - 1) / 2;
    Shape s;
    if (nbl <= 256) {
        s.cg = std::max(1, std::min(std::min(nchan, CG_MAX), 256 / nbl));
        // small problems: fewer channels per block, so that the blocks cover
        // every SM twice (the FP64 pipe of each SM is the limit there)
        const long long fit = std::max(1LL, (long long)ntime * nchan / (2LL * std::max(nsm, 1)));
        s.cg = (int)std::min<long long>(s.cg, fit);
        s.m = 1;
        s.nt = 256;
    } else {
        s.cg = 1;
        s.m = 2;
        s.nt = nbl <= 512 ? 256 : 512;
    }
    s.ngroups = (nchan + s.cg - 1) / s.cg;
    return s;
}

template <typename T>
static size_t smem_bytes(int na, int cg) {
    using C = Cfg<T>;
    return (size_t)cg * C::SC * na * sizeof(typename C::T2)      // K (times E) per (channel, source, antenna)
           + (size_t)cg * C::SC * sizeof(typename C::T4)         // scaled Stokes per (channel, source)
           + (size_t)C::SC * sizeof(typename C::T4)              // Gaussian coefficients per source
           + 32 * sizeof(double);                                // reduction scratch
}

// K = exp(2 pi i nu tau) for the delay stored for (t, s, a).
__device__ __forceinline__ float2 phase_of(const float2 *tau, long long di, const ChanF &ch) {
    return f32::phase_factor(tau[di], ch);
}
__device__ __forceinline__ double2 phase_of(const double *tau, long long di, const ChanD &ch) {
    const double ph = ch.nu * tau[di];     // turns
    const double r = ph - round_int_d(ph);
    double sn, cs;
    sincospi(2.0 * r, &sn, &cs);
    return make_double2(cs, sn);
}
// E of eq. 4 (or the Jinc model) at C nu[GHz] rho.
__device__ __forceinline__ float beam_of(float rho, const ChanF &ch) { return f32::beam(rho, ch); }
__device__ __forceinline__ double beam_of(double rho, const ChanD &ch) { return beam_E(ch.beam, ch.cnu * rho); }
// (nu / nu_ref)^alpha = 2^(2 alpha hlr)
__device__ __forceinline__ float spectral(float alpha, const ChanF &ch) { return exp2f(2.0f * alpha * ch.hlr); }
__device__ __forceinline__ double spectral(double alpha, const ChanD &ch) { return exp2(2.0 * alpha * ch.hlr); }
// Shape factor from the quadratic form e of the baseline: Gaussian exp(e)
// (log2 units in FP32, natural in FP64, as the upload kernel stores the
// coefficients), exponential disk (1 + e)^(-3/2)
__device__ __forceinline__ float gauss_of(float e) { return ex2_approx(e); }
__device__ __forceinline__ double gauss_of(double e) { return exp(e); }
__device__ __forceinline__ float disk_of(float e) {
    const float r = rsqrtf(1.0f + e);
    return r * r * r;
}
__device__ __forceinline__ double disk_of(double e) {
    const double r = rsqrt(1.0 + e);
    return r * r * r;
}
__device__ __forceinline__ float nu2_of(const ChanF &ch) { return ch.nu2; }
__device__ __forceinline__ double nu2_of(const ChanD &ch) { return ch.nu2; }

template <typename T, int M, int THREADS, int MODE>
__global__ void __launch_bounds__(THREADS) k_narrow(const FusedParams P, const int cg, const int ngroups) {
    using C = Cfg<T>;
    using T2 = typename C::T2;
    using T4 = typename C::T4;
    using Chan = typename C::Chan;
    constexpr int SC = C::SC;
    constexpr bool CHI2 = MODE != MODE_PREDICT, WRITE = MODE == MODE_PREDICT, GRAD = MODE == MODE_GRAD;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int na = P.na;
    T2 *sA = reinterpret_cast<T2 *>(smem_raw);                       // [cg][SC][na]
    T4 *sSt = reinterpret_cast<T4 *>(sA + (size_t)cg * SC * na);     // [cg][SC]
    T4 *sG = sSt + cg * SC;                                          // [SC]
    double *sRed = reinterpret_cast<double *>(sG + SC);              // [32]
    __shared__ int sLast;

    if (inputs_bad(P.status)) return;
    const int tid = threadIdx.x;
    const int tl = blockIdx.x / ngroups;
    const int t = P.t_begin + tl;
    const int k0 = (blockIdx.x - tl * ngroups) * cg;
    const int ncg = min(cg, P.nchan - k0);
    const int nbl = (int)P.nbl;
    const Chan *chan = reinterpret_cast<const Chan *>(P.chan);
    const bool pointing = P.has_pointing != 0;

    // ---- this thread's pairs: j = tid + THREADS i -> channel j / nbl, baseline j % nbl ----
    bool act[M];
    int kk[M], bb[M], pp[M], qq[M], offp[M], offq[M], offs[M];
    T du2[M], dudv[M], dv2[M];
#pragma unroll
    for (int i = 0; i < M; i++) {
        const int j = tid + THREADS * i;
        const int c = j / nbl, b = j - c * nbl;
        act[i] = c < ncg;
        int p = 0, r = b;
        while (r >= na - 1 - p) {   // row p of the upper triangle holds na - 1 - p baselines
            r -= na - 1 - p;
            p++;
        }
        const int q = p + 1 + r;
        kk[i] = k0 + (act[i] ? c : 0);
        bb[i] = b;
        pp[i] = p;
        qq[i] = q;
        offp[i] = (act[i] ? c : 0) * SC * na + p;
        offq[i] = (act[i] ? c : 0) * SC * na + q;
        offs[i] = (act[i] ? c : 0) * SC;
        if constexpr (sizeof(T) == 4) {
            // FP32 inputs are FP32 values: one rounding in the difference (the
            // FP64 pipe runs at 1/64 of the FP32 rate; this setup is per pair)
            const float4 xp = P.uvw_f[(long long)t * na + p], xq = P.uvw_f[(long long)t * na + q];
            const float du = xp.x - xq.x, dv = xp.y - xq.y, nu2 = nu2_of(chan[kk[i]]);
            du2[i] = nu2 * du * du;
            dudv[i] = nu2 * du * dv;
            dv2[i] = nu2 * dv * dv;
        } else {
            const double *xp = P.uvw + 3 * ((long long)t * na + p);
            const double *xq = P.uvw + 3 * ((long long)t * na + q);
            const double du = xp[0] - xq[0], dv = xp[1] - xq[1];
            const double nu2 = nu2_of(chan[kk[i]]);
            du2[i] = nu2 * du * du;
            dudv[i] = nu2 * du * dv;
            dv2[i] = nu2 * dv * dv;
        }
    }

    T acc[M][8];
#pragma unroll
    for (int i = 0; i < M; i++)
#pragma unroll
        for (int c = 0; c < 8; c++) acc[i][c] = T(0);

    const auto *tau = reinterpret_cast<const typename std::conditional<sizeof(T) == 4, float2, double>::type *>(P.tau);
    const T *rho = reinterpret_cast<const T *>(P.rho);
    const T *stokes = reinterpret_cast<const T *>(P.stokes) + (long long)t * P.stokes_tstride;
    const T *gauss = reinterpret_cast<const T *>(P.gauss);
    const T *alpha = reinterpret_cast<const T *>(P.alpha);

    for (int s0 = P.src0; s0 < P.src1; s0 += SC) {
        const int sc = min(SC, P.src1 - s0);
        __syncthreads();
        // ---- stage K (times E with pointing errors) per (channel, source, antenna) ----
        const int per_c = sc * na;
        for (int i = tid; i < ncg * per_c; i += THREADS) {
            const int c = i / per_c, r = i - c * per_c;
            const int s = r / na, a = r - s * na;
            const Chan ch = chan[k0 + c];
            const long long di = ((long long)t * P.nsrc + s0 + s) * na + a;
            T2 v = phase_of(tau, di, ch);
            if (pointing) {
                const T E = beam_of(rho[di], ch);
                v.x *= E;
                v.y *= E;
            }
            sA[(c * SC + s) * na + a] = v;
        }
        // ---- Stokes scaled by the spectral factor (and E^2 without pointing errors) ----
        for (int i = tid; i < ncg * sc; i += THREADS) {
            const int c = i / sc, s = i - c * sc;
            const Chan ch = chan[k0 + c];
            T f = spectral(alpha[s0 + s], ch);
            if (!pointing) {
                const T E = beam_of(rho[((long long)t * P.nsrc + s0 + s) * na], ch);
                f *= E * E;
            }
            const T *x = stokes + 4 * (long long)(s0 + s);
            sSt[c * SC + s] = T4{x[0] * f, x[1] * f, x[2] * f, x[3] * f};
        }
        if (tid < sc) {
            const T *g = gauss + 4 * (long long)(s0 + tid);
            sG[tid] = T4{g[0], g[1], g[2], g[3]};
        }
        __syncthreads();

        // ---- source sum of this thread's pairs ----
#pragma unroll 2
        for (int s = 0; s < sc; s++) {
            const T4 g = sG[s];
            const bool is_gauss = g.w != T(0), is_disk = g.w > T(1.5);
#pragma unroll
            for (int i = 0; i < M; i++) {
                if (!act[i]) continue;
                const T2 ap = sA[offp[i] + s * na], aq = sA[offq[i] + s * na];
                T zr = ap.x * aq.x + ap.y * aq.y;
                T zi = ap.y * aq.x - ap.x * aq.y;
                if (is_gauss) {
                    const T e = g.x * du2[i] + g.y * dudv[i] + g.z * dv2[i];
                    const T gg = is_disk ? disk_of(e) : gauss_of(e);
                    zr *= gg;
                    zi *= gg;
                }
                const T4 st = sSt[offs[i] + s];
                acc[i][0] += zr * st.x; acc[i][1] += zi * st.x;
                acc[i][2] += zr * st.y; acc[i][3] += zi * st.y;
                acc[i][4] += zr * st.z; acc[i][5] += zi * st.z;
                acc[i][6] += zr * st.w; acc[i][7] += zi * st.w;
            }
        }
    }

    // ---- epilogue: S (eq. 2), gains (eq. 1), chi^2 terms (eq. 7) ----
    double chi = 0.0;
    const T2 *gains = reinterpret_cast<const T2 *>(P.gains);
    const T2 *data = reinterpret_cast<const T2 *>(P.data);
    const T *weight = reinterpret_cast<const T *>(P.weight);
    T2 *vis = reinterpret_cast<T2 *>(P.vis_out);
    const T2 one{T(1), T(0)}, zero{T(0), T(0)};
    const T2 I2[4] = {one, zero, zero, one};
#pragma unroll
    for (int i = 0; i < M; i++) {
        if (!act[i]) continue;
        const T *a = acc[i];
        T2 Sm[4];
        Sm[0] = T2{a[0] + a[2], a[1] + a[3]};   // I + Q
        Sm[1] = T2{a[4] - a[7], a[5] + a[6]};   // U + iV
        Sm[2] = T2{a[4] + a[7], a[5] - a[6]};   // U - iV
        Sm[3] = T2{a[0] - a[2], a[1] - a[3]};   // I - Q
        const int p = pp[i], q = qq[i], k = kk[i];
        T2 gp[4], gq[4], V[4], tmp[4], gqh[4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            gp[c] = P.has_gains ? gains[4 * (((long long)t * na + p) * P.nchan + k) + c] : I2[c];
            gq[c] = P.has_gains ? gains[4 * (((long long)t * na + q) * P.nchan + k) + c] : I2[c];
        }
        mmul(gp, Sm, tmp);      // eq. 1: V = G_p S G_q^H
        mherm(gq, gqh);
        mmul(tmp, gqh, V);
        const long long row = ((long long)t * P.nbl + bb[i]) * P.nchan + k;
        if constexpr (WRITE) {
#pragma unroll
            for (int c = 0; c < 4; c++) vis[4 * row + c] = V[c];
        }
        if constexpr (CHI2) {
            T r2 = T(0);
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const T2 D = data[4 * row + c];
                const T dr = V[c].x - D.x, dim = V[c].y - D.y;
                r2 += dr * dr + dim * dim;
            }
            const T w = P.has_weight ? weight[row] : T(1);
            chi += (double)(w * r2);
            if constexpr (GRAD) {
                // the Stokes-projected adjoint of this visibility and its gains
                // gradient (eq. 7 through eq. 1), as the tiled kernel's gradient mode
                T2 D[4], Y[4], dGp[4], dGq[4];
#pragma unroll
                for (int c = 0; c < 4; c++) D[c] = data[4 * row + c];
                grad_terms<T, T2>(V, Sm, D, w, gp, gq, Y, dGp, dGq);
                T2 *yo = reinterpret_cast<T2 *>(P.yout) + 4 * row;
#pragma unroll
                for (int c = 0; c < 4; c++) yo[c] = Y[c];
                if (P.dgain) {   // this visibility's terms of the gains gradient
                    T2 *go = reinterpret_cast<T2 *>(P.dgain) + 4 * row;
                    const long long plane = 4ll * P.ntime * P.nbl * P.nchan;
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        go[c] = dGp[c];
                        go[plane + c] = dGq[c];
                    }
                }
            }
        }
    }
    if constexpr (CHI2) {
        const double bsum = block_sum<THREADS>(chi, sRed);
        finish_chi2<THREADS>(bsum, P, sRed, &sLast);
    }
}

template <typename T, int M, int NT>
static cudaError_t launch_t(const FusedParams &P, int mode, const Shape &s, int blocks, size_t smem,
                            cudaStream_t stream) {
    auto kern = mode == MODE_PREDICT ? k_narrow<T, M, NT, MODE_PREDICT>
                : mode == MODE_CHI2  ? k_narrow<T, M, NT, MODE_CHI2>
                                     : k_narrow<T, M, NT, MODE_GRAD>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<blocks, NT, smem, stream>>>(P, s.cg, s.ngroups);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_shape(const FusedParams &P, int mode, const Shape &s, int blocks, size_t smem,
                                cudaStream_t stream) {
    if (s.m == 1) return launch_t<T, 1, 256>(P, mode, s, blocks, smem, stream);
    if (s.nt == 256) return launch_t<T, 2, 256>(P, mode, s, blocks, smem, stream);
    return launch_t<T, 2, 512>(P, mode, s, blocks, smem, stream);
}

}  // namespace narrow

bool narrow_applies(const rime_ctx *c) {
    if (c->kernel == RIME_KERNEL_TILED) return false;
    if (c->kernel == RIME_KERNEL_NARROW) return true;   // na <= NARROW_MAX_NA, checked when set
    // measured crossovers: the FP32 tiled kernel is as fast from ~33 antennas on
    // (packed FP32 pairs, 8 baselines per thread); the FP64 one uses 32-antenna
    // units that leave blocks part empty up to 64 antennas
    return c->dims.na <= (c->dims.precision == RIME_FP64 ? NARROW_MAX_NA : NARROW_AUTO_NA_F32);
}

cudaError_t launch_narrow(rime_ctx *c, int mode, void *vis_out, double *result, int src0, int src1, void *yout,
                          void *dgain) {
    FusedParams P{};
    fill_fused_params(c, P, vis_out, result, yout, dgain);
    P.src0 = src0;
    P.src1 = src1;
    return launch_narrow_params(c, mode, P, c->dims.ntime);
}

long long narrow_blocks_per_time(rime_ctx *c) {
    if (c->nsm <= 0 && cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
        c->nsm = 152;
    return narrow::shape_for(c->dims.na, c->dims.ntime, c->dims.nchan, c->nsm).ngroups;
}

cudaError_t launch_narrow_params(rime_ctx *c, int mode, const FusedParams &P, int nt, cudaStream_t stream) {
    if (!stream) stream = c->stream;
    using namespace narrow;
    if (c->nsm <= 0 && cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
        c->nsm = 152;
    const Shape s = shape_for(c->dims.na, c->dims.ntime, c->dims.nchan, c->nsm);
    const long long blocks = (long long)nt * s.ngroups;
    if (blocks == 0) return cudaSuccess;
    if (blocks > (long long)c->partials_cap) return cudaErrorInvalidValue;   // cannot happen: <= fused blocks
    const bool f64 = c->dims.precision == RIME_FP64;
    const size_t smem = f64 ? smem_bytes<double>(c->dims.na, s.cg) : smem_bytes<float>(c->dims.na, s.cg);
    if (f64) return launch_shape<double>(P, mode, s, (int)blocks, smem, stream);
    return launch_shape<float>(P, mode, s, (int)blocks, smem, stream);
}

cudaError_t launch_fused_auto(rime_ctx *c, void *vis_out, double *result, bool chi2) {
    if (narrow_applies(c))
        return launch_narrow(c, chi2 ? MODE_CHI2 : MODE_PREDICT, vis_out, result, 0, c->nsrc);
    return launch_fused(c, vis_out, result, chi2);
}

}  // namespace rime
