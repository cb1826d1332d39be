// rime_chains.cu -- per-chain residuals for samplers whose proposals move a
// few sources at a time (the BIRO loop of Sec. 2.3, Fig. 3, with Metropolis
// moves).
//
// Chain c keeps N_c = D - V_c resident in device memory, V_c the model
// visibilities of the chain's current sky model. A proposal that gives m of
// the chain's sources new parameters changes the model by
//   dV = V(new values) - V(current values) = V(new values, current values
//        with the Stokes vector negated),
// eqs. 1-2 being linear in the Stokes vector; so its chi^2 (eq. 7) is
//   sum w |V_c + dV - D|^2 = sum w |dV - N_c|^2,
// the fused predict + chi^2 of a 2m-source sky model against the "data" N_c.
// Accepting the proposal subtracts dV from N_c. A proposal then costs the
// predict of its 2m sources and one read of N_c and the weights, where a
// fresh evaluation predicts the whole sky model; HBM holds the chains'
// residuals (nchains x 32 B per visibility in FP32).
#include "rime_internal.cuh"
#include "rime_dev.cuh"
#include "rime_fused_common.cuh"

#include <algorithm>
#include <climits>
#include <type_traits>
#include <vector>

namespace rime {
namespace {

// N = D - V for every chain (V: one chain's predict, in `vis`)
template <typename T2>
__global__ void k_chain_init(long long n, int nchains, const T2 *data, const T2 *vis, T2 *N) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const T2 d = data[i], v = vis[i];
        const T2 r{d.x - v.x, d.y - v.y};
        for (int c = 0; c < nchains; c++) N[(long long)c * n + i] = r;
    }
}

// N -= dV
template <typename T2>
__global__ void k_chain_sub(long long n, T2 *N, const T2 *dv) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        T2 a = N[i];
        const T2 b = dv[i];
        a.x -= b.x;
        a.y -= b.y;
        N[i] = a;
    }
}

// the Stokes vectors of the staged "current" sources, negated: sources
// c * 2m + m .. c * 2m + 2m - 1 of each chain c
__global__ void k_negate_current(int nchains, int m, double *stokes) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nchains * m * 4) return;
    const int c = i / (4 * m), r = i - c * 4 * m;
    stokes[(long long)c * 8 * m + 4 * m + r] *= -1.0;
}

unsigned grid_for(long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 152LL * 16); }

constexpr int DTHREADS = 256;
constexpr int kPerThread = 8;   // visibilities per thread: fewer, longer-lived blocks
constexpr int kMaxList = 1000;   // chains per launch (kernel arguments stay under 4 KB)
struct ChainList {
    int n;
    int chain[kMaxList];
};

// Row p of baseline b in the canonical order (p < q, row-major): the largest
// p with first(p) = p na - p (p + 1) / 2 <= b, from the quadratic's root,
// corrected by one step either way against rounding.
// The root is taken in FP32 (the FP64 pipe runs at 1/64 of the FP32 rate;
// this runs once per visibility): its error only costs correction steps.
__device__ __forceinline__ void baseline_pq(int b, int na, int &p, int &q) {
    const float A = 2.0f * na - 1.0f;
    int r = (int)floorf((A - sqrtf(fmaxf(A * A - 8.0f * (float)b, 0.0f))) * 0.5f);
    r = max(0, min(r, na - 2));
    auto first = [&](int x) { return x * na - x * (x + 1) / 2; };
    while (r > 0 && first(r) > b) r--;
    while (r < na - 2 && first(r + 1) <= b) r++;
    p = r;
    q = b - first(r) + r + 1;
}

__device__ __forceinline__ float2 phase_t(const float2 *tau, long long di, const ChanF &ch) {
    return f32::phase_factor(tau[di], ch);
}
__device__ __forceinline__ double2 phase_t(const double *tau, long long di, const ChanD &ch) {
    const double ph = ch.nu * tau[di];
    const double r = ph - round_int_d(ph);
    double sn, cs;
    sincospi(2.0 * r, &sn, &cs);
    return make_double2(cs, sn);
}
__device__ __forceinline__ float shape_g(float e, float flag) {
    if (flag > 1.5f) {
        const float r = rsqrtf(1.0f + e);
        return r * r * r;
    }
    return exp2f(e);   // log2 units in FP32
}
__device__ __forceinline__ double shape_g(double e, double flag) {
    if (flag > 1.5) {
        const double r = rsqrt(1.0 + e);
        return r * r * r;
    }
    return exp(e);
}
__device__ __forceinline__ float spec_t(float alpha, const ChanF &ch) { return exp2f(2.0f * alpha * ch.hlr); }
__device__ __forceinline__ double spec_t(double alpha, const ChanD &ch) { return exp2(2.0 * alpha * ch.hlr); }

// The visibilities dV of the sources [m2 c, m2 (c + 1)) of the staged pair
// model (chain c's proposed values and its current values with negated
// Stokes vectors), one thread per (baseline, channel), channels fastest so
// that the residual rows are read in order; the few sources' factors are
// computed per thread (eqs. 1-4 as in the fused kernels).
//   CHI2: partials[c][t][block] = sum w |dV - N_c|^2 (eq. 7);
//   SUB:  N_c -= dV (the chain moves to its proposal).
template <typename T, bool SUB>
__global__ void __launch_bounds__(DTHREADS) k_chain_delta(const FusedParams P, const ChainList L, int m2, void *resid,
                                                         long long per_chain, double *partials) {
    using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    using Chan = typename std::conditional<sizeof(T) == 4, ChanF, ChanD>::type;
    using TauT = typename std::conditional<sizeof(T) == 4, float2, double>::type;
    __shared__ double red[32];
    // this block's sources staged in shared memory (every thread reads them):
    // delays and beam radii per (source, antenna), Stokes, shape coefficients
    // and spectral index per source
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TauT *sTau = reinterpret_cast<TauT *>(smem_raw);                       // [m2][na]
    T *sRho = reinterpret_cast<T *>(sTau + (size_t)m2 * P.na);               // [m2][na]
    T *sSrc = sRho + (size_t)m2 * P.na;                                      // [m2][9]: IQUV, shape, alpha
    T *sF = sSrc + (size_t)m2 * 9;                                           // [m2][nchan]: spectral x beam^2
    if (inputs_bad(P.status)) return;
    const int c = L.chain[blockIdx.z];
    const int t = blockIdx.y;
    const int na = P.na, nchan = P.nchan, nbl = (int)P.nbl;
    {
        const TauT *tau = reinterpret_cast<const TauT *>(P.tau);
        const T *rho = reinterpret_cast<const T *>(P.rho);
        for (int j = threadIdx.x; j < m2 * na; j += DTHREADS) {
            const int s = m2 * c + j / na, a = j - (j / na) * na;
            const long long d = ((long long)t * P.nsrc + s) * na + a;
            sTau[j] = tau[d];
            sRho[j] = rho[d];
        }
        for (int j = threadIdx.x; j < m2 * 9; j += DTHREADS) {
            const int s = m2 * c + j / 9, e = j - (j / 9) * 9;
            sSrc[j] = e < 4 ? reinterpret_cast<const T *>(P.stokes)[4 * (long long)s + e]
                    : e < 8 ? reinterpret_cast<const T *>(P.gauss)[4 * (long long)s + e - 4]
                            : reinterpret_cast<const T *>(P.alpha)[s];
        }
        if (!P.has_pointing) {
            // without pointing errors every antenna sees the same beam: the
            // spectral factor times E^2 per (source, channel)
            const Chan *chan = reinterpret_cast<const Chan *>(P.chan);
            for (int j = threadIdx.x; j < m2 * nchan; j += DTHREADS) {
                const int js = j / nchan, k = j - js * nchan, s = m2 * c + js;
                const Chan ch = chan[k];
                const T E = beam_E(ch.beam, ch.cnu * rho[((long long)t * P.nsrc + s) * na]);
                sF[j] = spec_t(reinterpret_cast<const T *>(P.alpha)[s], ch) * E * E;
            }
        }
        __syncthreads();
    }
    const unsigned nvis_t = (unsigned)nbl * (unsigned)nchan;   // < 2^31 (checked on the host)
    T chi = T(0);
    // each thread takes kPerThread visibilities, DTHREADS apart (coalesced)
    for (int it = 0; it < kPerThread; it++) {
    const unsigned i = (blockIdx.x * kPerThread + it) * DTHREADS + threadIdx.x;
    const bool act = i < nvis_t;
    if (act) {
        const int b = (int)(i / (unsigned)nchan), k = (int)(i - (unsigned)b * (unsigned)nchan);
        int p, q;
        baseline_pq(b, na, p, q);
        const Chan ch = reinterpret_cast<const Chan *>(P.chan)[k];
        const bool pointing = P.has_pointing != 0;
        T du, dv;
        if constexpr (sizeof(T) == 4) {   // FP32 inputs are FP32 values: one rounding in the difference
            const float4 xp = P.uvw_f[(long long)t * na + p], xq = P.uvw_f[(long long)t * na + q];
            du = xp.x - xq.x;
            dv = xp.y - xq.y;
        } else {
            const double *up = P.uvw + 3 * ((long long)t * na + p), *uq = P.uvw + 3 * ((long long)t * na + q);
            du = up[0] - uq[0];
            dv = up[1] - uq[1];
        }
        const T nu2 = (T)ch.nu2;
        const T du2 = du * du * nu2, dudv = du * dv * nu2, dv2 = dv * dv * nu2;
        T acc[8];
#pragma unroll
        for (int x = 0; x < 8; x++) acc[x] = T(0);
        for (int j = 0; j < m2; j++) {
            T2 ap = phase_t(sTau + j * na, p, ch), aq = phase_t(sTau + j * na, q, ch);
            const T *src = sSrc + 9 * j;
            T f;
            if (pointing) {
                const T Ep = beam_E(ch.beam, ch.cnu * sRho[j * na + p]), Eq = beam_E(ch.beam, ch.cnu * sRho[j * na + q]);
                f = spec_t(src[8], ch) * Ep * Eq;
            } else {
                f = sF[j * nchan + k];
            }
            T zr = ap.x * aq.x + ap.y * aq.y, zi = ap.y * aq.x - ap.x * aq.y;
            const T *g = src + 4;
            if (g[3] != T(0)) {
                const T gg = shape_g(g[0] * du2 + g[1] * dudv + g[2] * dv2, g[3]);
                zr *= gg;
                zi *= gg;
            }
            zr *= f;
            zi *= f;
            const T *x = src;
#pragma unroll
            for (int X = 0; X < 4; X++) {
                acc[2 * X] += zr * x[X];
                acc[2 * X + 1] += zi * x[X];
            }
        }
        T2 Sm[4];
        Sm[0] = T2{acc[0] + acc[2], acc[1] + acc[3]};   // I + Q   (eq. 2)
        Sm[1] = T2{acc[4] - acc[7], acc[5] + acc[6]};   // U + iV
        Sm[2] = T2{acc[4] + acc[7], acc[5] - acc[6]};   // U - iV
        Sm[3] = T2{acc[0] - acc[2], acc[1] - acc[3]};   // I - Q
        const T2 one{T(1), T(0)}, zero{T(0), T(0)};
        const T2 I2[4] = {one, zero, zero, one};
        const T2 *gains = reinterpret_cast<const T2 *>(P.gains);
        T2 gp[4], gq[4], V[4], tmp[4], gqh[4];
#pragma unroll
        for (int x = 0; x < 4; x++) {
            gp[x] = P.has_gains ? gains[4 * (((long long)t * na + p) * nchan + k) + x] : I2[x];
            gq[x] = P.has_gains ? gains[4 * (((long long)t * na + q) * nchan + k) + x] : I2[x];
        }
        mmul(gp, Sm, tmp);      // eq. 1
        mherm(gq, gqh);
        mmul(tmp, gqh, V);
        const long long row = ((long long)t * nbl + b) * nchan + k;
        T2 *N = reinterpret_cast<T2 *>(resid) + (long long)c * per_chain + 4 * row;
        if constexpr (SUB) {
#pragma unroll
            for (int x = 0; x < 4; x++) {
                T2 v = N[x];
                v.x -= V[x].x;
                v.y -= V[x].y;
                N[x] = v;
            }
        } else {
            T r2 = T(0);
#pragma unroll
            for (int x = 0; x < 4; x++) {
                const T2 n = N[x];
                const T dr = V[x].x - n.x, di = V[x].y - n.y;
                r2 += dr * dr + di * di;
            }
            const T w = P.has_weight ? reinterpret_cast<const T *>(P.weight)[row] : T(1);
            chi += w * r2;
        }
    }
    }
    if constexpr (!SUB) {
        // warp sums in the compute precision (positive terms; FP64 operations
        // run at 1/64 of the FP32 rate and one per visibility dominated this
        // kernel), the block's eight warp sums in FP64 in fixed order
        T v = chi;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int wi = 0; wi < DTHREADS / 32; wi++) tot += red[wi];
            partials[((long long)c * gridDim.y + t) * gridDim.x + blockIdx.x] = tot;
        }
    }
}

// blocks per (chain, timestep)
long long chain_nbx(const rime_ctx *c) {
    const long long per_block = (long long)DTHREADS * kPerThread;
    return ((long long)c->nbl * c->dims.nchan + per_block - 1) / per_block;
}

// shared memory of k_chain_delta for 2m = m2 staged sources
constexpr size_t kMaxChainSmem = 96 * 1024;
size_t chain_smem(const rime_ctx *c, int m2) {
    const size_t ts = c->tsize();
    const size_t taus = ts == 4 ? sizeof(float2) : sizeof(double);
    return (size_t)m2 * c->dims.na * (taus + ts) + (size_t)m2 * 9 * ts + (size_t)m2 * c->dims.nchan * ts;
}

template <bool SUB>
cudaError_t launch_delta(rime_ctx *c, const ChainList &L, int m2, double *partials) {
    if (L.n == 0) return cudaSuccess;
    FusedParams P{};
    fill_fused_params(c, P, nullptr, nullptr, nullptr, nullptr);
    const long long nvis_t = (long long)c->nbl * c->dims.nchan;
    const dim3 grid((unsigned)chain_nbx(c), (unsigned)c->dims.ntime, (unsigned)L.n);
    const long long per_chain = (long long)c->dims.ntime * nvis_t * 4;
    const size_t smem = chain_smem(c, m2);
    if (smem > kMaxChainSmem) return cudaErrorInvalidValue;   // rime_chains_propose checks it first
    if (c->dims.precision == RIME_FP64) {
        auto k = k_chain_delta<double, SUB>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxChainSmem);
        if (e != cudaSuccess) return e;
        k<<<grid, DTHREADS, smem, c->stream>>>(P, L, m2, c->d_chainN, per_chain, partials);
    } else {
        auto k = k_chain_delta<float, SUB>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxChainSmem);
        if (e != cudaSuccess) return e;
        k<<<grid, DTHREADS, smem, c->stream>>>(P, L, m2, c->d_chainN, per_chain, partials);
    }
    return cudaGetLastError();
}

}  // namespace
}  // namespace rime

using namespace rime;

#define CKC2(c, call, what)                                        \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail_ctx(c, e_, what);  \
    } while (0)

extern "C" {

rime_status rime_chains_init(rime_ctx *c, int32_t nchains) {
    if (!c) return fail_ctx(nullptr, RIME_E_INVALID, "ctx is NULL");
    if (nchains < 1) return fail_ctx(c, RIME_E_INVALID, "nchains must be >= 1");
    if (!c->sources_set) return fail_ctx(c, RIME_E_STATE, "rime_set_sources has not been called");
    if (!c->has_data) return fail_ctx(c, RIME_E_STATE, "no observed data (rime_set_data)");
    if (c->time_varying) return fail_ctx(c, RIME_E_INVALID, "chains need static brightness (time_varying = 0)");
    if (c->tc_mode != RIME_TC_OFF) return fail_ctx(c, RIME_E_STATE, "chains use the direct kernels (RIME_TC_OFF)");
    const long long n = (long long)c->dims.ntime * c->nbl * c->dims.nchan * 4;   // complex values per chain
    const size_t csz = 2 * c->tsize();
    if ((unsigned long long)n * csz > (unsigned long long)LLONG_MAX / (unsigned long long)nchains)
        return fail_ctx(c, RIME_E_INVALID, "nchains too large");
    void *old[] = {c->d_chainN, c->d_chain_scratch, c->d_chain_part};
    for (void *p : old)
        if (p) cudaFree(p);
    c->d_chainN = c->d_chain_scratch = nullptr;
    c->d_chain_part = nullptr;
    c->chains_n = 0;
    const long long nbx = chain_nbx(c);
    Alloc alloc{c};
    CKC2(c, alloc(&c->d_chainN, (size_t)nchains * n * csz), "allocating the chains' residuals");
    CKC2(c, alloc(&c->d_chain_scratch, (size_t)n * csz), "allocating the chains' scratch");
    CKC2(c, alloc((void **)&c->d_chain_part, (size_t)nchains * c->dims.ntime * nbx * sizeof(double)),
         "allocating the chains' partials");
    CKC2(c, launch_fused_auto(c, c->d_chain_scratch, nullptr, false), "predict kernel");
    if (c->dims.precision == RIME_FP64)
        k_chain_init<double2><<<grid_for(n), 256, 0, c->stream>>>(n, nchains, (const double2 *)c->d_data,
                                                                 (const double2 *)c->d_chain_scratch,
                                                                 (double2 *)c->d_chainN);
    else
        k_chain_init<float2><<<grid_for(n), 256, 0, c->stream>>>(n, nchains, (const float2 *)c->d_data,
                                                                (const float2 *)c->d_chain_scratch,
                                                                (float2 *)c->d_chainN);
    CKC2(c, cudaGetLastError(), "chain residuals");
    c->chains_n = nchains;
    c->chains_move = 0;
    return RIME_OK;
}

rime_status rime_chains_propose(rime_ctx *c, int32_t nmove, const rime_sources *proposed,
                                const rime_sources *current, double *chi2_dev) {
    if (!c) return fail_ctx(nullptr, RIME_E_INVALID, "ctx is NULL");
    if (c->chains_n < 1) return fail_ctx(c, RIME_E_STATE, "rime_chains_init has not been called");
    if (nmove < 1) return fail_ctx(c, RIME_E_INVALID, "nmove must be >= 1");
    if (!proposed || !current || !chi2_dev) return fail_ctx(c, RIME_E_INVALID, "proposed, current or chi2_dev is NULL");
    const int K = c->chains_n;
    const long long nm = (long long)K * nmove;
    if (proposed->nsrc != nm || current->nsrc != nm)
        return fail_ctx(c, RIME_E_INVALID, "proposed and current must hold nchains * nmove sources");
    if (proposed->time_varying || current->time_varying)
        return fail_ctx(c, RIME_E_INVALID, "chains need static brightness (time_varying = 0)");
    const rime_sources *both[2] = {proposed, current};
    for (const rime_sources *s : both)
        if (!s->lm || !s->stokes || !s->alpha) return fail_ctx(c, RIME_E_INVALID, "lm, stokes and alpha must not be NULL");
    if ((proposed->shape == nullptr) != (current->shape == nullptr) ||
        (proposed->kind == nullptr) != (current->kind == nullptr))
        return fail_ctx(c, RIME_E_INVALID, "proposed and current must both give (or both omit) shape and kind");
    if (2 * nm > INT_MAX) return fail_ctx(c, RIME_E_INVALID, "too many sources");
    if ((long long)c->nbl * c->dims.nchan >= (1LL << 31) - (long long)DTHREADS * kPerThread)
        return fail_ctx(c, RIME_E_INVALID, "nbl * nchan too large for the chains");
    if (chain_smem(c, 2 * nmove) > kMaxChainSmem)
        return fail_ctx(c, RIME_E_INVALID, "nmove too large for this array (the moved sources' per-antenna "
                                           "delays must fit in shared memory)");
    // stage the pair sky model: chain c's sources c 2m .. c 2m + m - 1 are
    // its proposed values, c 2m + m .. c 2m + 2m - 1 its current values
    const size_t ns = (size_t)2 * nm;
    if (ns > c->pair_cap) {
        if (c->d_pair) cudaFree(c->d_pair);
        if (c->d_pair_kind) cudaFree(c->d_pair_kind);
        c->d_pair = nullptr;
        c->d_pair_kind = nullptr;
        c->pair_cap = 0;
        Alloc alloc{c};
        CKC2(c, alloc((void **)&c->d_pair, ns * 10 * sizeof(double)), "allocating the proposal model");
        CKC2(c, alloc((void **)&c->d_pair_kind, ns * sizeof(int32_t)), "allocating the proposal model");
        c->pair_cap = ns;
    }
    double *lm = c->d_pair, *st = lm + 2 * ns, *al = st + 4 * ns, *sh = al + ns;
    const size_t m = (size_t)nmove;
    struct Field {
        double *dst;
        const void *src[2];
        size_t bytes;   // per source
    } fields[] = {{lm, {proposed->lm, current->lm}, 2 * sizeof(double)},
                  {st, {proposed->stokes, current->stokes}, 4 * sizeof(double)},
                  {al, {proposed->alpha, current->alpha}, sizeof(double)},
                  {sh, {proposed->shape, current->shape}, 3 * sizeof(double)}};
    for (const Field &f : fields)
        for (int h = 0; h < 2; h++) {
            if (!f.src[h]) continue;
            char *dst = reinterpret_cast<char *>(f.dst) + h * m * f.bytes;
            CKC2(c, cudaMemcpy2DAsync(dst, 2 * m * f.bytes, f.src[h], m * f.bytes, m * f.bytes, K, cudaMemcpyDefault,
                                      c->stream),
                 "staging the proposal model");
        }
    if (proposed->kind)
        for (int h = 0; h < 2; h++)
            CKC2(c, cudaMemcpy2DAsync(c->d_pair_kind + h * m, 2 * m * sizeof(int32_t), h ? current->kind : proposed->kind,
                                      m * sizeof(int32_t), m * sizeof(int32_t), K, cudaMemcpyDefault, c->stream),
                 "staging the proposal model");
    k_negate_current<<<(unsigned)((nm * 4 + 255) / 256), 256, 0, c->stream>>>(K, nmove, st);
    CKC2(c, cudaGetLastError(), "staging the proposal model");
    rime_sources pair{(int32_t)ns, 0, lm, st, al, proposed->shape ? sh : nullptr,
                      proposed->kind ? c->d_pair_kind : nullptr};
    rime_status s = rime_set_sources(c, &pair);
    if (s != RIME_OK) return s;
    const size_t csz = 2 * c->tsize();
    const long long per_chain = (long long)c->dims.ntime * chain_nbx(c);
    for (int k0 = 0; k0 < K; k0 += kMaxList) {
        ChainList L;
        L.n = std::min(kMaxList, K - k0);
        for (int j = 0; j < L.n; j++) L.chain[j] = k0 + j;
        CKC2(c, launch_delta<false>(c, L, 2 * nmove, c->d_chain_part), "proposal chi2 kernel");
    }
    CKC2(c, launch_set_sums(c, K, (int)per_chain, c->d_chain_part, chi2_dev), "proposal chi2 sums");
    c->chains_move = nmove;
    return RIME_OK;
}

rime_status rime_chains_accept(rime_ctx *c, const int32_t *accept) {
    if (!c) return fail_ctx(nullptr, RIME_E_INVALID, "ctx is NULL");
    if (c->chains_n < 1 || c->chains_move < 1)
        return fail_ctx(c, RIME_E_STATE, "no proposal to accept (rime_chains_propose)");
    if (!accept) return fail_ctx(c, RIME_E_INVALID, "accept is NULL");
    const int m = c->chains_move;
    ChainList L;
    L.n = 0;
    for (int k = 0; k < c->chains_n; k++) {
        if (!accept[k]) continue;
        L.chain[L.n++] = k;
        if (L.n == kMaxList) {
            CKC2(c, launch_delta<true>(c, L, 2 * m, nullptr), "chain residual update");
            L.n = 0;
        }
    }
    CKC2(c, launch_delta<true>(c, L, 2 * m, nullptr), "chain residual update");
    return RIME_OK;
}

}  // extern "C"
