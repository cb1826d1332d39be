// rime_grad.cu -- the adjoint of the fused chi^2: d chi^2 / d(source
// parameters) and d chi^2 / d(gains), recomputing K and E instead of storing
// them.
//
// For a visibility with residual R = V - D (eq. 7) the fused kernel in
// gradient mode (rime_fused.cu) forms Sh = 2 w G_p^H R G_q and the four
// Stokes projections Y_X of it, so that a source with coherency c B0 (eq. 2,
// c = f g E_p E_q K_p K_q^*) changes chi^2 by Re(dc sum_X X Y_X). It also
// accumulates the gains gradient. The kernel here then runs one thread per
// (source, baseline group) over the baselines of a unit, with the Y_X of each
// baseline broadcast from shared memory, and accumulates per source:
//   a_X  = sum Re(g z Y_X)                   (Stokes; z = A_p conj(A_q))
//   b_u, b_v, b_w = sum Im(g z beta) du, dv, dw   (phase of eq. 3, beta = sum_X X Y_X)
//   c_uu, c_uv, c_vv = sum Re(g z beta) du^2, du dv, dv^2   (Gaussian shape)
//   e_l, e_m = sum Re(g z beta) (dlnE_p + dlnE_q)             (beam with pointing errors)
// and turns them into d/d(l, m, I, Q, U, V, alpha, major, minor, pa) with the
// channel's and the source's factors. One partial per (t, k, unit) and
// source is written; k_grad_reduce sums them in a fixed order.
#include "rime_internal.cuh"

#include <algorithm>
#include <type_traits>
#include <vector>

namespace rime {
void build_units(int na, int precision, std::vector<Unit> &units, std::vector<Tile> &tiles);

namespace {

constexpr int GTHREADS = 256;
constexpr int BLC = 128;        // baselines staged per step
constexpr int GNLOC = 96;       // antennas of a unit, at most
constexpr int NACC = 12;
constexpr int NGRAD = 10;

template <typename T> struct GCfg;
template <> struct GCfg<float> {
    static constexpr int SG = 64;                 // sources per block
    using T2 = float2;
    using Chan = ChanF;
};
template <> struct GCfg<double> {
    static constexpr int SG = 32;
    using T2 = double2;
    using Chan = ChanD;
};

struct GradParams {
    int na, ntime, nchan, nsrc, nunits, nsch;
    long long nbl;
    int has_pointing;
    double ref_freq_hz;
    const Unit *units;
    const uint16_t *bls;
    const void *chan;
    const double *uvw;
    const double *pointing;     // [ntime][na][2] or null
    const void *tau, *rho;
    const void *stokes, *gauss, *alpha, *extra;
    const void *yin;
    double *partials;
    const DevStatus *status;
};

__device__ __forceinline__ float round_i(float x) {
    const float M = 12582912.0f;
    return __fsub_rn(__fadd_rn(x, M), M);
}
__device__ __forceinline__ double round_i(double x) {
    const double M = 6755399441055744.0;
    return __dsub_rn(__dadd_rn(x, M), M);
}

// K = exp(2 pi i nu tau) (eq. 3), FP32: double-float delay, exact reduction
__device__ __forceinline__ float2 phase(const float2 *tau, long long i, const ChanF &ch) {
    float2 tv = tau[i];
    float p = ch.nu_hi * tv.x;
    float e = fmaf(ch.nu_hi, tv.x, -p);
    float r = p - round_i(p);
    float f = r + (e + fmaf(ch.nu_hi, tv.y, ch.nu_lo * tv.x));
    float sn, cs;
    sincospif(2.0f * f, &sn, &cs);
    return make_float2(cs, sn);
}
__device__ __forceinline__ double2 phase(const double *tau, long long i, const ChanD &ch) {
    double ph = ch.nu * tau[i];
    double r = ph - round_i(ph);
    double sn, cs;
    sincospi(2.0 * r, &sn, &cs);
    return make_double2(cs, sn);
}
__device__ __forceinline__ float gexp(float e) { return exp2f(e); }     // log2 units (FP32 coefficients)
__device__ __forceinline__ double gexp(double e) { return exp(e); }     // natural units (FP64 coefficients)

template <typename T>
__device__ __forceinline__ T nu_of(const typename GCfg<T>::Chan &ch);
template <> __device__ __forceinline__ float nu_of<float>(const ChanF &ch) { return ch.nu_hi + ch.nu_lo; }
template <> __device__ __forceinline__ double nu_of<double>(const ChanD &ch) { return ch.nu; }

// Beam E = cos^3(x), x = C nu rho (eq. 4), and dlnE/dx-related factor:
// returns E and t3 = -3 tan(x) / x (so dlnE/dl = t3 cnu^2 (l - dl)); both 0
// past the first null.
template <typename T>
__device__ __forceinline__ void beam_d(T cnu, T rho, T &E, T &t3) {
    T x = cnu * rho;
    if (x >= T(1.5707963267948966)) {
        E = 0;
        t3 = 0;
        return;
    }
    T sn, cs;
    if (sizeof(T) == 4) {
        float s_, c_;
        sincosf((float)x, &s_, &c_);
        sn = s_;
        cs = c_;
    } else {
        double s_, c_;
        sincos((double)x, &s_, &c_);
        sn = (T)s_;
        cs = (T)c_;
    }
    E = cs * cs * cs;
    T tx = (x < T(1e-4)) ? T(1) + x * x / T(3) : sn / (cs * x);   // tan(x) / x
    t3 = T(-3) * tx;
}

template <typename T>
__global__ void __launch_bounds__(GTHREADS) k_grad_src(const GradParams P) {
    using C = GCfg<T>;
    using T2 = typename C::T2;
    using Chan = typename C::Chan;
    constexpr int SG = C::SG, NG = GTHREADS / SG;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *sA = reinterpret_cast<T2 *>(smem_raw);                  // [GNLOC][SG]
    T2 *sY = sA + GNLOC * SG;                                    // [BLC][4]
    T *sB = reinterpret_cast<T *>(sY + BLC * 4);                // [BLC][4]: du, dv, dw, (p | q << 8)
    T *sRed = sB + BLC * 4;                                      // [NG][SG][NACC]
    T2 *sE = reinterpret_cast<T2 *>(sRed + NG * SG * NACC);      // [GNLOC][SG] dlnE/dl, dlnE/dm (pointing)

    if (inputs_bad(P.status)) return;
    const int tid = threadIdx.x;
    const int sl = tid % SG, grp = tid / SG;
    int bid = blockIdx.x;
    const int sch = bid % P.nsch;
    bid /= P.nsch;
    const int u = bid % P.nunits;
    bid /= P.nunits;
    const int k = bid % P.nchan;
    const int t = bid / P.nchan;
    const Unit U = P.units[u];
    const Chan ch = reinterpret_cast<const Chan *>(P.chan)[k];
    const int s = sch * SG + sl;
    const bool sact = s < P.nsrc;
    const int sidx = sact ? s : 0;
    const int nloc = U.diag ? U.nr : U.nr + U.nc;
    const bool pointing = P.has_pointing != 0;
    const T *extra = reinterpret_cast<const T *>(P.extra) + 8 * sidx;
    const T l = extra[0], m = extra[1], l_n = extra[2], m_n = extra[3];

    // ---- stage A (= K, or E K with pointing errors) for (antenna, source) ----
    for (int i = tid; i < nloc * SG; i += GTHREADS) {
        const int a = i / SG, ss = i - a * SG;
        const int src = min(sch * SG + ss, P.nsrc - 1);
        const int ant = a < U.nr ? U.r0 + a : U.c0 + (a - U.nr);
        const long long di = ((long long)t * P.nsrc + src) * P.na + ant;
        using TauT = typename std::conditional<sizeof(T) == 4, float2, double>::type;
        T2 v = phase(reinterpret_cast<const TauT *>(P.tau), di, ch);
        if (pointing) {
            // A = E K; dlnE/dl = t3 cnu^2 (l - dl_ta), dlnE/dm likewise (eq. 4)
            const T rho = reinterpret_cast<const T *>(P.rho)[di];
            const T *ex = reinterpret_cast<const T *>(P.extra) + 8 * src;
            const double *pt = P.pointing + 2 * ((long long)t * P.na + ant);
            T E, t3;
            beam_d<T>(ch.cnu, rho, E, t3);
            v.x *= E;
            v.y *= E;
            T2 d;
            d.x = t3 * ch.cnu * ch.cnu * (ex[0] - (T)pt[0]);
            d.y = t3 * ch.cnu * ch.cnu * (ex[1] - (T)pt[1]);
            sE[a * SG + ss] = d;
        }
        sA[a * SG + ss] = v;
    }

    // ---- per-source constants of this thread ----
    const T *st = reinterpret_cast<const T *>(P.stokes) + 4 * sidx;
    const T sI = st[0], sQ = st[1], sU = st[2], sV = st[3];
    const T *gq = reinterpret_cast<const T *>(P.gauss) + 4 * sidx;
    const bool is_gauss = gq[3] != T(0);
    const T gA = gq[0] * ch.nu2, gB = gq[1] * ch.nu2, gC = gq[2] * ch.nu2;

    T acc[NACC];
#pragma unroll
    for (int i = 0; i < NACC; i++) acc[i] = T(0);

    const uint16_t *bls = P.bls + U.tile0;
    const int nb = U.nbody;
    const T2 *yin = reinterpret_cast<const T2 *>(P.yin);
    for (int b0 = 0; b0 < nb; b0 += BLC) {
        const int cnt = min(BLC, nb - b0);
        __syncthreads();   // previous step done with sY / sB (and sA staged on the first)
        for (int i = tid; i < cnt; i += GTHREADS) {
            const uint16_t e = bls[b0 + i];
            const int pl = e & 0xff, ql = e >> 8;
            const int p = U.r0 + pl, q = U.c0 + ql;
            const long long bl = (long long)p * P.na - (long long)p * (p + 1) / 2 + (q - p - 1);
            const long long row = ((long long)t * P.nbl + bl) * P.nchan + k;
#pragma unroll
            for (int c = 0; c < 4; c++) sY[4 * i + c] = yin[4 * row + c];
            const double *xp = P.uvw + 3 * ((long long)t * P.na + p);
            const double *xq = P.uvw + 3 * ((long long)t * P.na + q);
            sB[4 * i + 0] = (T)(xp[0] - xq[0]);
            sB[4 * i + 1] = (T)(xp[1] - xq[1]);
            sB[4 * i + 2] = (T)(xp[2] - xq[2]);
            const int la = pl, lb = U.diag ? ql : U.nr + ql;
            sB[4 * i + 3] = (T)(la | (lb << 8));
        }
        __syncthreads();
        for (int i = grp; i < cnt; i += NG) {
            const T du = sB[4 * i], dv = sB[4 * i + 1], dw = sB[4 * i + 2];
            const int pq = (int)sB[4 * i + 3];
            const int la = pq & 0xff, lb = pq >> 8;
            const T2 ap = sA[la * SG + sl], aq = sA[lb * SG + sl];
            T zr = ap.x * aq.x + ap.y * aq.y;   // z = A_p conj(A_q)
            T zi = ap.y * aq.x - ap.x * aq.y;
            if (is_gauss) {
                const T e = gA * du * du + gB * du * dv + gC * dv * dv;
                const T g = gexp(e);
                zr *= g;
                zi *= g;
            }
            const T2 y0 = sY[4 * i], y1 = sY[4 * i + 1], y2 = sY[4 * i + 2], y3 = sY[4 * i + 3];
            acc[0] += zr * y0.x - zi * y0.y;
            acc[1] += zr * y1.x - zi * y1.y;
            acc[2] += zr * y2.x - zi * y2.y;
            acc[3] += zr * y3.x - zi * y3.y;
            const T br = sI * y0.x + sQ * y1.x + sU * y2.x + sV * y3.x;
            const T bi = sI * y0.y + sQ * y1.y + sU * y2.y + sV * y3.y;
            const T re = zr * br - zi * bi, im = zr * bi + zi * br;   // z beta
            acc[4] += im * du;
            acc[5] += im * dv;
            acc[6] += im * dw;
            if (is_gauss) {
                acc[7] += re * du * du;
                acc[8] += re * du * dv;
                acc[9] += re * dv * dv;
            }
            if (pointing) {
                const T2 ep = sE[la * SG + sl], eq = sE[lb * SG + sl];
                acc[10] += re * (ep.x + eq.x);
                acc[11] += re * (ep.y + eq.y);
            }
        }
    }
    // ---- combine the baseline groups, then the channel and source factors ----
#pragma unroll
    for (int i = 0; i < NACC; i++) sRed[(grp * SG + sl) * NACC + i] = acc[i];
    __syncthreads();
    if (grp == 0 && sact) {
        double a[NACC];
        for (int i = 0; i < NACC; i++) {
            double v = 0.0;
            for (int g = 0; g < NG; g++) v += (double)sRed[(g * SG + sl) * NACC + i];
            a[i] = v;
        }
        const double nu = (double)nu_of<T>(ch);
        // spectral factor f = (nu/nu_ref)^alpha and, without pointing errors,
        // the beam E_s^2 shared by both antennas
        const double alpha = (double)reinterpret_cast<const T *>(P.alpha)[s];
        const double lnr = log(nu / P.ref_freq_hz);
        double w = exp(alpha * lnr);
        double dlnE2_l = 0.0, dlnE2_m = 0.0;
        if (!pointing) {
            const T rho = reinterpret_cast<const T *>(P.rho)[((long long)t * P.nsrc + s) * P.na];
            T E, t3;
            beam_d<T>(ch.cnu, rho, E, t3);
            w *= (double)E * (double)E;
            const double cnu2 = (double)ch.cnu * (double)ch.cnu;
            dlnE2_l = 2.0 * (double)t3 * cnu2 * (double)l;
            dlnE2_m = 2.0 * (double)t3 * cnu2 * (double)m;
        }
        const double aR = (double)sI * a[0] + (double)sQ * a[1] + (double)sU * a[2] + (double)sV * a[3];
        const double k2pi = 2.0 * 3.141592653589793 * nu / 299792458.0;
        double out[NGRAD];
        out[0] = w * (-k2pi * (a[4] - (double)l_n * a[6]) + (pointing ? a[10] : aR * dlnE2_l));
        out[1] = w * (-k2pi * (a[5] - (double)m_n * a[6]) + (pointing ? a[11] : aR * dlnE2_m));
        out[2] = w * a[0];
        out[3] = w * a[1];
        out[4] = w * a[2];
        out[5] = w * a[3];
        out[6] = w * aR * lnr;
        out[7] = out[8] = out[9] = 0.0;
        if (is_gauss) {
            // ln g = nu^2 (A du^2 + B du dv + C dv^2) with
            // A = -K (maj^2 sp^2 + min^2 cp^2), B = -K 2 sp cp (maj^2 - min^2),
            // C = -K (maj^2 cp^2 + min^2 sp^2), K = pi^2 / (4 ln 2 c^2)
            const double K = kGaussK / (kCLight * kCLight) * nu * nu;
            const double maj = (double)extra[4], mn = (double)extra[5], sp = (double)extra[6], cp = (double)extra[7];
            const double dd = maj * maj - mn * mn;
            const double Au = a[7], Auv = a[8], Av = a[9];
            out[7] = w * -K * (2 * maj * sp * sp * Au + 4 * maj * sp * cp * Auv + 2 * maj * cp * cp * Av);
            out[8] = w * -K * (2 * mn * cp * cp * Au - 4 * mn * sp * cp * Auv + 2 * mn * sp * sp * Av);
            out[9] = w * -K * (2 * sp * cp * dd * Au + 2 * dd * (cp * cp - sp * sp) * Auv - 2 * sp * cp * dd * Av);
        }
        const long long prow = (((long long)t * P.nchan + k) * P.nunits + u);
        double *o = P.partials + (prow * P.nsrc + s) * NGRAD;
#pragma unroll
        for (int i = 0; i < NGRAD; i++) o[i] = out[i];
    }
}

// grad_src[s][j] = sum over (t, k, unit) of the partials, in index order.
__global__ void k_grad_reduce(long long nrows, int nsrc, const double *partials, double *grad_src,
                              const DevStatus *status) {
    if (inputs_bad(status)) return;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = (long long)nsrc * NGRAD;
    if (i >= n) return;
    double acc = 0.0;
    for (long long r = 0; r < nrows; r++) acc += partials[r * n + i];
    grad_src[i] = acc;
}

}  // namespace

// Gradient work units: the FP32 forward decomposition, with each unit's
// baselines listed as (p | q << 8) local antenna pairs.
static cudaError_t ensure_grad_units(rime_ctx *c) {
    if (c->d_gunits) return cudaSuccess;
    std::vector<Unit> units;
    std::vector<Tile> tiles;
    build_units(c->dims.na, RIME_FP32, units, tiles);
    std::vector<uint16_t> bls;
    for (Unit &u : units) {
        u.tile0 = (int)bls.size();
        for (int p = 0; p < u.nr; p++)
            for (int q = 0; q < (u.diag ? u.nr : u.nc); q++)
                if (!u.diag || p < q) bls.push_back((uint16_t)(p | (q << 8)));
        u.nbody = (int)bls.size() - u.tile0;
        u.nhead = 0;
    }
    cudaError_t e = cudaMalloc(&c->d_gunits, units.size() * sizeof(Unit));
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&c->d_gbl, std::max<size_t>(bls.size(), 1) * sizeof(uint16_t));
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(c->d_gunits, units.data(), units.size() * sizeof(Unit), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(c->d_gbl, bls.data(), bls.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return e;
    c->ngunits = (int)units.size();
    return cudaStreamSynchronize(c->stream);   // host vectors go out of scope
}

cudaError_t launch_grad_src(rime_ctx *c, double *grad_src) {
    if (c->nsrc == 0) return cudaSuccess;
    cudaError_t e = ensure_grad_units(c);
    if (e != cudaSuccess) return e;
    const bool f64 = c->dims.precision == RIME_FP64;
    const int SG = f64 ? GCfg<double>::SG : GCfg<float>::SG;
    const int nsch = (c->nsrc + SG - 1) / SG;
    const long long nrows = (long long)c->dims.ntime * c->dims.nchan * c->ngunits;
    const size_t need = (size_t)nrows * c->nsrc * NGRAD;
    if (need > c->gpart_cap) {
        if (c->d_gpart) cudaFree(c->d_gpart);
        c->d_gpart = nullptr;
        c->gpart_cap = 0;
        e = cudaMalloc((void **)&c->d_gpart, need * sizeof(double));
        if (e != cudaSuccess) return e;
        c->gpart_cap = need;
    }
    GradParams P{};
    P.na = c->dims.na;
    P.ntime = c->dims.ntime;
    P.nchan = c->dims.nchan;
    P.nsrc = c->nsrc;
    P.nunits = c->ngunits;
    P.nsch = nsch;
    P.nbl = c->nbl;
    P.has_pointing = c->has_pointing;
    P.ref_freq_hz = c->dims.ref_freq_hz;
    P.units = c->d_gunits;
    P.bls = c->d_gbl;
    P.chan = c->d_chan;
    P.uvw = c->d_uvw;
    P.pointing = c->has_pointing ? c->d_pointing : nullptr;
    P.tau = c->d_tau;
    P.rho = c->d_rho;
    P.stokes = c->d_stokes;
    P.gauss = c->d_gauss;
    P.alpha = c->d_alpha;
    P.extra = c->d_src_extra;
    P.yin = c->d_yadj;
    P.partials = c->d_gpart;
    P.status = c->d_status;
    const long long blocks = nrows * nsch;
    const size_t ts = f64 ? 8 : 4;
    const size_t t2 = 2 * ts;
    size_t smem = (size_t)GNLOC * SG * t2 + (size_t)BLC * 4 * t2 + (size_t)BLC * 4 * ts +
                  (size_t)(GTHREADS / SG) * SG * NACC * ts;
    if (c->has_pointing) smem += (size_t)GNLOC * SG * t2;
    if (f64) {
        e = cudaFuncSetAttribute(k_grad_src<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_grad_src<double><<<(unsigned)blocks, GTHREADS, smem, c->stream>>>(P);
    } else {
        e = cudaFuncSetAttribute(k_grad_src<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_grad_src<float><<<(unsigned)blocks, GTHREADS, smem, c->stream>>>(P);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long n = (long long)c->nsrc * NGRAD;
    k_grad_reduce<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(nrows, c->nsrc, c->d_gpart, grad_src,
                                                                     c->d_status);
    return cudaGetLastError();
}

}  // namespace rime
