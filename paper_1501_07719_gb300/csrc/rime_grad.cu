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
// channel's and the source's factors. A block loops over a group of
// channels (the delays and the baseline table are staged once); one partial
// per (t, channel group, unit) and source is written and k_colsum sums them
// in a fixed order.
#include "rime_internal.cuh"
#include "rime_beam.cuh"
#include "rime_fused_common.cuh"

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
constexpr int NBMAX = 2048;     // baselines of a unit, at most (64 x 32 off-diagonal)

template <typename T> struct GCfg;
template <> struct GCfg<float> {
    static constexpr int SG = 32;                 // sources per block
    using T2 = float2;
    using Chan = ChanF;
};
template <> struct GCfg<double> {
    static constexpr int SG = 16;
    using T2 = double2;
    using Chan = ChanD;
};

struct GradParams {
    int na, ntime, nchan, nsrc, nunits, nsch;
    int chan_group, ncg;          // channels per block, channel groups
    long long nbl;
    int has_pointing;
    int has_disk;                // the sky model may hold exponential disks (a kind array was given)
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

__device__ __forceinline__ void cp16(void *smem, const void *gmem) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

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
template <typename T> __device__ __forceinline__ T int_bits(int v);
template <> __device__ __forceinline__ float int_bits<float>(int v) { return __int_as_float(v); }
template <> __device__ __forceinline__ double int_bits<double>(int v) { return __longlong_as_double((long long)v); }
__device__ __forceinline__ int bits_int(float x) { return __float_as_int(x); }
__device__ __forceinline__ int bits_int(double x) { return (int)__double_as_longlong(x); }
__device__ __forceinline__ float gexp(float e) { return exp2f(e); }     // log2 units (FP32 coefficients)
__device__ __forceinline__ double gexp(double e) { return exp(e); }     // natural units (FP64 coefficients)

template <typename T>
__device__ __forceinline__ T nu_of(const typename GCfg<T>::Chan &ch);
template <> __device__ __forceinline__ float nu_of<float>(const ChanF &ch) { return ch.nu_hi + ch.nu_lo; }
template <> __device__ __forceinline__ double nu_of<double>(const ChanD &ch) { return ch.nu; }

template <typename T>
struct GSmem {
    using T2 = typename GCfg<T>::T2;
    using TauT = typename std::conditional<sizeof(T) == 4, float2, double>::type;
    static constexpr int SG = GCfg<T>::SG;
    static size_t bytes(bool pointing) {
        size_t b = (size_t)SG * GNLOC * (sizeof(TauT) + sizeof(T));   // raw delays and beam radii
        b += (size_t)GNLOC * SG * sizeof(T2);                          // A
        if (pointing) b += (size_t)GNLOC * SG * sizeof(T2);            // dlnE/dl, dlnE/dm
        b += (size_t)NBMAX * 4 * sizeof(T);                            // baseline table
        b += (size_t)2 * BLC * 4 * sizeof(T2);                         // Y chunks (double buffer)
        // the final combine: one FP64 row of NGRAD per (baseline group, source);
        // a thread of the FP32 kernel holds two sources
        const size_t red = (size_t)(sizeof(T) == 4 ? 2 : 1) * GTHREADS * NGRAD * sizeof(double);
        return std::max(b, red);
    }
};

// One block: timestep t, a group of channels, one antenna unit, SG sources;
// thread (source sl, baseline group grp).
template <typename T>
__global__ void __launch_bounds__(GTHREADS) k_grad_src(const GradParams P) {
    using C = GCfg<T>;
    using T2 = typename C::T2;
    using Chan = typename C::Chan;
    using TauT = typename std::conditional<sizeof(T) == 4, float2, double>::type;
    constexpr int SG = C::SG;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // layout: raw tau | raw rho | A | [dlnE] | baseline table | Y chunk
    TauT *rTau = reinterpret_cast<TauT *>(smem_raw);
    T *rRho = reinterpret_cast<T *>(rTau + SG * GNLOC);
    T2 *sA = reinterpret_cast<T2 *>(rRho + SG * GNLOC);
    T2 *sE = sA + GNLOC * SG;
    T *sB = reinterpret_cast<T *>(P.has_pointing ? sE + GNLOC * SG : sE);
    T2 *sY = reinterpret_cast<T2 *>(sB + 4 * NBMAX);
    double *sRed = reinterpret_cast<double *>(smem_raw);   // reused at the end

    if (inputs_bad(P.status)) return;
    const int tid = threadIdx.x;
    int bid = blockIdx.x;
    const int sch = bid % P.nsch;
    // NS sources x NG baseline groups: a chunk with fewer than SG sources (the
    // list's last) gives its threads more baseline groups rather than idle
    // duplicate sources (NS the power of two that covers them, NS NG = GTHREADS)
    const int nact = min(SG, P.nsrc - sch * SG);
    int NS = SG;
    while (NS / 2 >= nact) NS /= 2;
    const int NG = GTHREADS / NS;
    const int sl = tid % NS, grp = tid / NS;
    bid /= P.nsch;
    const int u = bid % P.nunits;
    bid /= P.nunits;
    const int cg = bid % P.ncg;
    const int t = bid / P.ncg;
    const Unit U = P.units[u];
    const int nb = U.nbody;
    const int s = sch * SG + sl;
    const bool sact = s < P.nsrc;
    const int sidx = sact ? s : P.nsrc - 1;
    const int nloc = U.diag ? U.nr : U.nr + U.nc;
    const bool pointing = P.has_pointing != 0;
    const int k0 = cg * P.chan_group, k1 = min(P.nchan, k0 + P.chan_group);

    // ---- per block: delays of every (antenna, source) and the baseline table ----
    for (int j = tid; j < nloc * NS; j += GTHREADS) {   // the source slots the threads read
        const int a = j / NS, ss = j - a * NS, i = a * SG + ss;
        const int src = min(sch * SG + ss, P.nsrc - 1);
        const int ant = a < U.nr ? U.r0 + a : U.c0 + (a - U.nr);
        const long long di = ((long long)t * P.nsrc + src) * P.na + ant;
        rTau[i] = reinterpret_cast<const TauT *>(P.tau)[di];
        rRho[i] = reinterpret_cast<const T *>(P.rho)[di];
    }
    const uint16_t *bls = P.bls + U.tile0;
    for (int i = tid; i < nb; i += GTHREADS) {
        const uint16_t e = bls[i];
        const int pl = e & 0xff, ql = e >> 8;
        const int p = U.r0 + pl, q = U.c0 + ql;
        const double *xp = P.uvw + 3 * ((long long)t * P.na + p);
        const double *xq = P.uvw + 3 * ((long long)t * P.na + q);
        const int la = pl, lb = U.diag ? ql : U.nr + ql;
        T *b = sB + 4 * i;
        b[0] = (T)(xp[0] - xq[0]);
        b[1] = (T)(xp[1] - xq[1]);
        b[2] = (T)(xp[2] - xq[2]);
        b[3] = int_bits<T>((la * SG) | ((lb * SG) << 16));   // shared offsets of A_p, A_q
    }

    // ---- per-source constants of this thread ----
    const T *st = reinterpret_cast<const T *>(P.stokes) + 4 * sidx;
    const T sI = st[0], sQ = st[1], sU = st[2], sV = st[3];
    const T *gq = reinterpret_cast<const T *>(P.gauss) + 4 * sidx;
    const bool is_gauss = gq[3] != T(0), is_disk = gq[3] > T(1.5);
    const T *extra = reinterpret_cast<const T *>(P.extra) + 8 * sidx;
    const double l = extra[0], m = extra[1], l_n = extra[2], m_n = extra[3];
    const double maj = extra[4], mn = extra[5], sp = extra[6], cp = extra[7];
    const double alpha = (double)reinterpret_cast<const T *>(P.alpha)[sidx];
    const double *ptab = pointing ? P.pointing + 2 * (long long)t * P.na : nullptr;
    const T2 *yin = reinterpret_cast<const T2 *>(P.yin);

    double out[NGRAD];
#pragma unroll
    for (int i = 0; i < NGRAD; i++) out[i] = 0.0;

    // Y chunks of (channel, baseline chunk) in order, double-buffered: chunk j
    // is prefetched while chunk j - 1 is summed.
    const int nchunk = (nb + BLC - 1) / BLC;
    auto issue_y = [&](int j) {
        const int kk = k0 + j / nchunk, b0 = (j % nchunk) * BLC;
        const int cnt = min(BLC, nb - b0);
        T2 *dst = sY + (j & 1) * BLC * 4;
        for (int i = tid; i < 2 * cnt; i += GTHREADS) {   // 2 x 16 bytes per baseline (FP32)
            const int jj = i >> 1, half = i & 1;
            const uint16_t e = bls[b0 + jj];
            const int p = U.r0 + (e & 0xff), q = U.c0 + (e >> 8);
            const long long bl = (long long)p * P.na - (long long)p * (p + 1) / 2 + (q - p - 1);
            const T2 *src = yin + 4 * (((long long)t * P.nbl + bl) * P.nchan + kk);
            if (sizeof(T) == 4) {
                cp16(dst + 4 * jj + 2 * half, src + 2 * half);
            } else {
                cp16(dst + 4 * jj + 2 * half, src + 2 * half);
                cp16(dst + 4 * jj + 2 * half + 1, src + 2 * half + 1);
            }
        }
        cp_commit();
    };
    const int njobs = (k1 - k0) * nchunk;
    if (njobs > 0) issue_y(0);
    int job = 0;
    for (int k = k0; k < k1; k++) {
        const Chan ch = reinterpret_cast<const Chan *>(P.chan)[k];
        __syncthreads();   // delays staged / the previous channel is done with sA
        // ---- A (= K, or E K with pointing errors) of every (antenna, source) ----
        for (int j = tid; j < nloc * NS; j += GTHREADS) {
            const int i = (j / NS) * SG + (j % NS);
            T2 v = phase(rTau + i, 0, ch);
            if (pointing) {
                const int a = i / SG, ss = i - a * SG;
                const int src = min(sch * SG + ss, P.nsrc - 1);
                const int ant = a < U.nr ? U.r0 + a : U.c0 + (a - U.nr);
                const T *ex = reinterpret_cast<const T *>(P.extra) + 8 * src;
                T E, t3;
                beam_Ed(ch.beam, ch.cnu * rRho[i], E, t3);
                v.x *= E;
                v.y *= E;
                T2 d;   // dlnE/dl, dlnE/dm = t3 cnu^2 (l - dl_ta, m - dm_ta)  (eq. 4)
                d.x = t3 * ch.cnu * ch.cnu * (ex[0] - (T)ptab[2 * ant]);
                d.y = t3 * ch.cnu * ch.cnu * (ex[1] - (T)ptab[2 * ant + 1]);
                sE[i] = d;
            }
            sA[i] = v;
        }
        const T gA = gq[0] * ch.nu2, gB = gq[1] * ch.nu2, gC = gq[2] * ch.nu2;
        T acc[NACC];
#pragma unroll
        for (int i = 0; i < NACC; i++) acc[i] = T(0);
        for (int b0 = 0; b0 < nb; b0 += BLC, job++) {
            const int cnt = min(BLC, nb - b0);
            cp_wait_all();
            __syncthreads();   // chunk `job` landed; everyone is done with the other buffer
            if (job + 1 < njobs) issue_y(job + 1);
            const T2 *yb = sY + (job & 1) * BLC * 4;
#pragma unroll 2
            for (int i = grp; i < cnt; i += NG) {
                const T *b = sB + 4 * (b0 + i);
                const T du = b[0], dv = b[1], dw = b[2];
                const int pq = bits_int(b[3]);
                const int oa = pq & 0xffff, ob = pq >> 16;
                const T2 ap = sA[oa + sl], aq = sA[ob + sl];
                T zr = ap.x * aq.x + ap.y * aq.y;   // z = A_p conj(A_q)
                T zi = ap.y * aq.x - ap.x * aq.y;
                T hq = T(1);   // (dg/dq) / g in units of the form's derivative: 1 Gaussian, -3/2 / (1 + q) disk
                if (is_gauss) {
                    const T e = gA * du * du + gB * du * dv + gC * dv * dv;
                    T g;
                    if (is_disk) {
                        const T r = rsqrt(T(1) + e);
                        g = r * r * r;
                        hq = T(-1.5) * r * r;
                    } else {
                        g = gexp(e);
                    }
                    zr *= g;
                    zi *= g;
                }
                const T2 y0 = yb[4 * i], y1 = yb[4 * i + 1], y2 = yb[4 * i + 2], y3 = yb[4 * i + 3];
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
                    const T rh = re * hq;
                    acc[7] += rh * du * du;
                    acc[8] += rh * du * dv;
                    acc[9] += rh * dv * dv;
                }
                if (pointing) {
                    const T2 ep = sE[oa + sl], eq = sE[ob + sl];
                    acc[10] += re * (ep.x + eq.x);
                    acc[11] += re * (ep.y + eq.y);
                }
            }
        }
        // ---- this channel's factors (derivatives of eqs. 2-4), in the kernel's
        // precision; the sums over channels are kept in FP64 ----
        const T nu = nu_of<T>(ch);
        const T lnr = log(nu / (T)P.ref_freq_hz);
        T w = exp((T)alpha * lnr);              // spectral factor f
        T dlnE2_l = 0, dlnE2_m = 0;
        if (!pointing) {
            T E, t3;                            // the beam E_s^2 shared by both antennas
            beam_Ed(ch.beam, ch.cnu * rRho[sl], E, t3);
            w *= E * E;
            const T cnu2 = ch.cnu * ch.cnu;
            dlnE2_l = T(2) * t3 * cnu2 * (T)l;
            dlnE2_m = T(2) * t3 * cnu2 * (T)m;
        }
        const T aR = sI * acc[0] + sQ * acc[1] + sU * acc[2] + sV * acc[3];
        const T k2pi = T(2.0 * kPi / kCLight) * nu;
        out[0] += (double)(w * (-k2pi * (acc[4] - (T)l_n * acc[6]) + (pointing ? acc[10] : aR * dlnE2_l)));
        out[1] += (double)(w * (-k2pi * (acc[5] - (T)m_n * acc[6]) + (pointing ? acc[11] : aR * dlnE2_m)));
        out[2] += (double)(w * acc[0]);
        out[3] += (double)(w * acc[1]);
        out[4] += (double)(w * acc[2]);
        out[5] += (double)(w * acc[3]);
        out[6] += (double)(w * aR * lnr);
        if (is_gauss) {
            // Gaussian: ln g = nu^2 (A du^2 + B du dv + C dv^2), A = -K (maj^2 sp^2 + min^2 cp^2),
            // B = -2 K sp cp (maj^2 - min^2), C = -K (maj^2 cp^2 + min^2 sp^2), K = pi^2/(4 ln 2 c^2);
            // disk: q = the same form with -K -> 4 pi^2 / c^2, its -3/2 / (1 + q) in the moments
            const T K = is_disk ? T(-4.0 * kPi * kPi / (kCLight * kCLight)) * nu * nu
                                : T(kGaussK / (kCLight * kCLight)) * nu * nu;
            const T mj = (T)maj, mi = (T)mn, sps = (T)sp, cps = (T)cp;
            const T dd = mj * mj - mi * mi;
            const T Au = acc[7], Auv = acc[8], Av = acc[9];
            out[7] += (double)(w * -K * (2 * mj * sps * sps * Au + 4 * mj * sps * cps * Auv + 2 * mj * cps * cps * Av));
            out[8] += (double)(w * -K * (2 * mi * cps * cps * Au - 4 * mi * sps * cps * Auv + 2 * mi * sps * sps * Av));
            out[9] += (double)(w * -K * (2 * sps * cps * dd * Au + 2 * dd * (cps * cps - sps * sps) * Auv -
                                         2 * sps * cps * dd * Av));
        }
    }
    // ---- combine the baseline groups in a fixed order: one partial per source ----
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NGRAD; i++) sRed[(grp * NS + sl) * NGRAD + i] = out[i];
    __syncthreads();
    if (grp == 0 && sact) {
        const long long prow = ((long long)t * P.ncg + cg) * P.nunits + u;
        double *o = P.partials + (prow * P.nsrc + s) * NGRAD;
        for (int i = 0; i < NGRAD; i++) {
            double v = 0.0;
            for (int g = 0; g < NG; g++) v += sRed[(g * NS + sl) * NGRAD + i];
            o[i] = v;
        }
    }
}

// FP32 version with two sources per thread: thread (source pair sp, baseline
// group grp of 16); the pair's z, Gaussian factors and moments are computed
// on packed FP32 pairs (one instruction for both sources), the baseline data
// and Y_X are shared by the pair. Same staging, moments and channel factors as
// k_grad_src, with the per-antenna factors of a source pair staged as
// (re, re', im, im') (one load gives both pairs) and each thread's next
// baseline found by arithmetic along the row-major baseline list, so that
// the factor loads do not wait for a table load.
__device__ __forceinline__ float2 pf2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 pdup(float a) { return make_float2(a, a); }

template <bool GENERAL>
__global__ void __launch_bounds__(GTHREADS, 2) k_grad_src_f32x2(const GradParams P) {
    // GENERAL = false: eq. 4's cos^3 beam, points and Gaussians (the code of
    // the general case costs this register-bound kernel ~3 %)
    const int beam_model = GENERAL ? reinterpret_cast<const ChanF *>(P.chan)[0].beam : RIME_BEAM_COS3;
    using T = float;
    using T2 = float2;
    constexpr int SG = GCfg<float>::SG;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *rTau = reinterpret_cast<float2 *>(smem_raw);
    T *rRho = reinterpret_cast<T *>(rTau + SG * GNLOC);
    T2 *sA = reinterpret_cast<T2 *>(rRho + SG * GNLOC);
    T2 *sE = sA + GNLOC * SG;
    T *sB = reinterpret_cast<T *>(P.has_pointing ? sE + GNLOC * SG : sE);
    T2 *sY = reinterpret_cast<T2 *>(sB + 4 * NBMAX);
    double *sRed = reinterpret_cast<double *>(smem_raw);   // reused at the end

    if (inputs_bad(P.status)) return;
    const int tid = threadIdx.x;
    int bid = blockIdx.x;
    const int sch = bid % P.nsch;
    // NP source pairs x NG baseline groups: a chunk with fewer than SG
    // sources (the list's last) gives its threads more baseline groups
    // rather than idle duplicate sources (NP the power of two that covers its
    // pairs, NP NG = GTHREADS)
    const int npair = (min(SG, P.nsrc - sch * SG) + 1) / 2;
    int NP = SG / 2;
    while (NP / 2 >= npair) NP /= 2;
    const int NG = GTHREADS / NP;
    const int sp = tid % NP, grp = tid / NP;
    bid /= P.nsch;
    const int u = bid % P.nunits;
    bid /= P.nunits;
    const int cg = bid % P.ncg;
    const int t = bid / P.ncg;
    const Unit U = P.units[u];
    const int nb = U.nbody;
    const int nloc = U.diag ? U.nr : U.nr + U.nc;
    const bool pointing = P.has_pointing != 0;
    const int k0 = cg * P.chan_group, k1 = min(P.nchan, k0 + P.chan_group);

    const int nss = 2 * NP;   // source slots the threads read (the rest are never staged)
    for (int j = tid; j < nloc * nss; j += GTHREADS) {
        const int a = j / nss, ss = j - a * nss, i = a * SG + ss;
        const int src = min(sch * SG + ss, P.nsrc - 1);
        const int ant = a < U.nr ? U.r0 + a : U.c0 + (a - U.nr);
        const long long di = ((long long)t * P.nsrc + src) * P.na + ant;
        rTau[i] = reinterpret_cast<const float2 *>(P.tau)[di];
        rRho[i] = reinterpret_cast<const T *>(P.rho)[di];
    }
    const uint16_t *bls = P.bls + U.tile0;
    for (int i = tid; i < nb; i += GTHREADS) {
        const uint16_t e = bls[i];
        const int pl = e & 0xff, ql = e >> 8;
        const int p = U.r0 + pl, q = U.c0 + ql;
        const double *xp = P.uvw + 3 * ((long long)t * P.na + p);
        const double *xq = P.uvw + 3 * ((long long)t * P.na + q);
        const int la = pl, lb = U.diag ? ql : U.nr + ql;
        T *b = sB + 4 * i;
        b[0] = (T)(xp[0] - xq[0]);
        b[1] = (T)(xp[1] - xq[1]);
        b[2] = (T)(xp[2] - xq[2]);
        b[3] = int_bits<T>((la * SG) | ((lb * SG) << 16));
    }

    // ---- per-source constants of this thread's two sources (the rest is read
    // from the L1-resident tables once per channel, outside the baseline loop)
    int sidx[2];
    bool sact[2], is_gauss[2], is_disk[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int s = sch * SG + 2 * sp + h;
        sact[h] = s < P.nsrc;
        sidx[h] = sact[h] ? s : P.nsrc - 1;
        is_gauss[h] = reinterpret_cast<const T *>(P.gauss)[4 * sidx[h] + 3] != T(0);
        is_disk[h] = GENERAL && P.has_disk && reinterpret_cast<const T *>(P.gauss)[4 * sidx[h] + 3] > T(1.5);
    }
    const bool any_gauss = is_gauss[0] || is_gauss[1];
    const bool any_disk = GENERAL && (is_disk[0] || is_disk[1]);
    const float4 st0 = reinterpret_cast<const float4 *>(P.stokes)[sidx[0]];
    const float4 st1 = reinterpret_cast<const float4 *>(P.stokes)[sidx[1]];
    const float2 sI = pf2(st0.x, st1.x), sQ = pf2(st0.y, st1.y);
    const float2 sU = pf2(st0.z, st1.z), sV = pf2(st0.w, st1.w);
    const double *ptab = pointing ? P.pointing + 2 * (long long)t * P.na : nullptr;
    const T2 *yin = reinterpret_cast<const T2 *>(P.yin);

    // per-block sums over the block's channels in FP32 (at most 8 terms each;
    // FP64 adds at 1/64 of the FP32 rate kept the FP64 pipe 11 % busy); the
    // block partials are combined in FP64
    float out[2][NGRAD];
#pragma unroll
    for (int h = 0; h < 2; h++)
#pragma unroll
        for (int i = 0; i < NGRAD; i++) out[h][i] = 0.f;

    const int nchunk = (nb + BLC - 1) / BLC;
    const int qend = U.diag ? U.nr : U.nc, cofs = U.diag ? 0 : U.nr;   // columns of a row; their offset
    auto issue_y = [&](int j) {
        const int kk = k0 + j / nchunk, b0 = (j % nchunk) * BLC;
        const int cnt = min(BLC, nb - b0);
        T2 *dst = sY + (j & 1) * BLC * 4;
        for (int i = tid; i < 2 * cnt; i += GTHREADS) {
            const int jj = i >> 1, half = i & 1;
            const uint16_t e = bls[b0 + jj];
            const int p = U.r0 + (e & 0xff), q = U.c0 + (e >> 8);
            const long long bl = (long long)p * P.na - (long long)p * (p + 1) / 2 + (q - p - 1);
            const T2 *src = yin + 4 * (((long long)t * P.nbl + bl) * P.nchan + kk);
            cp16(dst + 4 * jj + 2 * half, src + 2 * half);
        }
        cp_commit();
    };
    const int njobs = (k1 - k0) * nchunk;
    if (njobs > 0) issue_y(0);
    int job = 0;
    for (int k = k0; k < k1; k++) {
        const ChanF ch = reinterpret_cast<const ChanF *>(P.chan)[k];
        __syncthreads();
        for (int j = tid; j < nloc * nss; j += GTHREADS) {
            const int i = (j / nss) * SG + (j % nss);
            T2 v = f32::phase_factor(rTau[i], ch);   // the forward kernels' K
            if (pointing) {
                const int a = i / SG, ss = i - a * SG;
                const int src = min(sch * SG + ss, P.nsrc - 1);
                const int ant = a < U.nr ? U.r0 + a : U.c0 + (a - U.nr);
                const T *exq = reinterpret_cast<const T *>(P.extra) + 8 * src;
                T E, t3;
                beam_Ed(beam_model, ch.cnu * rRho[i], E, t3);
                v.x *= E;
                v.y *= E;
                T2 d;
                d.x = t3 * ch.cnu * ch.cnu * (exq[0] - (T)ptab[2 * ant]);
                d.y = t3 * ch.cnu * ch.cnu * (exq[1] - (T)ptab[2 * ant + 1]);
                float *oe = reinterpret_cast<float *>(sE) + 2 * (i & ~1) + (i & 1);
                oe[0] = d.x;
                oe[2] = d.y;
            }
            float *o = reinterpret_cast<float *>(sA) + 2 * (i & ~1) + (i & 1);   // (re, re', im, im')
            o[0] = v.x;
            o[2] = v.y;
        }
        const float4 gq0 = reinterpret_cast<const float4 *>(P.gauss)[sidx[0]];
        const float4 gq1 = reinterpret_cast<const float4 *>(P.gauss)[sidx[1]];
        const float2 gA = pf2(gq0.x * ch.nu2, gq1.x * ch.nu2);
        const float2 gB = pf2(gq0.y * ch.nu2, gq1.y * ch.nu2);
        const float2 gC = pf2(gq0.z * ch.nu2, gq1.z * ch.nu2);
        float2 acc[NACC];
#pragma unroll
        for (int i = 0; i < NACC; i++) acc[i] = pf2(0.f, 0.f);
        for (int b0 = 0; b0 < nb; b0 += BLC, job++) {
            const int cnt = min(BLC, nb - b0);
            cp_wait_all();
            __syncthreads();
            if (job + 1 < njobs) issue_y(job + 1);
            const T2 *yb = sY + (job & 1) * BLC * 4;
            // local (row, column) of this thread's baseline b0 + i
            int pl = 0, ql = 0;
            if (grp < cnt) {
                const uint16_t e = bls[b0 + grp];
                pl = e & 0xff;
                ql = e >> 8;
            }
#pragma unroll 2
            for (int i = grp; i < cnt; i += NG) {
                const float4 bb = *reinterpret_cast<const float4 *>(sB + 4 * (b0 + i));
                const T du = bb.x, dv = bb.y, dw = bb.z;
                const int oa = pl * SG, ob = (cofs + ql) * SG;
                const float4 ap = *reinterpret_cast<const float4 *>(sA + oa + 2 * sp);
                const float4 aq = *reinterpret_cast<const float4 *>(sA + ob + 2 * sp);
                if (i + NG < cnt) {   // the next baseline of this thread (it exists: the walk ends)
                    ql += NG;
                    for (int w = 0; w < GNLOC && ql >= qend; w++) {
                        pl++;
                        ql -= qend - (U.diag ? pl + 1 : 0);
                    }
                }
                const float2 apr = pf2(ap.x, ap.y), api = pf2(ap.z, ap.w);
                const float2 aqr = pf2(aq.x, aq.y), aqi = pf2(aq.z, aq.w);
                // z = A_p conj(A_q) for both sources
                float2 zr = __ffma2_rn(apr, aqr, __fmul2_rn(api, aqi));
                float2 zi = __ffma2_rn(api, aqr, __fmul2_rn(pf2(-apr.x, -apr.y), aqi));
                float2 hq = pf2(1.f, 1.f);   // as in k_grad_src: 1 Gaussian, -3/2 / (1 + q) disk
                if (any_gauss) {
                    const float2 e = __ffma2_rn(gA, pdup(du * du), __ffma2_rn(gB, pdup(du * dv), __fmul2_rn(gC, pdup(dv * dv))));
                    float2 g;
                    if (any_disk) {
                        const float r0 = rsqrtf(1.f + e.x), r1 = rsqrtf(1.f + e.y);
                        g.x = is_disk[0] ? r0 * r0 * r0 : ex2_approx(e.x);
                        g.y = is_disk[1] ? r1 * r1 * r1 : ex2_approx(e.y);
                        hq.x = is_disk[0] ? -1.5f * r0 * r0 : 1.f;
                        hq.y = is_disk[1] ? -1.5f * r1 * r1 : 1.f;
                    } else {
                        g = pf2(ex2_approx(e.x), ex2_approx(e.y));   // the forward kernels' exp2
                    }
                    zr = __fmul2_rn(zr, g);
                    zi = __fmul2_rn(zi, g);
                }
                const float4 y01 = *reinterpret_cast<const float4 *>(yb + 4 * i);
                const float4 y23 = *reinterpret_cast<const float4 *>(yb + 4 * i + 2);
                const float2 nzi = pf2(-zi.x, -zi.y);
                acc[0] = __ffma2_rn(zr, pdup(y01.x), __ffma2_rn(nzi, pdup(y01.y), acc[0]));
                acc[1] = __ffma2_rn(zr, pdup(y01.z), __ffma2_rn(nzi, pdup(y01.w), acc[1]));
                acc[2] = __ffma2_rn(zr, pdup(y23.x), __ffma2_rn(nzi, pdup(y23.y), acc[2]));
                acc[3] = __ffma2_rn(zr, pdup(y23.z), __ffma2_rn(nzi, pdup(y23.w), acc[3]));
                const float2 br = __ffma2_rn(sI, pdup(y01.x), __ffma2_rn(sQ, pdup(y01.z),
                                  __ffma2_rn(sU, pdup(y23.x), __fmul2_rn(sV, pdup(y23.z)))));
                const float2 bi = __ffma2_rn(sI, pdup(y01.y), __ffma2_rn(sQ, pdup(y01.w),
                                  __ffma2_rn(sU, pdup(y23.y), __fmul2_rn(sV, pdup(y23.w)))));
                const float2 re = __ffma2_rn(zr, br, __fmul2_rn(nzi, bi));   // z beta
                const float2 im = __ffma2_rn(zr, bi, __fmul2_rn(zi, br));
                acc[4] = __ffma2_rn(im, pdup(du), acc[4]);
                acc[5] = __ffma2_rn(im, pdup(dv), acc[5]);
                acc[6] = __ffma2_rn(im, pdup(dw), acc[6]);
                if (any_gauss) {
                    const float2 rh = any_disk ? __fmul2_rn(re, hq) : re;
                    acc[7] = __ffma2_rn(rh, pdup(du * du), acc[7]);
                    acc[8] = __ffma2_rn(rh, pdup(du * dv), acc[8]);
                    acc[9] = __ffma2_rn(rh, pdup(dv * dv), acc[9]);
                }
                if (pointing) {
                    const float4 ep = *reinterpret_cast<const float4 *>(sE + oa + 2 * sp);
                    const float4 eq = *reinterpret_cast<const float4 *>(sE + ob + 2 * sp);
                    acc[10] = __ffma2_rn(re, pf2(ep.x + eq.x, ep.y + eq.y), acc[10]);
                    acc[11] = __ffma2_rn(re, pf2(ep.z + eq.z, ep.w + eq.w), acc[11]);
                }
            }
        }
        const T nu = nu_of<T>(ch);
        const T lnr = log(nu / (T)P.ref_freq_hz);
        const T k2pi = T(2.0 * kPi / kCLight) * nu;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            T a[NACC];
#pragma unroll
            for (int i = 0; i < NACC; i++) a[i] = h ? acc[i].y : acc[i].x;
            const T *ex = reinterpret_cast<const T *>(P.extra) + 8 * sidx[h];
            const T l = ex[0], m = ex[1], l_n = ex[2], m_n = ex[3];
            const float4 st = h ? st1 : st0;
            T w = exp(reinterpret_cast<const T *>(P.alpha)[sidx[h]] * lnr);
            T dlnE2_l = 0, dlnE2_m = 0;
            if (!pointing) {
                T E, t3;
                beam_Ed(beam_model, ch.cnu * rRho[2 * sp + h], E, t3);
                w *= E * E;
                const T cnu2 = ch.cnu * ch.cnu;
                dlnE2_l = T(2) * t3 * cnu2 * l;
                dlnE2_m = T(2) * t3 * cnu2 * m;
            }
            const T aR = st.x * a[0] + st.y * a[1] + st.z * a[2] + st.w * a[3];
            out[h][0] += (w * (-k2pi * (a[4] - l_n * a[6]) + (pointing ? a[10] : aR * dlnE2_l)));
            out[h][1] += (w * (-k2pi * (a[5] - m_n * a[6]) + (pointing ? a[11] : aR * dlnE2_m)));
            out[h][2] += (w * a[0]);
            out[h][3] += (w * a[1]);
            out[h][4] += (w * a[2]);
            out[h][5] += (w * a[3]);
            out[h][6] += (w * aR * lnr);
            if (is_gauss[h]) {
                const T K = is_disk[h] ? T(-4.0 * kPi * kPi / (kCLight * kCLight)) * nu * nu
                                       : T(kGaussK / (kCLight * kCLight)) * nu * nu;
                const T mj = ex[4], mi = ex[5], sps = ex[6], cps = ex[7];
                const T dd = mj * mj - mi * mi;
                const T Au = a[7], Auv = a[8], Av = a[9];
                out[h][7] += (w * -K * (2 * mj * sps * sps * Au + 4 * mj * sps * cps * Auv + 2 * mj * cps * cps * Av));
                out[h][8] += (w * -K * (2 * mi * cps * cps * Au - 4 * mi * sps * cps * Auv + 2 * mi * sps * sps * Av));
                out[h][9] += (w * -K * (2 * sps * cps * dd * Au + 2 * dd * (cps * cps - sps * sps) * Auv -
                                                2 * sps * cps * dd * Av));
            }
        }
    }
    // ---- combine the baseline groups in a fixed order: one partial per source ----
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; h++)
#pragma unroll
        for (int i = 0; i < NGRAD; i++) sRed[(grp * 2 * NP + 2 * sp + h) * NGRAD + i] = out[h][i];
    __syncthreads();
    if (grp == 0) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
            if (!sact[h]) continue;
            const long long prow = ((long long)t * P.ncg + cg) * P.nunits + u;
            double *o = P.partials + (prow * P.nsrc + sidx[h]) * NGRAD;
            for (int i = 0; i < NGRAD; i++) {
                double v = 0.0;
                for (int g = 0; g < NG; g++) v += sRed[(g * 2 * NP + 2 * sp + h) * NGRAD + i];
                o[i] = v;
            }
        }
    }
}

// Channel-parallel variant for units with few baselines (arrays of up to 23
// antennas): a block owns (t, CPC channels, unit, CPS sources) and a thread
// one (source, channel), summing the 12 adjoint moments over all the unit's
// baselines and forming that channel's 10 gradients (the same formulas as
// k_grad_src). The baseline-group threads of k_grad_src would each see one
// or two of a small unit's baselines per channel and walk its channels one
// after another; here the channels run side by side.
constexpr int CPS = 16;   // sources per block
template <typename T> struct CpCfg;
template <> struct CpCfg<float> { static constexpr int CPC = 16; };    // channels per block
template <> struct CpCfg<double> { static constexpr int CPC = 8; };
constexpr int NBCP = 256;   // baselines of a unit, at most

template <typename T>
struct CpSmem {
    using T2 = typename GCfg<T>::T2;
    using TauT = typename std::conditional<sizeof(T) == 4, float2, double>::type;
    static size_t bytes(int nloc, bool pointing) {
        constexpr int CPC = CpCfg<T>::CPC;
        size_t b = (size_t)CPS * nloc * (sizeof(TauT) + sizeof(T));           // raw delays, beam radii
        b += (size_t)CPC * nloc * CPS * sizeof(T2) * (pointing ? 2 : 1);       // A (and dlnE) per channel
        b += (size_t)NBCP * 4 * sizeof(T);                                     // baseline table
        b = (b + 7) & ~(size_t)7;
        b += (size_t)CPC * CPS * NGRAD * sizeof(double);                        // per-thread results
        return b;
    }
};

template <typename T>
__global__ void __launch_bounds__(CPS * CpCfg<T>::CPC) k_grad_src_cp(const GradParams P) {
    using C = GCfg<T>;
    using T2 = typename C::T2;
    using Chan = typename C::Chan;
    using TauT = typename std::conditional<sizeof(T) == 4, float2, double>::type;
    constexpr int CPC = CpCfg<T>::CPC, NT = CPS * CPC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (inputs_bad(P.status)) return;
    const int tid = threadIdx.x;
    const int sl = tid % CPS, kc = tid / CPS;
    int bid = blockIdx.x;
    const int sch = bid % P.nsch;
    bid /= P.nsch;
    const int u = bid % P.nunits;
    bid /= P.nunits;
    const int cg = bid % P.ncg;
    const int t = bid / P.ncg;
    const Unit U = P.units[u];
    const int nb = U.nbody;
    const int nloc = U.diag ? U.nr : U.nr + U.nc;
    TauT *rTau = reinterpret_cast<TauT *>(smem_raw);                  // [nloc][CPS]
    T *rRho = reinterpret_cast<T *>(rTau + nloc * CPS);               // [nloc][CPS]
    T2 *sA = reinterpret_cast<T2 *>(rRho + nloc * CPS);               // [CPC][nloc][CPS]
    const bool pointing = P.has_pointing != 0;
    T2 *sE = sA + CPC * nloc * CPS;                                   // [CPC][nloc][CPS] with pointing
    T *sB = reinterpret_cast<T *>(pointing ? sE + CPC * nloc * CPS : sE);
    double *sRed = reinterpret_cast<double *>(
        (reinterpret_cast<uintptr_t>(sB + 4 * NBCP) + 7) & ~(uintptr_t)7);   // [CPC][CPS][NGRAD]
    const int s = sch * CPS + sl;
    const bool sact = s < P.nsrc;
    const int sidx = sact ? s : P.nsrc - 1;
    const int k0 = cg * P.chan_group;
    const int k = k0 + kc;
    const bool kact = kc < P.chan_group && k < P.nchan;
    const Chan *chan = reinterpret_cast<const Chan *>(P.chan);
    const double *ptab = pointing ? P.pointing + 2 * (long long)t * P.na : nullptr;

    // ---- delays and radii of every (antenna, source); the baseline table ----
    for (int i = tid; i < nloc * CPS; i += NT) {
        const int a = i / CPS, ss = i - a * CPS;
        const int src = min(sch * CPS + ss, P.nsrc - 1);
        const int ant = a < U.nr ? U.r0 + a : U.c0 + (a - U.nr);
        const long long di = ((long long)t * P.nsrc + src) * P.na + ant;
        rTau[i] = reinterpret_cast<const TauT *>(P.tau)[di];
        rRho[i] = reinterpret_cast<const T *>(P.rho)[di];
    }
    const uint16_t *bls = P.bls + U.tile0;
    for (int i = tid; i < nb; i += NT) {
        const uint16_t e = bls[i];
        const int pl = e & 0xff, ql = e >> 8;
        const int p = U.r0 + pl, q = U.c0 + ql;
        const double *xp = P.uvw + 3 * ((long long)t * P.na + p);
        const double *xq = P.uvw + 3 * ((long long)t * P.na + q);
        const int la = pl, lb = U.diag ? ql : U.nr + ql;
        T *b = sB + 4 * i;
        b[0] = (T)(xp[0] - xq[0]);
        b[1] = (T)(xp[1] - xq[1]);
        b[2] = (T)(xp[2] - xq[2]);
        b[3] = int_bits<T>((la * CPS) | ((lb * CPS) << 16));
    }
    __syncthreads();
    // ---- A = K (E K with pointing errors) for every (channel, antenna, source) ----
    for (int i = tid; i < CPC * nloc * CPS; i += NT) {
        const int c = i / (nloc * CPS), r = i - c * (nloc * CPS);
        const int kk = min(k0 + c, P.nchan - 1);
        const Chan ch = chan[kk];
        T2 v = phase(rTau + r, 0, ch);
        if (pointing) {
            const int a = r / CPS, ss = r - a * CPS;
            const int src = min(sch * CPS + ss, P.nsrc - 1);
            const int ant = a < U.nr ? U.r0 + a : U.c0 + (a - U.nr);
            const T *ex = reinterpret_cast<const T *>(P.extra) + 8 * src;
            T E, t3;
            beam_Ed(ch.beam, ch.cnu * rRho[r], E, t3);
            v.x *= E;
            v.y *= E;
            T2 d;
            d.x = t3 * ch.cnu * ch.cnu * (ex[0] - (T)ptab[2 * ant]);
            d.y = t3 * ch.cnu * ch.cnu * (ex[1] - (T)ptab[2 * ant + 1]);
            sE[i] = d;
        }
        sA[i] = v;
    }
    __syncthreads();

    double out[NGRAD];
#pragma unroll
    for (int i = 0; i < NGRAD; i++) out[i] = 0.0;
    if (kact) {
        const Chan ch = chan[k];
        const T *st = reinterpret_cast<const T *>(P.stokes) + 4 * sidx;
        const T sI = st[0], sQ = st[1], sU = st[2], sV = st[3];
        const T *gq = reinterpret_cast<const T *>(P.gauss) + 4 * sidx;
        const bool is_gauss = gq[3] != T(0), is_disk = gq[3] > T(1.5);
        const T gA = gq[0] * ch.nu2, gB = gq[1] * ch.nu2, gC = gq[2] * ch.nu2;
        const T2 *cA = sA + kc * nloc * CPS, *cE = sE + kc * nloc * CPS;
        const T2 *yin = reinterpret_cast<const T2 *>(P.yin);
        T acc[NACC];
#pragma unroll
        for (int i = 0; i < NACC; i++) acc[i] = T(0);
        for (int i = 0; i < nb; i++) {
            const T *b = sB + 4 * i;
            const T du = b[0], dv = b[1], dw = b[2];
            const int pq = bits_int(b[3]);
            const int oa = pq & 0xffff, ob = pq >> 16;
            const T2 ap = cA[oa + sl], aq = cA[ob + sl];
            T zr = ap.x * aq.x + ap.y * aq.y;
            T zi = ap.y * aq.x - ap.x * aq.y;
            T hq = T(1);
            if (is_gauss) {
                const T e = gA * du * du + gB * du * dv + gC * dv * dv;
                T g;
                if (is_disk) {
                    const T r = rsqrt(T(1) + e);
                    g = r * r * r;
                    hq = T(-1.5) * r * r;
                } else {
                    g = gexp(e);
                }
                zr *= g;
                zi *= g;
            }
            const uint16_t e16 = bls[i];
            const int p = U.r0 + (e16 & 0xff), q = U.c0 + (e16 >> 8);
            const long long bl = (long long)p * P.na - (long long)p * (p + 1) / 2 + (q - p - 1);
            const T2 *y = yin + 4 * (((long long)t * P.nbl + bl) * P.nchan + k);
            const T2 y0 = y[0], y1 = y[1], y2 = y[2], y3 = y[3];
            acc[0] += zr * y0.x - zi * y0.y;
            acc[1] += zr * y1.x - zi * y1.y;
            acc[2] += zr * y2.x - zi * y2.y;
            acc[3] += zr * y3.x - zi * y3.y;
            const T br = sI * y0.x + sQ * y1.x + sU * y2.x + sV * y3.x;
            const T bi = sI * y0.y + sQ * y1.y + sU * y2.y + sV * y3.y;
            const T re = zr * br - zi * bi, im = zr * bi + zi * br;
            acc[4] += im * du;
            acc[5] += im * dv;
            acc[6] += im * dw;
            if (is_gauss) {
                const T rh = re * hq;
                acc[7] += rh * du * du;
                acc[8] += rh * du * dv;
                acc[9] += rh * dv * dv;
            }
            if (pointing) {
                const T2 ep = cE[oa + sl], eq = cE[ob + sl];
                acc[10] += re * (ep.x + eq.x);
                acc[11] += re * (ep.y + eq.y);
            }
        }
        // ---- this channel's factors (as in k_grad_src) ----
        const T *extra = reinterpret_cast<const T *>(P.extra) + 8 * sidx;
        const T l = extra[0], m = extra[1], l_n = extra[2], m_n = extra[3];
        const T nu = nu_of<T>(ch);
        const T lnr = log(nu / (T)P.ref_freq_hz);
        T w = exp(reinterpret_cast<const T *>(P.alpha)[sidx] * lnr);
        T dlnE2_l = 0, dlnE2_m = 0;
        if (!pointing) {
            T E, t3;
            beam_Ed(ch.beam, ch.cnu * rRho[sl], E, t3);
            w *= E * E;
            const T cnu2 = ch.cnu * ch.cnu;
            dlnE2_l = T(2) * t3 * cnu2 * l;
            dlnE2_m = T(2) * t3 * cnu2 * m;
        }
        const T aR = sI * acc[0] + sQ * acc[1] + sU * acc[2] + sV * acc[3];
        const T k2pi = T(2.0 * kPi / kCLight) * nu;
        out[0] = (double)(w * (-k2pi * (acc[4] - l_n * acc[6]) + (pointing ? acc[10] : aR * dlnE2_l)));
        out[1] = (double)(w * (-k2pi * (acc[5] - m_n * acc[6]) + (pointing ? acc[11] : aR * dlnE2_m)));
        out[2] = (double)(w * acc[0]);
        out[3] = (double)(w * acc[1]);
        out[4] = (double)(w * acc[2]);
        out[5] = (double)(w * acc[3]);
        out[6] = (double)(w * aR * lnr);
        if (is_gauss) {
            const T K = is_disk ? T(-4.0 * kPi * kPi / (kCLight * kCLight)) * nu * nu
                                : T(kGaussK / (kCLight * kCLight)) * nu * nu;
            const T mj = extra[4], mi = extra[5], sps = extra[6], cps = extra[7];
            const T dd = mj * mj - mi * mi;
            const T Au = acc[7], Auv = acc[8], Av = acc[9];
            out[7] = (double)(w * -K * (2 * mj * sps * sps * Au + 4 * mj * sps * cps * Auv + 2 * mj * cps * cps * Av));
            out[8] = (double)(w * -K * (2 * mi * cps * cps * Au - 4 * mi * sps * cps * Auv + 2 * mi * sps * sps * Av));
            out[9] = (double)(w * -K * (2 * sps * cps * dd * Au + 2 * dd * (cps * cps - sps * sps) * Auv -
                                        2 * sps * cps * dd * Av));
        }
    }
    // ---- combine the channels in a fixed order: one partial per source ----
#pragma unroll
    for (int i = 0; i < NGRAD; i++) sRed[(kc * CPS + sl) * NGRAD + i] = out[i];
    __syncthreads();
    if (kc == 0 && sact) {
        const long long prow = ((long long)t * P.ncg + cg) * P.nunits + u;
        double *o = P.partials + (prow * P.nsrc + s) * NGRAD;
        for (int i = 0; i < NGRAD; i++) {
            double v = 0.0;
            for (int c = 0; c < CPC; c++) v += sRed[(c * CPS + sl) * NGRAD + i];
            o[i] = v;
        }
    }
}

// Column sums of a [nrows][ncols] array in fixed order: block (x, y) sums
// rows [y rpb, (y+1) rpb) of 32 columns with 8 row phases, then the phases.
constexpr int RTX = 32, RTY = 8;
__global__ void k_colsum(long long nrows, long long ncols, long long rpb, const double *in, double *out,
                         const DevStatus *status) {
    __shared__ double red[RTY][RTX];
    if (inputs_bad(status)) return;
    const long long c = (long long)blockIdx.x * RTX + threadIdx.x;
    const long long r0 = (long long)blockIdx.y * rpb;
    const long long r1 = min(nrows, r0 + rpb);
    double acc = 0.0;
    if (c < ncols)
        for (long long r = r0 + threadIdx.y; r < r1; r += RTY) acc += in[r * ncols + c];
    red[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0 && c < ncols) {
        double v = 0.0;
        for (int i = 0; i < RTY; i++) v += red[i][threadIdx.x];
        out[(long long)blockIdx.y * ncols + c] = v;
    }
}

// d chi^2 / dG per (t, antenna a, channel k, Jones entry) from the terms the
// forward kernel stored per visibility row (t, baseline, k): the dG_q terms
// of the baselines (p, a), p ascending, then the dG_p terms of (a, q), q
// ascending, summed in the context's precision (the terms carry its rounding
// already; at most na - 1 of them). One thread per (t, a, k), k fastest, so
// that a warp reads one baseline's rows of consecutive channels from one
// plane; the order of the sum is fixed, and the result bit-reproducible.
template <typename T>
__device__ __forceinline__ void add_terms(T (&s)[8], const T *r) {
#pragma unroll
    for (int i = 0; i < 8; i++) s[i] += __ldcs(r + i);
}
template <>
__device__ __forceinline__ void add_terms<float>(float (&s)[8], const float *r) {
    const float4 a = __ldcs(reinterpret_cast<const float4 *>(r)), b = __ldcs(reinterpret_cast<const float4 *>(r) + 1);
    s[0] += a.x; s[1] += a.y; s[2] += a.z; s[3] += a.w;
    s[4] += b.x; s[5] += b.y; s[6] += b.z; s[7] += b.w;
}

template <typename T>
__global__ void __launch_bounds__(256) k_gains_grad(int na, int nchan, long long nbl, long long n, const T *dg,
                                                   long long plane, double *gg, const DevStatus *status) {
    if (inputs_bad(status)) return;
    for (long long i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
        const int k = (int)(i % nchan);
        const long long ta = i / nchan;
        const int a = (int)(ta % na);
        const long long t = ta / na;
        const T *dgp = dg + 8 * (t * nbl * nchan + k);      // plane 0, row (t, baseline 0, k)
        const T *dgq = dgp + plane;                         // plane 1
        const long long bstride = 8ll * nchan;              // the next baseline's row
        T s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int p = 0; p < a; p++) {
            const long long bl = (long long)p * na - (long long)p * (p + 1) / 2 + (a - p - 1);
            add_terms<T>(s, dgq + bl * bstride);
        }
        const long long b0 = (long long)a * na - (long long)a * (a + 1) / 2;   // baseline (a, a + 1)
        for (int q = a + 1; q < na; q++) add_terms<T>(s, dgp + (b0 + (q - a - 1)) * bstride);
        double2 *o = reinterpret_cast<double2 *>(gg + 8 * i);
#pragma unroll
        for (int c = 0; c < 4; c++) o[c] = make_double2((double)s[2 * c], (double)s[2 * c + 1]);
    }
}

}  // namespace

cudaError_t launch_gains_grad(rime_ctx *c, double *grad_gains) {
    const long long n = (long long)c->dims.ntime * c->dims.na * c->dims.nchan;
    if (n == 0) return cudaSuccess;
    if (c->nsm <= 0 && cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
        c->nsm = 152;
    const long long grid = std::min<long long>((n + 255) / 256, (long long)c->nsm * 16);
    const long long plane = 8ll * c->dims.ntime * c->nbl * c->dims.nchan;   // elements per plane
    if (c->dims.precision == RIME_FP64)
        k_gains_grad<double><<<(unsigned)grid, 256, 0, c->stream>>>(c->dims.na, c->dims.nchan, c->nbl, n,
                                                                    static_cast<const double *>(c->d_dgain), plane,
                                                                    grad_gains, c->d_status);
    else
        k_gains_grad<float><<<(unsigned)grid, 256, 0, c->stream>>>(c->dims.na, c->dims.nchan, c->nbl, n,
                                                                  static_cast<const float *>(c->d_dgain), plane,
                                                                  grad_gains, c->d_status);
    return cudaGetLastError();
}

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
    // units with few baselines (one unit of up to 23 antennas): the
    // channel-parallel kernel
    const bool cp = c->dims.na <= 23;
    const int SG = cp ? CPS : f64 ? GCfg<double>::SG : GCfg<float>::SG;
    const int nsch = (c->nsrc + SG - 1) / SG;
    const int chan_group = cp ? (f64 ? CpCfg<double>::CPC : CpCfg<float>::CPC) : 8;
    const int ncg = (c->dims.nchan + chan_group - 1) / chan_group;
    const long long nrows = (long long)c->dims.ntime * ncg * c->ngunits;
    const long long ncols = (long long)c->nsrc * NGRAD;
    const long long rpb = 64;                    // rows per first-level block
    const long long nrb = (nrows + rpb - 1) / rpb;
    const size_t need = (size_t)(nrows + nrb) * ncols;
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
    P.chan_group = chan_group;
    P.ncg = ncg;
    P.nbl = c->nbl;
    P.has_pointing = c->has_pointing;
    P.has_disk = c->has_kind;
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
    if (cp) {
        const int nloc = c->dims.na;   // one diagonal unit
        if (f64) {
            const size_t smem = CpSmem<double>::bytes(nloc, c->has_pointing);
            e = cudaFuncSetAttribute(k_grad_src_cp<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            k_grad_src_cp<double><<<(unsigned)blocks, CPS * CpCfg<double>::CPC, smem, c->stream>>>(P);
        } else {
            const size_t smem = CpSmem<float>::bytes(nloc, c->has_pointing);
            e = cudaFuncSetAttribute(k_grad_src_cp<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            k_grad_src_cp<float><<<(unsigned)blocks, CPS * CpCfg<float>::CPC, smem, c->stream>>>(P);
        }
    } else if (f64) {
        const size_t smem = GSmem<double>::bytes(c->has_pointing);
        e = cudaFuncSetAttribute(k_grad_src<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_grad_src<double><<<(unsigned)blocks, GTHREADS, smem, c->stream>>>(P);
    } else {
        const size_t smem = GSmem<float>::bytes(c->has_pointing);
        auto kern = (c->beam_model != RIME_BEAM_COS3 || c->has_kind) ? k_grad_src_f32x2<true> : k_grad_src_f32x2<false>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)blocks, GTHREADS, smem, c->stream>>>(P);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double *level1 = c->d_gpart + nrows * ncols;
    const dim3 tb(RTX, RTY);
    const unsigned gx = (unsigned)((ncols + RTX - 1) / RTX);
    k_colsum<<<dim3(gx, (unsigned)nrb), tb, 0, c->stream>>>(nrows, ncols, rpb, c->d_gpart, level1, c->d_status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_colsum<<<dim3(gx, 1), tb, 0, c->stream>>>(nrb, ncols, nrb, level1, grad_src, c->d_status);
    return cudaGetLastError();
}

}  // namespace rime
