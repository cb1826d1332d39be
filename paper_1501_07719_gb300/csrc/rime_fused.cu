// rime_fused.cu -- the fused RIME predict + chi^2 kernels (eqs. 1-7).
//
// The paper runs three kernels (Sec. 4.2): EK (Algorithm 1) writes the
// per-antenna factor A_tpsk = E_tpsk K_tpsk to DRAM, B Sum (Algorithm 2)
// reads A for both antennas of each baseline and forms the chi^2 terms, and
// a tree reduction sums them. Here one kernel does all three:
//
//  * a thread block owns one timestep t, one channel k and one "unit" of
//    antenna pairs (up to 64 row antennas against up to 64 (diagonal unit)
//    or 32 (off-diagonal unit) column antennas; na <= 64 is one unit);
//  * per chunk of sources it stages the per-antenna factors A = E K in
//    shared memory, so each is computed once and reused by all ~na/2
//    baselines that share the antenna; the spectral factor (nu/nu_ref)^alpha
//    of eq. 2 multiplies the source's Stokes vector instead;
//  * each thread accumulates a fixed set of baselines with four complex
//    accumulators per baseline, sum_s z_s X_s for X in (I, Q, U, V),
//    z = A_p conj(A_q) g (g the Gaussian shape factor, 1 for points);
//  * the epilogue forms S from the Stokes sums (eq. 2), applies the gains
//    (eq. 1) and either writes V or forms w |V - D|^2 (eq. 7);
//  * chi^2: thread -> warp shuffle -> block (FP64) -> one partial per block;
//    the last block to finish sums the partials in index order, so the
//    result is deterministic.
//
// FP32 kernel: the phase nu tau (up to ~1e2 turns) is formed as a
// double-float product and reduced to [-1/2, 1/2] turns without rounding
// error before sincospi; the FP64 delays come from the upload kernels, so the
// kernel issues no FP64 instruction outside the final reduction.
#include "rime_internal.cuh"
#include "rime_dev.cuh"
#include "rime_fused_common.cuh"

#include <algorithm>
#include <vector>

namespace rime {

// ===========================================================================
// Shared device helpers
// ===========================================================================
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ===========================================================================
// FP64 kernel: 2 x 2 antenna tiles, 32-antenna units
// ===========================================================================
namespace f64 {
constexpr int TP = 2, TQ = 2, NB = TP * TQ;
constexpr int ROWS = 32, COLS = 32;
constexpr int THREADS = 256;
constexpr int SC = 16;
constexpr int ASTRIDE = ROWS + 4;
struct D4 { double x, y, z, w; };
constexpr int NLOCMAX = ROWS + COLS;
constexpr size_t smem_bytes() {
    return 2 * SC * ASTRIDE * sizeof(double2) + 2 * SC * sizeof(D4) + 64 * sizeof(double);
}

__device__ __forceinline__ double2 antenna_factor(double tau, double rho, double alpha, const ChanD &ch) {
    double ph = ch.nu * tau;                 // eq. 3 phase in turns
    double r = ph - round_int_d(ph);
    double sn, cs;
    sincospi(2.0 * r, &sn, &cs);
    double E = beam_E(ch.beam, ch.cnu * rho);   // eq. 4 at C nu[GHz] rho
    double amp = E * exp2(alpha * ch.hlr);   // sqrt of eq. 2's spectral factor
    return make_double2(amp * cs, amp * sn);
}

template <int MODE>
__global__ void __launch_bounds__(THREADS, 1) k_fused_f64(const FusedParams P) {
    constexpr bool CHI2 = MODE != MODE_PREDICT, WRITE = MODE == MODE_PREDICT, GRAD = MODE == MODE_GRAD;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *sA = reinterpret_cast<double2 *>(smem_raw);            // [2][SC][ASTRIDE]
    D4 *sSt = reinterpret_cast<D4 *>(sA + 2 * SC * ASTRIDE);         // [SC]
    D4 *sGq = sSt + SC;                                              // [SC]
    double *sRed = reinterpret_cast<double *>(sGq + SC);             // [64]
    __shared__ int sLast;

    if (inputs_bad(P.status)) return;
    const int tid = threadIdx.x;
    const int u = blockIdx.x % P.nunits;
    const int rest = blockIdx.x / P.nunits;
    const int k = rest % P.nchan;
    const int t = P.t_begin + rest / P.nchan;
    const Unit U = P.units[u];
    const bool active = tid < U.nbody;
    const ChanD ch = reinterpret_cast<const ChanD *>(P.chan)[k];

    int pl = 0, ql = 0;
    if (active) {
        Tile tl = P.tiles[U.tile0 + tid];
        pl = tl.p;
        ql = tl.q;
    }
    const int p0 = U.r0 + pl, q0 = U.c0 + ql;
    const int pend = U.r0 + U.nr, qend = U.c0 + U.nc;
    unsigned mask = 0;
#pragma unroll
    for (int i = 0; i < TP; i++)
#pragma unroll
        for (int j = 0; j < TQ; j++)
            if (active && p0 + i < pend && q0 + j < qend && p0 + i < q0 + j) mask |= 1u << (i * TQ + j);

    double du2[NB], dudv[NB], dv2[NB];
#pragma unroll
    for (int i = 0; i < TP; i++) {
        int pa = min(p0 + i, P.na - 1);
        double up = P.uvw[3 * ((long long)t * P.na + pa)], vp = P.uvw[3 * ((long long)t * P.na + pa) + 1];
#pragma unroll
        for (int j = 0; j < TQ; j++) {
            int qa = min(q0 + j, P.na - 1);
            double du = up - P.uvw[3 * ((long long)t * P.na + qa)];
            double dv = vp - P.uvw[3 * ((long long)t * P.na + qa) + 1];
            du2[i * TQ + j] = du * du;
            dudv[i * TQ + j] = du * dv;
            dv2[i * TQ + j] = dv * dv;
        }
    }

    double acc[NB][8];
#pragma unroll
    for (int b = 0; b < NB; b++)
#pragma unroll
        for (int c = 0; c < 8; c++) acc[b][c] = 0.0;

    const int nloc = U.diag ? U.nr : U.nr + U.nc;
    const double2 *Ar = sA;
    const double2 *Ac = U.diag ? sA : sA + SC * ASTRIDE;
    const double *gauss = reinterpret_cast<const double *>(P.gauss);
    const double *stokes = reinterpret_cast<const double *>(P.stokes) + (long long)t * P.stokes_tstride;
    const double *alpha = reinterpret_cast<const double *>(P.alpha);

    for (int s0 = P.src0; s0 < P.src1; s0 += SC) {
        const int sc = min(SC, P.src1 - s0);
        for (int j = tid; j < sc * nloc; j += THREADS) {
            int s = j / nloc, a = j - s * nloc;
            int ant = a < U.nr ? U.r0 + a : U.c0 + (a - U.nr);
            double2 *dst = (a < U.nr ? sA + a : sA + SC * ASTRIDE + (a - U.nr)) + s * ASTRIDE;
            long long di = ((long long)t * P.nsrc + s0 + s) * P.na + ant;
            *dst = antenna_factor(reinterpret_cast<const double *>(P.tau)[di],
                                  reinterpret_cast<const double *>(P.rho)[di], alpha[s0 + s], ch);
        }
        if (tid < sc) {
            const double *x = stokes + 4 * (long long)(s0 + tid);
            const double *g = gauss + 4 * (long long)(s0 + tid);
            sSt[tid] = D4{x[0], x[1], x[2], x[3]};
            sGq[tid] = D4{g[0] * ch.nu2, g[1] * ch.nu2, g[2] * ch.nu2, g[3]};
        }
        __syncthreads();
        if (active) {
            for (int s = 0; s < sc; s++) {
                const D4 st = sSt[s];
                const D4 gq = sGq[s];
                double2 ap[TP], aq[TQ];
#pragma unroll
                for (int i = 0; i < TP; i++) ap[i] = Ar[s * ASTRIDE + pl + i];
#pragma unroll
                for (int j = 0; j < TQ; j++) aq[j] = Ac[s * ASTRIDE + ql + j];
                const bool is_gauss = gq.w != 0.0, is_disk = gq.w > 1.5;
#pragma unroll
                for (int i = 0; i < TP; i++)
#pragma unroll
                    for (int j = 0; j < TQ; j++) {
                        const int b = i * TQ + j;
                        double zr = ap[i].x * aq[j].x + ap[i].y * aq[j].y;
                        double zi = ap[i].y * aq[j].x - ap[i].x * aq[j].y;
                        if (is_gauss) {
                            // Gaussian exp(e); exponential disk (1 + e)^(-3/2)
                            const double e = gq.x * du2[b] + gq.y * dudv[b] + gq.z * dv2[b];
                            double g;
                            if (is_disk) {
                                const double r = rsqrt(1.0 + e);
                                g = r * r * r;
                            } else {
                                g = exp(e);
                            }
                            zr *= g;
                            zi *= g;
                        }
                        acc[b][0] += zr * st.x; acc[b][1] += zi * st.x;
                        acc[b][2] += zr * st.y; acc[b][3] += zi * st.y;
                        acc[b][4] += zr * st.z; acc[b][5] += zi * st.z;
                        acc[b][6] += zr * st.w; acc[b][7] += zi * st.w;
                    }
            }
        }
        __syncthreads();
    }

    double chi = 0.0;
    const double2 *gains = reinterpret_cast<const double2 *>(P.gains);
    const double2 *data = reinterpret_cast<const double2 *>(P.data);
    const double *weight = reinterpret_cast<const double *>(P.weight);
    double2 *vis = reinterpret_cast<double2 *>(P.vis_out);
    const double2 I2[4] = {make_double2(1, 0), make_double2(0, 0), make_double2(0, 0), make_double2(1, 0)};
#pragma unroll
    for (int i = 0; i < TP; i++)
#pragma unroll
        for (int j = 0; j < TQ; j++) {
            const int b = i * TQ + j;
            if (!((mask >> b) & 1u)) continue;
            const int p = p0 + i, q = q0 + j;
            double2 Sm[4];
            Sm[0] = make_double2(acc[b][0] + acc[b][2], acc[b][1] + acc[b][3]);   // I + Q
            Sm[1] = make_double2(acc[b][4] - acc[b][7], acc[b][5] + acc[b][6]);   // U + iV
            Sm[2] = make_double2(acc[b][4] + acc[b][7], acc[b][5] - acc[b][6]);   // U - iV
            Sm[3] = make_double2(acc[b][0] - acc[b][2], acc[b][1] - acc[b][3]);   // I - Q
            double2 gp[4], gq[4], V[4], tmp[4], gqh[4];
#pragma unroll
            for (int c = 0; c < 4; c++) {
                gp[c] = P.has_gains ? gains[4 * (((long long)t * P.na + p) * P.nchan + k) + c] : I2[c];
                gq[c] = P.has_gains ? gains[4 * (((long long)t * P.na + q) * P.nchan + k) + c] : I2[c];
            }
            mmul(gp, Sm, tmp);      // eq. 1: V = G_p S G_q^H
            mherm(gq, gqh);
            mmul(tmp, gqh, V);
            const long long bl = (long long)p * P.na - (long long)p * (p + 1) / 2 + (q - p - 1);
            const long long row = ((long long)t * P.nbl + bl) * P.nchan + k;
            if constexpr (WRITE) {
#pragma unroll
                for (int c = 0; c < 4; c++) vis[4 * row + c] = V[c];
            }
            if constexpr (CHI2) {
                double2 D[4];
                double r2 = 0.0;
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    D[c] = data[4 * row + c];
                    double dr = V[c].x - D[c].x, di = V[c].y - D[c].y;
                    r2 += dr * dr + di * di;
                }
                const double w = P.has_weight ? weight[row] : 1.0;
                chi += w * r2;
                if constexpr (GRAD) {
                    double2 Y[4], dGp[4], dGq[4];
                    grad_terms<double, double2>(V, Sm, D, w, gp, gq, Y, dGp, dGq);
                    double2 *yo = reinterpret_cast<double2 *>(P.yout) + 4 * row;
#pragma unroll
                    for (int c = 0; c < 4; c++) yo[c] = Y[c];
                    if (P.dgain) {   // this visibility's terms of the gains gradient
                        double2 *go = reinterpret_cast<double2 *>(P.dgain) + 4 * row;
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
        double bsum = block_sum<THREADS>(chi, sRed);
        finish_chi2<THREADS>(bsum, P, sRed, &sLast);
    }
}
}  // namespace f64

// ===========================================================================
// FP32 kernel: 1 x 8 antenna tiles, 256 threads, 2 blocks per SM
// ===========================================================================
namespace f32 {
#ifndef RIME_F32_MIN_BLOCKS
#define RIME_F32_MIN_BLOCKS 2   // resident blocks per SM the register budget is sized for
#endif
#ifndef RIME_F32_SC
#define RIME_F32_SC 32          // sources per staged chunk
#endif
constexpr int THREADS = 256;
constexpr int SC = RIME_F32_SC;      // sources per chunk
constexpr int ROWS = 64, COLS = 32;  // unit shape (off-diagonal: 64 x 32)
constexpr int NLOC = ROWS + COLS;    // antennas staged per unit, at most
constexpr int RSTR = 96;             // staged row of a per-antenna quantity: 64 antennas, 4 pad per 8
constexpr int CSTR = 48;             // the same for the 32 column antennas of off-diagonal units
constexpr int NSLOT = 8;             // baselines per thread

// padded position of antenna a in a staged row of floats: 8 antennas per 12
// floats, so 8-antenna groups start 16-byte aligned in distinct bank groups
__device__ __forceinline__ int apad(int a) { return a + ((a >> 3) << 2); }

// The source sum runs on packed pairs of FP32 values (two FMAs per
// instruction) over pairs of adjacent baseline slots: the per-antenna factors
// are staged as separate real and imaginary rows, so the column factors of
// slots j and j+1 are one 8-byte pair.
//
// Body tiles are 2 x 4: rows p, p + 1 (p even) against columns q .. q + 3
// (q a multiple of 4) of another 8-antenna block, so that per source a thread
// loads its two row factors (two 8-byte loads), its four column factors (two
// 16-byte loads) and the source's scaled Stokes vector (one 16-byte broadcast
// load) for 48 packed FMAs; shared-memory bandwidth, not the FMA pipe, bounds
// tiles that load more per FMA (a 1 x 8 tile needs eight loads).
//
// The Gaussian exponent of baseline (p, q) for source s is the quadratic form
// e = A du^2 + B du dv + C dv^2 of the baseline (du, dv) = x_p - x_q: the
// three products of each baseline are formed once per work item and held in
// registers, and A, B, C (times nu^2) come with the source. A chunk of point
// sources runs a loop without shape factors.
struct Smem {
    float Kx[SC * RSTR], Ky[SC * RSTR];            // staged A = x + iy, row antennas
    float Cx[SC * CSTR], Cy[SC * CSTR];            // column antennas (off-diagonal units)
    float2 rTau[SC * NLOC];     // prefetched delays (hi, lo) of the next chunk
    float rRho[SC * NLOC];      // prefetched beam radii
    float4 rSt[SC];             // prefetched Stokes
    float4 rG[SC];              // prefetched Gaussian coefficients
    float rAl[SC];              // prefetched spectral indices
    float4 St[SC];              // (I, Q, U, V) scaled (see staging)
    float4 Gq[SC];              // shape form (A, B, C) nu^2 of the baseline (du, dv); w: kind
                                // (0 point, 1 Gaussian, 2 exponential disk)
    float2 uv[NLOC];            // antenna (u, v) at this timestep, unit order
    double red[32];
};

// Local (row, column) antennas of slot j of a thread tile; rev = 1 when the
// tile forms the pair in the order (column, row) and the accumulated sums
// must be conjugated. Body tile: rows p, p + 1 against columns q .. q + 3,
// slot j = 4 r + c. Head tile: with x_i = b0 + ((fold + i) mod 8), slots 0..3
// pair x_0 with x_1..x_4 and slots 4..6 pair x_4 with x_5..x_7; slot 7 is
// unused.
__device__ __forceinline__ void slot_pair(const Tile &tl, int role, int j, int &p, int &q, bool &rev) {
    if (role == 2) {
        const int b0 = tl.p, r = tl.fold;
        const int a = j < 4 ? 0 : 4;
        const int xa = b0 + ((r + a) & 7), xb = b0 + ((r + j + 1) & 7);
        rev = xa > xb;
        p = rev ? xb : xa;
        q = rev ? xa : xb;
    } else {
        p = tl.p + (j >> 2);
        q = tl.q + (j & 3);
        rev = false;
    }
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Two slots: z = a conj(b) for rows (ax, ay) (as pairs over the two slots)
// and columns (bx, by), optionally times the shape factors, accumulated
// against (I, Q, U, V): acc.re holds the real parts of the two slots' sums,
// acc.im the imaginary parts.
struct Pair {
    float2 re[4], im[4];
};
template <bool SHAPE>
__device__ __forceinline__ void accumulate2(Pair &acc, float2 ax, float2 ay, float2 bx, float2 by, float2 g,
                                            const float2 (&X)[4]) {
    float2 zr = __ffma2_rn(ax, bx, __fmul2_rn(ay, by));
    float2 zi = __ffma2_rn(ay, bx, __fmul2_rn(f2(-ax.x, -ax.y), by));
    if (SHAPE) {
        zr = __fmul2_rn(zr, g);
        zi = __fmul2_rn(zi, g);
    }
#pragma unroll
    for (int c = 0; c < 4; c++) {
        acc.re[c] = __ffma2_rn(zr, X[c], acc.re[c]);
        acc.im[c] = __ffma2_rn(zi, X[c], acc.im[c]);
    }
}
// Shape factors of two slots from the quadratic form of their baselines,
// e = A du^2 + B du dv + C dv^2: Gaussian 2^e (log2 units), exponential disk
// (1 + e)^(-3/2) (only in the kernels built for general sky models).
struct Geo {
    float2 d2[4], dd[4], v2[4];   // (du^2, du dv, dv^2) of the slot pairs
};
template <bool GENERAL>
__device__ __forceinline__ float2 shape2(const float4 &q, const Geo &G, int h) {
    const float2 e = __ffma2_rn(f2(q.x, q.x), G.d2[h], __ffma2_rn(f2(q.y, q.y), G.dd[h], __fmul2_rn(f2(q.z, q.z), G.v2[h])));
    if (GENERAL && q.w > 1.5f) {
        const float r0 = rsqrtf(1.0f + e.x), r1 = rsqrtf(1.0f + e.y);
        return f2(r0 * r0 * r0, r1 * r1 * r1);
    }
    return f2(ex2_approx(e.x), ex2_approx(e.y));
}

// One chunk of sources for a 2 x 4 body tile (rows at ip, columns at iq of
// the staged rows; cstr the column rows' stride).
template <bool SHAPE, bool GENERAL>
__device__ __forceinline__ void body_chunk(Pair (&acc)[NSLOT / 2], const Smem &S, const float *KxC, const float *KyC,
                                           int cstr, int ip, int iq, int sc, const Geo &G) {
#pragma unroll 2
    for (int s = 0; s < sc; s++) {
        const float2 kr = *reinterpret_cast<const float2 *>(S.Kx + s * RSTR + ip);
        const float2 ki = *reinterpret_cast<const float2 *>(S.Ky + s * RSTR + ip);
        const float4 bx4 = *reinterpret_cast<const float4 *>(KxC + s * cstr + iq);
        const float4 by4 = *reinterpret_cast<const float4 *>(KyC + s * cstr + iq);
        const float4 x = S.St[s];
        const float2 X[4] = {f2(x.x, x.x), f2(x.y, x.y), f2(x.z, x.z), f2(x.w, x.w)};
        const float2 bx[2] = {f2(bx4.x, bx4.y), f2(bx4.z, bx4.w)}, by[2] = {f2(by4.x, by4.y), f2(by4.z, by4.w)};
        float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
        if (SHAPE) q = S.Gq[s];
#pragma unroll
        for (int h = 0; h < 4; h++) {
            const int r = h >> 1, c = h & 1;
            const float xr = r ? kr.y : kr.x, yr = r ? ki.y : ki.x;
            const float2 g = SHAPE ? shape2<GENERAL>(q, G, h) : f2(1.f, 1.f);
            accumulate2<SHAPE>(acc[h], f2(xr, xr), f2(yr, yr), bx[c], by[c], g, X);
        }
    }
}

// One chunk for a head tile: pairs inside one 8-antenna block, rows x_0 and x_4.
template <bool SHAPE, bool GENERAL>
__device__ __forceinline__ void head_chunk(Pair (&acc)[NSLOT / 2], const Smem &S, const Tile &tl, int sc,
                                           const Geo &G) {
    const int hb = apad(tl.p), r = tl.fold;
    int ho[8];   // shared-memory offsets of x_0..x_7 (one 8-antenna block)
#pragma unroll
    for (int i = 0; i < 8; i++) ho[i] = hb + ((r + i) & 7);
#pragma unroll 2
    for (int s = 0; s < sc; s++) {
        const float4 x = S.St[s];
        const float2 X[4] = {f2(x.x, x.x), f2(x.y, x.y), f2(x.z, x.z), f2(x.w, x.w)};
        const float *kx = S.Kx + s * RSTR, *ky = S.Ky + s * RSTR;
        const float2 ax[2] = {f2(kx[ho[0]], kx[ho[0]]), f2(kx[ho[4]], kx[ho[4]])};
        const float2 ay[2] = {f2(ky[ho[0]], ky[ho[0]]), f2(ky[ho[4]], ky[ho[4]])};
        float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
        if (SHAPE) q = S.Gq[s];
#pragma unroll
        for (int h = 0; h < 4; h++) {
            const int r2 = h < 2 ? 0 : 1;
            const int c0 = ho[2 * h + 1], c1 = h < 3 ? ho[2 * h + 2] : ho[0];   // slot 7 unused
            const float2 bx = f2(kx[c0], kx[c1]), by = f2(ky[c0], ky[c1]);
            const float2 g = SHAPE ? shape2<GENERAL>(q, G, h) : f2(1.f, 1.f);
            accumulate2<SHAPE>(acc[h], ax[r2], ay[r2], bx, by, g, X);
        }
    }
}

// One work item: timestep t, channel k, antenna unit u, sources [sb, se).
// Returns the block's chi^2 (in thread 0; chi^2 modes only). GENERAL = false
// builds the kernel for eq. 4's cos^3 beam and point / Gaussian sources
// alone; GENERAL = true takes the beam model from the channel constants and
// the exponential disks too. The kernel runs at its register limit: a
// run-time choice (the Bessel function's code beside cos^3 in the staging
// loop) cost the common case 1.5 %.
// Long source lists: every SEG sources the thread's 64 FP32 sums are added
// into running sums in a per-block scratch (a second FP32 set would not fit
// the registers) with the rounding error of each addition kept in a low part
// (two-sum), and restart at zero; so no FP32 sum runs over more than SEG terms
// (4096 sequential FP32 additions at |V| ~ 1e2 Jy would round away more than
// the chi^2 of a 0.01 Jy residual tolerates). Scratch layout per block:
// [hi | lo][64][THREADS] floats.
constexpr int SEG = 240;
__device__ __forceinline__ float *seg_base(const FusedParams &P) {
    return P.segsum + (size_t)blockIdx.x * 2 * 64 * THREADS + threadIdx.x;
}
__device__ __forceinline__ void zero_sums(Pair (&acc)[NSLOT / 2]) {
#pragma unroll
    for (int h = 0; h < NSLOT / 2; h++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[h].re[c] = acc[h].im[c] = f2(0.f, 0.f);
}
template <typename F>
__device__ __forceinline__ void each_sum(Pair (&acc)[NSLOT / 2], F &&f) {
#pragma unroll
    for (int h = 0; h < NSLOT / 2; h++)
#pragma unroll
        for (int c = 0; c < 4; c++) {
            f(16 * h + 4 * c + 0, acc[h].re[c].x);
            f(16 * h + 4 * c + 1, acc[h].re[c].y);
            f(16 * h + 4 * c + 2, acc[h].im[c].x);
            f(16 * h + 4 * c + 3, acc[h].im[c].y);
        }
}
__device__ __forceinline__ void fold_segment(const FusedParams &P, Pair (&acc)[NSLOT / 2], bool held) {
    float *hi = seg_base(P), *lo = hi + 64 * THREADS;
    each_sum(acc, [&](int f, float &v) {
        if (!held) {
            hi[f * THREADS] = v;
            lo[f * THREADS] = 0.f;
        } else {
            const float h = hi[f * THREADS];
            const float sm = h + v, bb = sm - h;
            lo[f * THREADS] += (h - (sm - bb)) + (v - bb);
            hi[f * THREADS] = sm;
        }
        v = 0.f;
    });
}
__device__ __forceinline__ void unfold_segments(const FusedParams &P, Pair (&acc)[NSLOT / 2]) {
    const float *hi = seg_base(P), *lo = hi + 64 * THREADS;
    each_sum(acc, [&](int f, float &v) { v = hi[f * THREADS] + (lo[f * THREADS] + v); });
}

// SUM: the source sum of [sb, se) is added into acc (the caller zeroes it);
// EPI: the epilogue of the item from acc (sb, se unused). The kernel of one
// launch per item runs both in one body (lists of up to 2 SEG sources); the
// persistent kernels sum through source_sum and then run the epilogue.
template <int MODE, bool GENERAL, bool SUM, bool EPI>
__device__ __forceinline__ double fused_item(const FusedParams &P, Smem &S, int t, int k, int u, int sb, int se,
                                             Pair (&acc)[NSLOT / 2]) {
    constexpr bool CHI2 = MODE != MODE_PREDICT, WRITE = MODE == MODE_PREDICT, GRAD = MODE == MODE_GRAD;
    const int tid = threadIdx.x;
    const Unit U = P.units[u];
    const ChanF ch = reinterpret_cast<const ChanF *>(P.chan)[k];
    const int nloc = U.diag ? U.nr : U.nr + U.nc;
    // this thread's items (s, a) of a chunk: start and stride in (s, a)
    const int it_s0 = tid / nloc, it_a0 = tid - (tid / nloc) * nloc;
    const int it_ds = THREADS / nloc, it_da = THREADS - (THREADS / nloc) * nloc;
    const float2 *tau = reinterpret_cast<const float2 *>(P.tau);
    const float *rho = reinterpret_cast<const float *>(P.rho);
    const float *stokes = reinterpret_cast<const float *>(P.stokes) + (long long)t * P.stokes_tstride;
    const float *gauss = reinterpret_cast<const float *>(P.gauss);
    const float *alpha = reinterpret_cast<const float *>(P.alpha);

    // prefetch of one chunk's per-(s, a) delays and per-source constants
    auto issue = [&](int s0) {
        const int sc = min(SC, se - s0);
        for (int s = it_s0, a = it_a0; s < sc;) {
            int ant = a < U.nr ? U.r0 + a : U.c0 + (a - U.nr);
            long long di = ((long long)t * P.nsrc + s0 + s) * P.na + ant;
            cp_async8(&S.rTau[s * NLOC + a], tau + di);
            cp_async4(&S.rRho[s * NLOC + a], rho + di);
            a += it_da;
            s += it_ds;
            if (a >= nloc) { a -= nloc; s += 1; }
        }
        if (tid < sc) {
            cp_async16(&S.rSt[tid], stokes + 4 * (long long)(s0 + tid));
            cp_async16(&S.rG[tid], gauss + 4 * (long long)(s0 + tid));
            cp_async4(&S.rAl[tid], alpha + s0 + tid);
        }
        cp_async_commit();
    };
    if constexpr (SUM) {
        if (se > sb) issue(sb);
        for (int a = tid; a < nloc; a += THREADS) {
            int ant = a < U.nr ? U.r0 + a : U.c0 + (a - U.nr);
            float4 x = P.uvw_f[(long long)t * P.na + ant];
            S.uv[a] = f2(x.x, x.y);
        }
    }

    // ---- this thread's 8 baselines ----
    const int hbase = (U.nbody + 31) & ~31;
    int role = 0;   // 0 idle, 1 body, 2 head
    Tile tl{0, 0, 0, 0};
    if (tid < U.nbody) {
        role = 1;
        tl = P.tiles[U.tile0 + tid];
    } else if (tid >= hbase && tid - hbase < U.nhead) {
        role = 2;
        tl = P.tiles[U.tile0 + U.nbody + (tid - hbase)];
    }
    const int qlim = U.diag ? U.nr : U.nc;
    unsigned mask = 0;
#pragma unroll
    for (int j = 0; j < NSLOT; j++) {
        int pj, qj;
        bool rev;
        slot_pair(tl, role, j, pj, qj, rev);
        bool ok = role != 0 && pj < U.nr && qj < qlim && U.r0 + pj < U.c0 + qj;
        if (role == 2 && j == 7) ok = false;
        if (ok) mask |= 1u << j;
    }
    const float *KxC = U.diag ? S.Kx : S.Cx;
    const float *KyC = U.diag ? S.Ky : S.Cy;
    const int cstr = U.diag ? RSTR : CSTR;
    const bool pointing = P.has_pointing != 0;

    Geo geo;   // the baselines' (du^2, du dv, dv^2), filled after the first barrier

    for (int s0 = sb; SUM && s0 < se; s0 += SC) {
        const int sc = min(SC, se - s0);
        cp_async_wait_all();
        __syncthreads();
        // ---- stage the per-antenna factors of the chunk (Algorithm 1) ----
        // With pointing errors A = E K per antenna; without, every antenna sees
        // the same beam E_s and A = K, the E_s^2 of the baseline going into the
        // source's Stokes scale below.
        for (int s = it_s0, a = it_a0; s < sc;) {
            float2 v = phase_factor(S.rTau[s * NLOC + a], ch);
            if (pointing) {
                float E = beam_E(GENERAL ? ch.beam : RIME_BEAM_COS3, ch.cnu * S.rRho[s * NLOC + a]);
                v.x *= E;
                v.y *= E;
            }
            if (a < U.nr) {
                const int o = s * RSTR + apad(a);
                S.Kx[o] = v.x; S.Ky[o] = v.y;
            } else {
                const int o = s * CSTR + apad(a - U.nr);
                S.Cx[o] = v.x; S.Cy[o] = v.y;
            }
            a += it_da;
            s += it_ds;
            if (a >= nloc) { a -= nloc; s += 1; }
        }
        bool ext = false;
        if (tid < sc) {
            // spectral factor (nu / nu_ref)^alpha = 2^(2 alpha hlr) of eq. 2
            float f = exp2f(2.0f * S.rAl[tid] * ch.hlr);
            if (!pointing) {
                float E = beam_E(GENERAL ? ch.beam : RIME_BEAM_COS3, ch.cnu * S.rRho[tid * NLOC]);
                f *= E * E;
            }
            float4 st = S.rSt[tid];
            S.St[tid] = make_float4(st.x * f, st.y * f, st.z * f, st.w * f);
            const float4 g = S.rG[tid];
            // the shape form in log2 units times nu^2 (Gaussians), or times nu^2
            // with the disk's constant (disks)
            S.Gq[tid] = make_float4(g.x * ch.nu2, g.y * ch.nu2, g.z * ch.nu2, g.w);
            ext = g.w != 0.f;
        }
        // the chunk has an extended source if any thread saw one
        ext = __syncthreads_or(ext) != 0;
        if (s0 + SC < se) issue(s0 + SC);
        if (s0 == sb) {
            // (du^2, du dv, dv^2) of each slot's baseline, in slot pairs
            float d2[NSLOT], dd[NSLOT], v2[NSLOT];
#pragma unroll
            for (int j = 0; j < NSLOT; j++) {
                int pj, qj;
                bool rev;
                slot_pair(tl, role, j, pj, qj, rev);
                const bool ok = (mask >> j) & 1u;
                const float2 a = S.uv[ok ? pj : 0], b = S.uv[ok ? (U.diag ? qj : U.nr + qj) : 0];
                const float du = a.x - b.x, dv = a.y - b.y;
                d2[j] = du * du;
                dd[j] = du * dv;
                v2[j] = dv * dv;
            }
#pragma unroll
            for (int h = 0; h < 4; h++) {
                geo.d2[h] = f2(d2[2 * h], d2[2 * h + 1]);
                geo.dd[h] = f2(dd[2 * h], dd[2 * h + 1]);
                geo.v2[h] = f2(v2[2 * h], v2[2 * h + 1]);
            }
        }

        // ---- source sum for this thread's baselines (Algorithm 2) ----
        if (role == 1) {
            const int ip = apad(tl.p), iq = apad(tl.q);
            if (ext) body_chunk<true, GENERAL>(acc, S, KxC, KyC, cstr, ip, iq, sc, geo);
            else body_chunk<false, GENERAL>(acc, S, KxC, KyC, cstr, ip, iq, sc, geo);
        } else if (role == 2) {
            if (ext) head_chunk<true, GENERAL>(acc, S, tl, sc, geo);
            else head_chunk<false, GENERAL>(acc, S, tl, sc, geo);
        }
    }
    if constexpr (!EPI) return 0.0;

    // ---- epilogue: S (eq. 2), gains (eq. 1), chi^2 terms (eq. 7) ----
    float chi = 0.f;
    const float2 *gains = reinterpret_cast<const float2 *>(P.gains);
    const float2 *data = reinterpret_cast<const float2 *>(P.data);
    const float *weight = reinterpret_cast<const float *>(P.weight);
    float2 *vis = reinterpret_cast<float2 *>(P.vis_out);
    const float2 I2[4] = {f2(1.f, 0.f), f2(0.f, 0.f), f2(0.f, 0.f), f2(1.f, 0.f)};
#pragma unroll
    for (int j = 0; j < NSLOT; j++) {
        if (!((mask >> j) & 1u)) continue;
        int pj, qj;
        bool rev;
        slot_pair(tl, role, j, pj, qj, rev);
        const int p = U.r0 + pj, q = U.c0 + qj;
        const Pair &a = acc[j >> 1];
        const bool hi = j & 1;
        // the sums of z for the reversed pair are the conjugates
        const float cj = rev ? -1.f : 1.f;
        const float Ir = hi ? a.re[0].y : a.re[0].x, Ii = cj * (hi ? a.im[0].y : a.im[0].x);
        const float Qr = hi ? a.re[1].y : a.re[1].x, Qi = cj * (hi ? a.im[1].y : a.im[1].x);
        const float Ur = hi ? a.re[2].y : a.re[2].x, Ui = cj * (hi ? a.im[2].y : a.im[2].x);
        const float Vr = hi ? a.re[3].y : a.re[3].x, Vi = cj * (hi ? a.im[3].y : a.im[3].x);
        float2 Sm[4];
        Sm[0] = make_float2(Ir + Qr, Ii + Qi);   // I + Q
        Sm[1] = make_float2(Ur - Vi, Ui + Vr);   // U + iV
        Sm[2] = make_float2(Ur + Vi, Ui - Vr);   // U - iV
        Sm[3] = make_float2(Ir - Qr, Ii - Qi);   // I - Q
        float2 gp[4], gq[4];
        if (P.has_gains) {
            const float4 *gp4 = reinterpret_cast<const float4 *>(gains + 4 * (((long long)t * P.na + p) * P.nchan + k));
            const float4 *gq4 = reinterpret_cast<const float4 *>(gains + 4 * (((long long)t * P.na + q) * P.nchan + k));
            const float4 a01 = gp4[0], a23 = gp4[1], b01 = gq4[0], b23 = gq4[1];
            gp[0] = f2(a01.x, a01.y); gp[1] = f2(a01.z, a01.w); gp[2] = f2(a23.x, a23.y); gp[3] = f2(a23.z, a23.w);
            gq[0] = f2(b01.x, b01.y); gq[1] = f2(b01.z, b01.w); gq[2] = f2(b23.x, b23.y); gq[3] = f2(b23.z, b23.w);
        } else {
#pragma unroll
            for (int c = 0; c < 4; c++) gp[c] = gq[c] = I2[c];
        }
        float2 V[4], tmp[4], gqh[4];
        mmul(gp, Sm, tmp);      // eq. 1: V = G_p S G_q^H
        mherm(gq, gqh);
        mmul(tmp, gqh, V);
        const long long bl = (long long)p * P.na - (long long)p * (p + 1) / 2 + (q - p - 1);
        const long long row = ((long long)t * P.nbl + bl) * P.nchan + k;
        if constexpr (WRITE) {
            float4 *o = reinterpret_cast<float4 *>(vis + 4 * row);
            o[0] = make_float4(V[0].x, V[0].y, V[1].x, V[1].y);
            o[1] = make_float4(V[2].x, V[2].y, V[3].x, V[3].y);
        }
        if constexpr (CHI2) {
            const float4 *d4 = reinterpret_cast<const float4 *>(data + 4 * row);
            const float4 d01 = d4[0], d23 = d4[1];
            const float2 D[4] = {f2(d01.x, d01.y), f2(d01.z, d01.w), f2(d23.x, d23.y), f2(d23.z, d23.w)};
            float r2 = 0.f;
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const float dr = V[c].x - D[c].x, di = V[c].y - D[c].y;
                r2 += dr * dr + di * di;
            }
            const float w = P.has_weight ? weight[row] : 1.f;
            chi += w * r2;
            if constexpr (GRAD) {
                float2 Y[4], dGp[4], dGq[4];
                grad_terms<float, float2>(V, Sm, D, w, gp, gq, Y, dGp, dGq);
                float4 *yo = reinterpret_cast<float4 *>(reinterpret_cast<float2 *>(P.yout) + 4 * row);
                yo[0] = make_float4(Y[0].x, Y[0].y, Y[1].x, Y[1].y);
                yo[1] = make_float4(Y[2].x, Y[2].y, Y[3].x, Y[3].y);
                if (P.dgain) {   // this visibility's terms of the gains gradient
                    float4 *go = reinterpret_cast<float4 *>(P.dgain) + 2 * row;
                    const long long plane = 2ll * P.ntime * P.nbl * P.nchan;
                    go[0] = make_float4(dGp[0].x, dGp[0].y, dGp[1].x, dGp[1].y);
                    go[1] = make_float4(dGp[2].x, dGp[2].y, dGp[3].x, dGp[3].y);
                    go[plane] = make_float4(dGq[0].x, dGq[0].y, dGq[1].x, dGq[1].y);
                    go[plane + 1] = make_float4(dGq[2].x, dGq[2].y, dGq[3].x, dGq[3].y);
                }
            }
        }
    }
    double bsum = 0.0;
    if constexpr (CHI2) {
        // thread and warp sums in FP32 (positive terms), block in FP64
        float w = chi;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
        bsum = block_sum<THREADS>((threadIdx.x & 31) == 0 ? (double)w : 0.0, S.red);
    }
    return bsum;
}

// The source sum of [sb, se) into acc: one FP32 sum for lists of up to
// 2 SEG sources, else segments of SEG sources folded into the block's running
// sums (P.segsum) between them. Every kernel that sums a source list goes
// through here, so a list's sums do not depend on the kernel that ran it.
template <int MODE, bool GENERAL>
__device__ __forceinline__ void source_sum(const FusedParams &P, Smem &S, int t, int k, int u, int sb, int se,
                                           Pair (&acc)[NSLOT / 2]) {
    const int len = se - sb > 2 * SEG ? SEG : se - sb;
    bool held = false;
    for (int s0 = sb;; s0 += len) {
        const int s1 = min(s0 + len, se);
        zero_sums(acc);
        fused_item<MODE, GENERAL, true, false>(P, S, t, k, u, s0, s1, acc);
        if (s1 >= se) break;
        fold_segment(P, acc, held);
        held = true;
    }
    if (held) unfold_segments(P, acc);
}

template <int MODE, bool GENERAL>
__global__ void __launch_bounds__(THREADS, RIME_F32_MIN_BLOCKS) k_fused_f32(const FusedParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>(smem_raw);
    __shared__ int sLast;
    if (inputs_bad(P.status)) return;
    const int u = blockIdx.x % P.nunits;
    const int rest = blockIdx.x / P.nunits;
    const int k = rest % P.nchan;
    const int t = P.t_begin + rest / P.nchan;
    Pair acc[NSLOT / 2];
    zero_sums(acc);
    const double bsum = fused_item<MODE, GENERAL, true, true>(P, S, t, k, u, P.src0, P.src1, acc);
    if constexpr (MODE != MODE_PREDICT) finish_chi2<THREADS>(bsum, P, S.red, &sLast);
}

// Long source lists: a persistent grid (its blocks' running sums fit a
// scratch of one slot per block) over the items of k_fused_f32; one partial
// per item at the item's index, the last block adds them in index order.
template <int MODE, bool GENERAL>
__global__ void __launch_bounds__(THREADS, RIME_F32_MIN_BLOCKS) k_fused_f32_seg(const FusedParams P, long long nitems) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>(smem_raw);
    __shared__ int sLast;
    if (inputs_bad(P.status)) return;
    for (long long item = blockIdx.x; item < nitems; item += gridDim.x) {
        __syncthreads();   // the previous item is done with the shared buffers
        const int u = (int)(item % P.nunits);
        const long long rest = item / P.nunits;
        const int k = (int)(rest % P.nchan);
        const int t = P.t_begin + (int)(rest / P.nchan);
        Pair acc[NSLOT / 2];
        source_sum<MODE, GENERAL>(P, S, t, k, u, P.src0, P.src1, acc);
        const double bsum = fused_item<MODE, GENERAL, false, true>(P, S, t, k, u, P.src0, P.src1, acc);
        if (MODE != MODE_PREDICT && threadIdx.x == 0) P.partials[item] = bsum;
    }
    if constexpr (MODE == MODE_PREDICT) return;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned ticket = atomicAdd(P.counter, 1u);
        sLast = ticket == gridDim.x - 1;
    }
    __syncthreads();
    if (!sLast) return;
    __threadfence();
    double s = 0.0;
    for (long long i = threadIdx.x; i < nitems; i += THREADS) s += __ldcg(&P.partials[i]);
    const double tot = block_sum<THREADS>(s, S.red);
    if (threadIdx.x == 0) {
        *P.result = tot;
        *P.counter = 0u;
    }
}

// Batched chi^2: many source sets against one observation in one persistent
// launch. A work item is (t, channel group, unit, group of sets); blocks take
// items from a counter. Items run in (t, channel group, unit) order and,
// within it, sets by rank (largest first by default), so the sets of one
// item share their data, weights and gains, which the later sets read from
// L1. One partial per (set, t, channel, unit): the sums do not depend on the
// schedule.
template <bool GENERAL>
__global__ void __launch_bounds__(THREADS, RIME_F32_MIN_BLOCKS) k_batched_f32(const FusedParams P, const BatchParams B) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>(smem_raw);
    __shared__ long long sItem;
    if (inputs_bad(P.status)) return;
    for (;;) {
        __syncthreads();   // the previous item is done with the shared buffers
        if (threadIdx.x == 0) sItem = (long long)atomicAdd(B.counter, 1ull);
        __syncthreads();
        const long long item = sItem;
        if (item >= B.nitems) break;
        const int w = (int)(item / B.ngroups);
        const int g = (int)(item - (long long)w * B.ngroups);
        const int u = w % P.nunits;
        const int rest = w / P.nunits;
        const int kc = rest % B.nkc;
        const int t = rest / B.nkc;
        const int k1 = min(P.nchan, (kc + 1) * B.cpi);
        const int r1 = min(B.nsets, (g + 1) * B.gsets);
        for (int rank = g * B.gsets; rank < r1; rank++) {
            const int j = B.order[rank];
            for (int k = kc * B.cpi; k < k1; k++) {
                Pair acc[NSLOT / 2];
                source_sum<MODE_CHI2, GENERAL>(P, S, t, k, u, B.offsets[j], B.offsets[j + 1], acc);
                const double bsum = fused_item<MODE_CHI2, GENERAL, false, true>(P, S, t, k, u, 0, 0, acc);
                if (threadIdx.x == 0)
                    B.partials[(long long)j * B.per_set + ((long long)t * P.nchan + k) * P.nunits + u] = bsum;
                __syncthreads();
            }
        }
    }
}
}  // namespace f32

// chi2[j] = sum of set j's per-item partials, in index order.
__global__ void k_set_sums(int per_set, const double *partials, double *chi2, const DevStatus *status) {
    __shared__ double red[32];
    if (inputs_bad(status)) return;
    const int j = blockIdx.x;
    double acc = 0.0;
    for (int i = threadIdx.x; i < per_set; i += 256) acc += partials[(long long)j * per_set + i];
    const double tot = block_sum<256>(acc, red);
    if (threadIdx.x == 0) chi2[j] = tot;
}

// ===========================================================================
// Host side: work units and launch
// ===========================================================================
// Emits the units and tiles of one precision through sink.unit(Unit) and
// sink.tile(Tile) (each returns false when its storage is full).
template <typename Sink>
static bool emit_units(int na, int precision, Sink &sink) {
    int ntile = 0;
    auto tile = [&](int p, int q, int fold) {
        ntile++;
        return sink.tile(Tile{(uint8_t)p, (uint8_t)q, (uint8_t)fold, 0});
    };
    if (precision == RIME_FP64) {
        using namespace f64;
        for (int r0 = 0; r0 < na; r0 += ROWS) {
            int nr = std::min(ROWS, na - r0);
            Unit d{r0, r0, nr, nr, ntile, 0, 0, 1};
            for (int pi = 0; pi < nr; pi += TP)
                for (int qj = 0; qj < nr; qj += TQ)
                    if (qj + TQ - 1 > pi && !tile(pi, qj, 0)) return false;
            d.nbody = ntile - d.tile0;
            if (!sink.unit(d)) return false;
            for (int c0 = r0 + ROWS; c0 < na; c0 += COLS) {
                int nc = std::min(COLS, na - c0);
                Unit o{r0, c0, nr, nc, ntile, 0, 0, 0};
                for (int pi = 0; pi < nr; pi += TP)
                    for (int qj = 0; qj < nc; qj += TQ)
                        if (!tile(pi, qj, 0)) return false;
                o.nbody = ntile - o.tile0;
                if (!sink.unit(o)) return false;
            }
        }
        return true;
    }
    using namespace f32;
    for (int r0 = 0; r0 < na; r0 += ROWS) {
        int nr = std::min(ROWS, na - r0);
        int nblk = (nr + 7) / 8;
        // diagonal unit: 2 x 4 body tiles (rows p, p + 1; columns q .. q + 3)
        // for column blocks past the rows' own 8-block, then 4 head tiles per
        // 8-block for the pairs inside the block
        Unit d{r0, r0, nr, nr, ntile, 0, 0, 1};
        for (int p = 0; p < nr; p += 2)
            for (int q = 8 * (p / 8 + 1); q < nr; q += 4)
                if (!tile(p, q, 0)) return false;
        d.nbody = ntile - d.tile0;
        for (int f = 0; f < 4; f++)
            for (int m = 0; m < nblk; m++)
                if (!tile(8 * m, 8 * m, f)) return false;
        d.nhead = ntile - d.tile0 - d.nbody;
        if (!sink.unit(d)) return false;
        for (int c0 = r0 + ROWS; c0 < na; c0 += COLS) {
            int nc = std::min(COLS, na - c0);
            Unit o{r0, c0, nr, nc, ntile, 0, 0, 0};
            for (int p = 0; p < nr; p += 2)
                for (int q = 0; q < nc; q += 4)
                    if (!tile(p, q, 0)) return false;
            o.nbody = ntile - o.tile0;
            if (!sink.unit(o)) return false;
        }
    }
    return true;
}

void build_units(int na, int precision, std::vector<Unit> &units, std::vector<Tile> &tiles) {
    struct {
        std::vector<Unit> *u;
        std::vector<Tile> *t;
        bool unit(const Unit &x) { u->push_back(x); return true; }
        bool tile(const Tile &x) { t->push_back(x); return true; }
    } sink{&units, &tiles};
    units.clear();
    tiles.clear();
    emit_units(na, precision, sink);
}

int build_units_fixed(int na, int precision, Unit *units, int max_units, Tile *tiles, int max_tiles,
                      int *ntiles) {
    struct {
        Unit *u;
        Tile *t;
        int mu, mt, nu = 0, nt = 0;
        bool unit(const Unit &x) { if (nu >= mu) return false; u[nu++] = x; return true; }
        bool tile(const Tile &x) { if (nt >= mt) return false; t[nt++] = x; return true; }
    } sink{units, tiles, max_units, max_tiles};
    if (!emit_units(na, precision, sink)) return -1;
    *ntiles = sink.nt;
    return sink.nu;
}

int fused_blocks(const rime_ctx *c) { return c->dims.ntime * c->dims.nchan * c->nunits; }

template <typename K>
static cudaError_t launch_k(K kernel, const FusedParams &P, int blocks, int threads, size_t smem,
                            cudaStream_t stream) {
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kernel<<<blocks, threads, smem, stream>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_fused(rime_ctx *c, void *vis_out, double *result, bool chi2) {
    return launch_fused_mode(c, chi2 ? MODE_CHI2 : MODE_PREDICT, vis_out, result, nullptr, nullptr);
}

void fill_fused_params(const rime_ctx *c, FusedParams &P, void *vis_out, double *result, void *yout,
                       void *dgain) {
    P.na = c->dims.na;
    P.ntime = c->dims.ntime;
    P.nchan = c->dims.nchan;
    P.nsrc = c->nsrc;
    P.nbl = c->nbl;
    P.stokes_tstride = c->time_varying ? 4 * c->nsrc : 0;
    P.nchp = c->dims.nchan;
    P.nunits = c->nunits;
    P.has_gains = c->has_gains;
    P.has_weight = c->has_weight;
    P.has_pointing = c->has_pointing;
    P.units = c->d_units;
    P.tiles = c->d_tiles;
    P.chan = c->d_chan;
    P.uvw = c->d_uvw;
    P.uvw_f = reinterpret_cast<const float4 *>(c->d_uvw_f);
    P.stokes = c->d_stokes;
    P.gauss = c->d_gauss;
    P.alpha = c->d_alpha;
    P.tau = c->d_tau;
    P.rho = c->d_rho;
    P.gains = c->d_gains;
    P.data = c->d_data;
    P.weight = c->d_weight;
    P.vis_out = vis_out;
    P.partials = c->d_partials;
    P.counter = c->d_counter;
    P.result = result;
    P.status = c->d_status;
    P.yout = yout;
    P.dgain = dgain;
    P.src0 = 0;
    P.src1 = c->nsrc;
    P.t_begin = 0;
}

cudaError_t launch_fused_mode(rime_ctx *c, int mode, void *vis_out, double *result, void *yout,
                              void *dgain) {
    FusedParams P{};
    fill_fused_params(c, P, vis_out, result, yout, dgain);
    return launch_tiled_params(c, mode, P, fused_blocks(c));
}

long long seg_source_threshold() { return 2 * f32::SEG; }
size_t seg_scratch_per_block() { return (size_t)2 * 64 * f32::THREADS * sizeof(float); }

// The running sums of long FP32 source lists: one scratch slot per resident
// block of a persistent grid (the context's own, or the caller's in a view).
cudaError_t ensure_segsum(rime_ctx *c) {
    if (c->nsm <= 0 && cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
        c->nsm = 152;
    if (!c->d_segsum && !c->view) {
        Alloc alloc{c};
        const size_t nb = (size_t)c->nsm * RIME_F32_MIN_BLOCKS;
        cudaError_t e = alloc((void **)&c->d_segsum, seg_scratch_per_block() * nb);
        if (e != cudaSuccess) return e;
        c->segsum_blocks = nb;
    }
    return c->d_segsum && c->segsum_blocks > 0 ? cudaSuccess : cudaErrorInvalidValue;
}
cudaError_t ensure_segsum2(rime_ctx *c) {
    cudaError_t e = ensure_segsum(c);
    if (e != cudaSuccess) return e;
    if (!c->d_segsum2 && !c->view) {
        Alloc alloc{c};
        e = alloc((void **)&c->d_segsum2, seg_scratch_per_block() * c->segsum_blocks);
        if (e != cudaSuccess) return e;
    }
    return c->d_segsum2 ? cudaSuccess : cudaErrorInvalidValue;
}

// Long source lists (FP32): the persistent kernel with per-block running sums.
static cudaError_t launch_seg_f32(rime_ctx *c, int mode, const FusedParams &P, long long nitems, cudaStream_t stream) {
    cudaError_t e0 = ensure_segsum(c);
    if (e0 != cudaSuccess) return e0;
    FusedParams Q = P;
    if (!Q.segsum) Q.segsum = c->d_segsum;   // a caller running launches side by side gives its own
    const long long grid = std::min<long long>(nitems, (long long)c->segsum_blocks);
    const size_t sm = sizeof(f32::Smem);
    auto go = [&](auto kernel) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        kernel<<<(unsigned)grid, f32::THREADS, sm, stream>>>(Q, nitems);
        return cudaGetLastError();
    };
    const bool general = c->beam_model != RIME_BEAM_COS3 || c->has_kind;
    switch (mode) {
        case MODE_PREDICT: return general ? go(f32::k_fused_f32_seg<MODE_PREDICT, true>) : go(f32::k_fused_f32_seg<MODE_PREDICT, false>);
        case MODE_CHI2: return general ? go(f32::k_fused_f32_seg<MODE_CHI2, true>) : go(f32::k_fused_f32_seg<MODE_CHI2, false>);
        default: return general ? go(f32::k_fused_f32_seg<MODE_GRAD, true>) : go(f32::k_fused_f32_seg<MODE_GRAD, false>);
    }
}

cudaError_t launch_tiled_params(rime_ctx *c, int mode, const FusedParams &P, long long nblocks, cudaStream_t stream) {
    if (!stream) stream = c->stream;
    if (nblocks == 0) return cudaSuccess;
    if (nblocks > (long long)c->partials_cap) return cudaErrorInvalidValue;   // one partial per block
    const int blocks = (int)nblocks;
    if (c->dims.precision == RIME_FP64) {
        size_t sm = f64::smem_bytes();
        switch (mode) {
            case MODE_PREDICT: return launch_k(f64::k_fused_f64<MODE_PREDICT>, P, blocks, f64::THREADS, sm, stream);
            case MODE_CHI2: return launch_k(f64::k_fused_f64<MODE_CHI2>, P, blocks, f64::THREADS, sm, stream);
            default: return launch_k(f64::k_fused_f64<MODE_GRAD>, P, blocks, f64::THREADS, sm, stream);
        }
    }
    size_t sm = sizeof(f32::Smem);
    if (P.src1 - P.src0 > seg_source_threshold()) return launch_seg_f32(c, mode, P, nblocks, stream);
    if (c->beam_model != RIME_BEAM_COS3 || c->has_kind) switch (mode) {
            case MODE_PREDICT: return launch_k(f32::k_fused_f32<MODE_PREDICT, true>, P, blocks, f32::THREADS, sm, stream);
            case MODE_CHI2: return launch_k(f32::k_fused_f32<MODE_CHI2, true>, P, blocks, f32::THREADS, sm, stream);
            default: return launch_k(f32::k_fused_f32<MODE_GRAD, true>, P, blocks, f32::THREADS, sm, stream);
        }
    switch (mode) {
        case MODE_PREDICT: return launch_k(f32::k_fused_f32<MODE_PREDICT, false>, P, blocks, f32::THREADS, sm, stream);
        case MODE_CHI2: return launch_k(f32::k_fused_f32<MODE_CHI2, false>, P, blocks, f32::THREADS, sm, stream);
        default: return launch_k(f32::k_fused_f32<MODE_GRAD, false>, P, blocks, f32::THREADS, sm, stream);
    }
}

cudaError_t launch_batched_f32(rime_ctx *c, const BatchParams &B, int grid) {
    FusedParams P{};
    fill_fused_params(c, P, nullptr, nullptr, nullptr, nullptr);
    if (grid <= 0 || B.nitems == 0) return cudaSuccess;
    if (B.max_set > seg_source_threshold()) {   // long sets fold into per-block running sums
        cudaError_t e = ensure_segsum(c);
        if (e != cudaSuccess) return e;
        P.segsum = c->d_segsum;
        grid = (int)std::min<long long>(grid, (long long)c->segsum_blocks);
    }
    const size_t sm = sizeof(f32::Smem);
    auto kern = (c->beam_model != RIME_BEAM_COS3 || c->has_kind) ? f32::k_batched_f32<true>
                                                                  : f32::k_batched_f32<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kern<<<grid, f32::THREADS, sm, c->stream>>>(P, B);
    return cudaGetLastError();
}

int batched_blocks_per_sm() {
    // both beam instances take the same registers and shared memory
    int n = 0;
    if (cudaFuncSetAttribute(f32::k_batched_f32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(f32::Smem)) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f32::k_batched_f32<false>, f32::THREADS,
                                                      sizeof(f32::Smem)) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_set_sums(rime_ctx *c, int nsets, int per_set, const double *partials, double *chi2) {
    if (nsets <= 0) return cudaSuccess;
    k_set_sums<<<nsets, 256, 0, c->stream>>>(per_set, partials, chi2, c->d_status);
    return cudaGetLastError();
}

cudaError_t launch_fused_f64_range(rime_ctx *c, int src0, int src1, double *result) {
    FusedParams P{};
    fill_fused_params(c, P, nullptr, result, nullptr, nullptr);
    P.src0 = src0;
    P.src1 = src1;
    const int blocks = fused_blocks(c);
    if (blocks == 0) return cudaSuccess;
    return launch_k(f64::k_fused_f64<MODE_CHI2>, P, blocks, f64::THREADS, f64::smem_bytes(), c->stream);
}

}  // namespace rime
