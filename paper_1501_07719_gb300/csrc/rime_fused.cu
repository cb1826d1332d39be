// rime_fused.cu -- the fused RIME predict + chi^2 kernel (eqs. 1-7).
//
// The paper runs three kernels (Sec. 4.2): EK (Algorithm 1) writes the
// per-antenna factor A_tpsk = E_tpsk K_tpsk to DRAM, B Sum (Algorithm 2)
// reads A for both antennas of each baseline and forms the chi^2 terms, and
// a tree reduction sums them. Here one kernel does all three:
//
//  * a thread block owns one timestep t, one channel k and one "unit" of
//    antenna pairs (a block of up to 64 row antennas against up to 64
//    column antennas; na <= 64 is a single unit);
//  * per chunk of SC sources it stages A = sqrt(f) E K for the unit's
//    antennas in shared memory (the spectral factor f = (nu/nu_ref)^alpha of
//    eq. 2 is split as sqrt(f) on each antenna), so every A is computed once
//    and reused by all ~na/2 baselines that share the antenna;
//  * each thread accumulates a TP x TQ antenna tile (TP*TQ baselines) with
//    four complex accumulators per baseline, sum_s z_s X_s for X in
//    (I, Q, U, V), z = A_p conj(A_q) g;
//  * the epilogue forms S from the Stokes sums (eq. 2), applies the gains
//    (eq. 1), and either writes V or forms w |V - D|^2 (eq. 7);
//  * chi^2: thread -> warp shuffle -> block in FP64 -> one partial per
//    block; the last block to finish sums the partials in index order, so
//    the result is deterministic.
//
// FP32 mode keeps the phase exact: nu tau (up to ~1e2 turns) is formed as a
// double-float product and reduced to [-1/2, 1/2] turns without rounding
// error before sincospi; the FP64 delays come from the upload kernels.
#include "rime_internal.cuh"

#include <algorithm>
#include <vector>

namespace rime {

template <typename T>
struct Shape;
// FP32: 4x2 antenna tiles, 64-antenna units.
template <>
struct Shape<float> {
    static constexpr int TP = 4;          // row antennas per thread tile
    static constexpr int TQ = 2;          // column antennas per thread tile
    static constexpr int NB = TP * TQ;    // baselines per thread
    static constexpr int ROWS = 64;       // row antennas per unit
    static constexpr int COLS = 32;       // column antennas per off-diagonal unit
    static constexpr int THREADS = 288;   // tiles of a 64-antenna diagonal unit (272), whole warps
    static constexpr int SC = 32;         // sources per staged chunk
    static constexpr int ASTRIDE = ROWS + 8;
    static constexpr int MINB = 1;
};
// FP64: 2x2 antenna tiles, 32-antenna units (the FP64 accumulators need the registers).
template <>
struct Shape<double> {
    static constexpr int TP = 2;
    static constexpr int TQ = 2;
    static constexpr int NB = TP * TQ;
    static constexpr int ROWS = 32;
    static constexpr int COLS = 32;
    static constexpr int THREADS = 256;
    static constexpr int SC = 16;
    static constexpr int ASTRIDE = ROWS + 4;
    static constexpr int MINB = 1;
};

template <typename T> struct Vec;
template <> struct Vec<float> { using T2 = float2; using T4 = float4; using Chan = ChanF; };
template <> struct Vec<double> { using T2 = double2; struct T4 { double x, y, z, w; }; using Chan = ChanD; };

// ---------------------------------------------------------------------------
// Per-antenna factor A = sqrt(f) E K for one (t, s, a, k)   (eqs. 2-4)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float round_int_f(float x) {
    // nearest integer for |x| < 2^22 (1.5 * 2^23 magic constant), ties to even
    const float M = 12582912.0f;
    return __fsub_rn(__fadd_rn(x, M), M);
}
__device__ __forceinline__ double round_int_d(double x) {
    const double M = 6755399441055744.0;   // 1.5 * 2^52
    return __dsub_rn(__dadd_rn(x, M), M);
}

__device__ __forceinline__ float2 antenna_factor(float2 tau, float rho, float alpha, const ChanF &ch) {
    // phase nu * tau in turns as a double-float product: nu_hi tau_hi = p + e
    // exactly, p - round(p) is exact, the small terms add the rest.
    float p = ch.nu_hi * tau.x;
    float e = fmaf(ch.nu_hi, tau.x, -p);
    float r = p - round_int_f(p);
    float f = r + (e + fmaf(ch.nu_hi, tau.y, ch.nu_lo * tau.x));
    float sn, cs;
    sincospif(2.0f * f, &sn, &cs);                 // eq. 3
    float x = ch.cnu * rho;                        // eq. 4: C nu[GHz] rho
    float cb = cosf(x);
    float E = (x < 1.57079632679f) ? cb * cb * cb : 0.0f;
    float amp = E * exp2f(alpha * ch.hlr);         // sqrt of eq. 2's spectral factor
    return make_float2(amp * cs, amp * sn);
}

__device__ __forceinline__ double2 antenna_factor(double tau, double rho, double alpha, const ChanD &ch) {
    double ph = ch.nu * tau;
    double r = ph - round_int_d(ph);
    double sn, cs;
    sincospi(2.0 * r, &sn, &cs);
    double x = ch.cnu * rho;
    double cb = cos(x);
    double E = (x < 1.5707963267948966) ? cb * cb * cb : 0.0;
    double amp = E * exp2(alpha * ch.hlr);
    return make_double2(amp * cs, amp * sn);
}

__device__ __forceinline__ float gauss_factor(float e) {
    float g;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(g) : "f"(e));
    return g;
}
__device__ __forceinline__ double gauss_factor(double e) { return exp(e); }

// ---------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------
template <typename T>
struct Smem {
    using T2 = typename Vec<T>::T2;
    using T4 = typename Vec<T>::T4;
    using Chan = typename Vec<T>::Chan;
    static constexpr int A_ELEMS = 2 * Shape<T>::SC * Shape<T>::ASTRIDE;
    static constexpr size_t bytes() {
        return A_ELEMS * sizeof(T2) + Shape<T>::SC * sizeof(T4) * 2 + sizeof(Chan) + 64 * sizeof(double);
    }
};

template <typename T, bool CHI2, bool WRITE>
__global__ void __launch_bounds__(Shape<T>::THREADS, Shape<T>::MINB) k_fused(const FusedParams P) {
    using S = Shape<T>;
    using T2 = typename Vec<T>::T2;
    using T4 = typename Vec<T>::T4;
    using Chan = typename Vec<T>::Chan;
    constexpr bool F32 = sizeof(T) == 4;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2 *sA = reinterpret_cast<T2 *>(smem_raw);                 // [2][SC][ASTRIDE]
    T4 *sSt = reinterpret_cast<T4 *>(sA + Smem<T>::A_ELEMS);    // [SC] stokes
    T4 *sGq = sSt + S::SC;                                      // [SC] gauss coeffs * nu^2, flag
    Chan *sCh = reinterpret_cast<Chan *>(sGq + S::SC);
    double *sRed = reinterpret_cast<double *>(sCh + 1);          // [32]
    __shared__ int sLast;

    if (inputs_bad(P.status)) return;

    const int tid = threadIdx.x;
    const int u = blockIdx.x % P.nunits;
    const int rest = blockIdx.x / P.nunits;
    const int k = rest % P.nchan;
    const int t = rest / P.nchan;
    const Unit U = P.units[u];
    const bool active = tid < U.ntiles;

    if (tid == 0) *sCh = reinterpret_cast<const Chan *>(P.chan)[k];

    int pl = 0, ql = 0;
    if (active) {
        Tile tl = P.tiles[U.tile0 + tid];
        pl = tl.p;
        ql = tl.q;
    }
    const int p0 = U.r0 + pl, q0 = U.c0 + ql;
    unsigned mask = 0;
#pragma unroll
    for (int i = 0; i < S::TP; i++)
#pragma unroll
        for (int j = 0; j < S::TQ; j++)
            if (active && p0 + i < q0 + j && q0 + j < P.na) mask |= 1u << (i * S::TQ + j);

    // baseline terms of the Gaussian exponent: du^2, du dv, dv^2 (metres^2)
    T du2[S::NB], dudv[S::NB], dv2[S::NB];
#pragma unroll
    for (int i = 0; i < S::TP; i++) {
        int pa = min(p0 + i, P.na - 1);
        T up, vp;
        if constexpr (F32) {
            float4 x = P.uvw_f[(long long)t * P.na + pa];
            up = x.x; vp = x.y;
        } else {
            up = P.uvw[3 * ((long long)t * P.na + pa)];
            vp = P.uvw[3 * ((long long)t * P.na + pa) + 1];
        }
#pragma unroll
        for (int j = 0; j < S::TQ; j++) {
            int qa = min(q0 + j, P.na - 1);
            T uq, vq;
            if constexpr (F32) {
                float4 x = P.uvw_f[(long long)t * P.na + qa];
                uq = x.x; vq = x.y;
            } else {
                uq = P.uvw[3 * ((long long)t * P.na + qa)];
                vq = P.uvw[3 * ((long long)t * P.na + qa) + 1];
            }
            T du = up - uq, dv = vp - vq;
            du2[i * S::TQ + j] = du * du;
            dudv[i * S::TQ + j] = du * dv;
            dv2[i * S::TQ + j] = dv * dv;
        }
    }

    T acc[S::NB][8];
#pragma unroll
    for (int b = 0; b < S::NB; b++)
#pragma unroll
        for (int c = 0; c < 8; c++) acc[b][c] = T(0);

    const int nloc = U.diag ? U.nr : U.nr + U.nc;
    const T2 *Ar = sA;
    const T2 *Ac = U.diag ? sA : sA + S::SC * S::ASTRIDE;
    const T *gauss = reinterpret_cast<const T *>(P.gauss);
    const T *stokes = reinterpret_cast<const T *>(P.stokes) + (long long)t * P.stokes_tstride;
    const T *alpha = reinterpret_cast<const T *>(P.alpha);
    __syncthreads();
    const Chan ch = *sCh;

    for (int s0 = 0; s0 < P.nsrc; s0 += S::SC) {
        const int sc = min(S::SC, P.nsrc - s0);
        // ---- stage A for the chunk (Algorithm 1, kept on chip) ----
        for (int j = tid; j < sc * nloc; j += S::THREADS) {
            int s = j / nloc, a = j - s * nloc;
            int ant = a < U.nr ? U.r0 + a : U.c0 + (a - U.nr);
            T2 *dst = (a < U.nr ? sA + a : sA + S::SC * S::ASTRIDE + (a - U.nr)) + s * S::ASTRIDE;
            T2 v;
            {
                long long di = ((long long)t * P.nsrc + s0 + s) * P.na + ant;
                if constexpr (F32)
                    v = antenna_factor(reinterpret_cast<const float2 *>(P.tau)[di],
                                       reinterpret_cast<const float *>(P.rho)[di], alpha[s0 + s], ch);
                else
                    v = antenna_factor(reinterpret_cast<const double *>(P.tau)[di],
                                       reinterpret_cast<const double *>(P.rho)[di], alpha[s0 + s], ch);
            }
            *dst = v;
        }
        if (tid < S::SC) {
            T4 st, gq;
            if (tid < sc) {
                const T *x = stokes + 4 * (long long)(s0 + tid);
                const T *g = gauss + 4 * (long long)(s0 + tid);
                st.x = x[0]; st.y = x[1]; st.z = x[2]; st.w = x[3];
                gq.x = g[0] * ch.nu2; gq.y = g[1] * ch.nu2; gq.z = g[2] * ch.nu2; gq.w = g[3];
            } else {
                st.x = st.y = st.z = st.w = T(0);
                gq.x = gq.y = gq.z = gq.w = T(0);
            }
            sSt[tid] = st;
            sGq[tid] = gq;
        }
        __syncthreads();
        // ---- source sum for this thread's baselines (Algorithm 2) ----
        if (active) {
#pragma unroll 2
            for (int s = 0; s < sc; s++) {
                const T4 st = sSt[s];
                const T4 gq = sGq[s];
                T2 ap[S::TP], aq[S::TQ];
#pragma unroll
                for (int i = 0; i < S::TP; i++) ap[i] = Ar[s * S::ASTRIDE + pl + i];
#pragma unroll
                for (int j = 0; j < S::TQ; j++) aq[j] = Ac[s * S::ASTRIDE + ql + j];
                const bool is_gauss = gq.w != T(0);
#pragma unroll
                for (int i = 0; i < S::TP; i++)
#pragma unroll
                    for (int j = 0; j < S::TQ; j++) {
                        const int b = i * S::TQ + j;
                        // z = A_p conj(A_q)
                        T zr = ap[i].x * aq[j].x + ap[i].y * aq[j].y;
                        T zi = ap[i].y * aq[j].x - ap[i].x * aq[j].y;
                        if (is_gauss) {
                            T g = gauss_factor(gq.x * du2[b] + gq.y * dudv[b] + gq.z * dv2[b]);
                            zr *= g;
                            zi *= g;
                        }
                        acc[b][0] += zr * st.x; acc[b][1] += zi * st.x;   // I
                        acc[b][2] += zr * st.y; acc[b][3] += zi * st.y;   // Q
                        acc[b][4] += zr * st.z; acc[b][5] += zi * st.z;   // U
                        acc[b][6] += zr * st.w; acc[b][7] += zi * st.w;   // V
                    }
            }
        }
        __syncthreads();
    }

    // ---- epilogue: S (eq. 2), gains (eq. 1), chi^2 terms (eq. 7) ----
    T chi = T(0);
    const T2 *gains = reinterpret_cast<const T2 *>(P.gains);
    const T2 *data = reinterpret_cast<const T2 *>(P.data);
    const T *weight = reinterpret_cast<const T *>(P.weight);
    T2 *vis = reinterpret_cast<T2 *>(P.vis_out);
#pragma unroll
    for (int i = 0; i < S::TP; i++) {
        const int p = p0 + i;
        T2 gp[4];
        if (P.has_gains && (mask >> (i * S::TQ)) & ((1u << S::TQ) - 1)) {
            const T2 *g = gains + 4 * (((long long)t * P.na + p) * P.nchan + k);
#pragma unroll
            for (int c = 0; c < 4; c++) gp[c] = g[c];
        }
#pragma unroll
        for (int j = 0; j < S::TQ; j++) {
            const int b = i * S::TQ + j;
            if (!((mask >> b) & 1u)) continue;
            const int q = q0 + j;
            // S from the Stokes sums: [[I+Q, U+iV], [U-iV, I-Q]]
            T2 Sm[4];
            Sm[0].x = acc[b][0] + acc[b][2]; Sm[0].y = acc[b][1] + acc[b][3];
            Sm[1].x = acc[b][4] - acc[b][7]; Sm[1].y = acc[b][5] + acc[b][6];
            Sm[2].x = acc[b][4] + acc[b][7]; Sm[2].y = acc[b][5] - acc[b][6];
            Sm[3].x = acc[b][0] - acc[b][2]; Sm[3].y = acc[b][1] - acc[b][3];
            T2 V[4];
            if (P.has_gains) {
                const T2 *gq_ = gains + 4 * (((long long)t * P.na + q) * P.nchan + k);
                T2 gq[4];
#pragma unroll
                for (int c = 0; c < 4; c++) gq[c] = gq_[c];
                // X = G_p S
                T2 X[4];
#pragma unroll
                for (int r = 0; r < 2; r++)
#pragma unroll
                    for (int cc = 0; cc < 2; cc++) {
                        T2 a = gp[2 * r], bb = gp[2 * r + 1], s0v = Sm[cc], s1v = Sm[2 + cc];
                        X[2 * r + cc].x = a.x * s0v.x - a.y * s0v.y + bb.x * s1v.x - bb.y * s1v.y;
                        X[2 * r + cc].y = a.x * s0v.y + a.y * s0v.x + bb.x * s1v.y + bb.y * s1v.x;
                    }
                // V = X G_q^H : V_rc = sum_m X_rm conj(Gq_cm)
#pragma unroll
                for (int r = 0; r < 2; r++)
#pragma unroll
                    for (int cc = 0; cc < 2; cc++) {
                        T2 x0 = X[2 * r], x1 = X[2 * r + 1], g0 = gq[2 * cc], g1 = gq[2 * cc + 1];
                        V[2 * r + cc].x = x0.x * g0.x + x0.y * g0.y + x1.x * g1.x + x1.y * g1.y;
                        V[2 * r + cc].y = x0.y * g0.x - x0.x * g0.y + x1.y * g1.x - x1.x * g1.y;
                    }
            } else {
#pragma unroll
                for (int c = 0; c < 4; c++) V[c] = Sm[c];
            }
            const long long bl = (long long)p * P.na - (long long)p * (p + 1) / 2 + (q - p - 1);
            const long long row = ((long long)t * P.nbl + bl) * P.nchan + k;
            if constexpr (WRITE) {
#pragma unroll
                for (int c = 0; c < 4; c++) vis[4 * row + c] = V[c];
            }
            if constexpr (CHI2) {
                T r2 = T(0);
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    T2 d = data[4 * row + c];
                    T dr = V[c].x - d.x, di = V[c].y - d.y;
                    r2 += dr * dr + di * di;
                }
                chi += (P.has_weight ? weight[row] : T(1)) * r2;
            }
        }
    }

    if constexpr (CHI2) {
        const int lane = tid & 31, warp = tid >> 5;
        T v = chi;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sRed[warp] = (double)v;
        __syncthreads();
        if (warp == 0) {
            double x = lane < S::THREADS / 32 ? sRed[lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) {
                P.partials[blockIdx.x] = x;
                __threadfence();
                unsigned ticket = atomicAdd(P.counter, 1u);
                sLast = (ticket == gridDim.x - 1);
            }
        }
        __syncthreads();
        if (sLast) {
            __threadfence();
            double s = 0.0;
            for (int i = tid; i < (int)gridDim.x; i += S::THREADS) s += __ldcg(&P.partials[i]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            __syncthreads();
            if (lane == 0) sRed[warp] = s;
            __syncthreads();
            if (warp == 0) {
                double x = lane < S::THREADS / 32 ? sRed[lane] : 0.0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
                if (lane == 0) {
                    *P.result = x;
                    *P.counter = 0u;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Host side: work units and launch
// ---------------------------------------------------------------------------
template <typename T>
static void build_units_t(int na, std::vector<Unit> &units, std::vector<Tile> &tiles) {
    using S = Shape<T>;
    units.clear();
    tiles.clear();
    for (int r0 = 0; r0 < na; r0 += S::ROWS) {
        int nr = std::min(S::ROWS, na - r0);
        // diagonal unit: tiles with at least one pair p < q
        {
            Unit u{r0, r0, nr, nr, (int)tiles.size(), 0, 1, 0};
            for (int pi = 0; pi < nr; pi += S::TP)
                for (int qj = 0; qj < nr; qj += S::TQ)
                    if (qj + S::TQ - 1 > pi) tiles.push_back(Tile{(uint8_t)pi, (uint8_t)qj});
            u.ntiles = (int)tiles.size() - u.tile0;
            units.push_back(u);
        }
        // off-diagonal units: all pairs valid
        for (int c0 = r0 + S::ROWS; c0 < na; c0 += S::COLS) {
            int nc = std::min(S::COLS, na - c0);
            Unit u{r0, c0, nr, nc, (int)tiles.size(), 0, 0, 0};
            for (int pi = 0; pi < nr; pi += S::TP)
                for (int qj = 0; qj < nc; qj += S::TQ) tiles.push_back(Tile{(uint8_t)pi, (uint8_t)qj});
            u.ntiles = (int)tiles.size() - u.tile0;
            units.push_back(u);
        }
    }
}

void build_units(int na, int precision, std::vector<Unit> &units, std::vector<Tile> &tiles) {
    if (precision == RIME_FP64) build_units_t<double>(na, units, tiles);
    else build_units_t<float>(na, units, tiles);
}

// The same work units as build_units, written into caller-provided arrays
// (no heap use). Returns the number of units, or -1 if an array is too small.
template <typename T>
static int build_units_fixed_t(int na, Unit *units, int max_units, Tile *tiles, int max_tiles, int *ntiles) {
    using S = Shape<T>;
    int nu = 0, nt = 0;
    for (int r0 = 0; r0 < na; r0 += S::ROWS) {
        int nr = std::min(S::ROWS, na - r0);
        if (nu >= max_units) return -1;
        Unit d{r0, r0, nr, nr, nt, 0, 1, 0};
        for (int pi = 0; pi < nr; pi += S::TP)
            for (int qj = 0; qj < nr; qj += S::TQ)
                if (qj + S::TQ - 1 > pi) {
                    if (nt >= max_tiles) return -1;
                    tiles[nt++] = Tile{(uint8_t)pi, (uint8_t)qj};
                }
        d.ntiles = nt - d.tile0;
        units[nu++] = d;
        for (int c0 = r0 + S::ROWS; c0 < na; c0 += S::COLS) {
            int nc = std::min(S::COLS, na - c0);
            if (nu >= max_units) return -1;
            Unit u{r0, c0, nr, nc, nt, 0, 0, 0};
            for (int pi = 0; pi < nr; pi += S::TP)
                for (int qj = 0; qj < nc; qj += S::TQ) {
                    if (nt >= max_tiles) return -1;
                    tiles[nt++] = Tile{(uint8_t)pi, (uint8_t)qj};
                }
            u.ntiles = nt - u.tile0;
            units[nu++] = u;
        }
    }
    *ntiles = nt;
    return nu;
}

int build_units_fixed(int na, int precision, Unit *units, int max_units, Tile *tiles, int max_tiles,
                      int *ntiles) {
    return precision == RIME_FP64 ? build_units_fixed_t<double>(na, units, max_units, tiles, max_tiles, ntiles)
                                  : build_units_fixed_t<float>(na, units, max_units, tiles, max_tiles, ntiles);
}

int fused_blocks(const rime_ctx *c) { return c->dims.ntime * c->dims.nchan * c->nunits; }

template <typename T, bool CHI2, bool WRITE>
static cudaError_t launch_t(const FusedParams &P, int blocks, cudaStream_t stream) {
    size_t smem = Smem<T>::bytes();
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_fused<T, CHI2, WRITE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_fused<T, CHI2, WRITE><<<blocks, Shape<T>::THREADS, smem, stream>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_fused(rime_ctx *c, void *vis_out, double *result, bool chi2) {
    FusedParams P{};
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
    int blocks = fused_blocks(c);
    if (blocks == 0) return cudaSuccess;
    bool f64 = c->dims.precision == RIME_FP64;
    if (chi2)
        return f64 ? launch_t<double, true, false>(P, blocks, c->stream)
                   : launch_t<float, true, false>(P, blocks, c->stream);
    return f64 ? launch_t<double, false, true>(P, blocks, c->stream)
               : launch_t<float, false, true>(P, blocks, c->stream);
}

}  // namespace rime
