// rime_fused_common.cuh -- device pieces shared by the fused predict + chi^2
// kernels (the tiled kernels of rime_fused.cu and the small-array kernel of
// rime_narrow.cu): the FP32 phase and beam factors and the deterministic
// chi^2 reduction.
#pragma once
#include "rime_internal.cuh"
#include "rime_dev.cuh"
#include "rime_beam.cuh"

namespace rime {

__device__ __forceinline__ float ex2_approx(float e) {
    float g;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(g) : "f"(e));
    return g;
}

// Block-wide deterministic FP64 sum of one value per thread; result valid in
// thread 0. red: >= 32 doubles of shared memory.
template <int THREADS>
__device__ __forceinline__ double block_sum(double v, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double x = 0.0;
    if (warp == 0) {
        x = lane < THREADS / 32 ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    }
    return x;
}

// One partial per block, then the last block to arrive sums them in index
// order and stores the total. All threads of the block must call it.
template <int THREADS>
__device__ void finish_chi2(double block_value, const FusedParams &P, double *red, int *sLast) {
    if (threadIdx.x == 0) {
        P.partials[blockIdx.x] = block_value;
        __threadfence();
        unsigned ticket = atomicAdd(P.counter, 1u);
        *sLast = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (*sLast) {
        __threadfence();
        double s = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += THREADS) s += __ldcg(&P.partials[i]);
        double tot = block_sum<THREADS>(s, red);
        if (threadIdx.x == 0) {
            *P.result = tot;
            *P.counter = 0u;
        }
    }
}

// Adjoint of the chi^2 term of one visibility (eq. 7 through eq. 1):
//   Sh = 2 w G_p^H R G_q with R = V - D; for a source with coherency c B0
//   (eq. 2), d chi^2 = Re(c sum_X X Y_X) with
//   Y_I = conj(Sh00 + Sh11), Y_Q = conj(Sh00 - Sh11), Y_U = conj(Sh01 + Sh10),
//   Y_V = i conj(Sh01 - Sh10);
//   dchi^2/dG_p = 2 w R G_q S^H, dchi^2/dG_q = 2 w R^H G_p S  (complex
//   gradient d/dRe + i d/dIm).
template <typename T, typename T2>
__device__ __forceinline__ void grad_terms(const T2 *V, const T2 *Sm, const T2 *D, T w, const T2 *gp, const T2 *gq,
                                           T2 *Y, T2 *dGp, T2 *dGq) {
    T2 R[4], Sh[4], tmp[4], gh[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
        R[c] = csub(V[c], D[c]);
        R[c].x *= 2 * w;
        R[c].y *= 2 * w;
    }
    mherm(gp, gh);
    mmul(gh, R, tmp);
    mmul(tmp, gq, Sh);
    Y[0] = cconj(cadd(Sh[0], Sh[3]));
    Y[1] = cconj(csub(Sh[0], Sh[3]));
    Y[2] = cconj(cadd(Sh[1], Sh[2]));
    T2 d = csub(Sh[1], Sh[2]);
    Y[3].x = d.y;
    Y[3].y = d.x;
    T2 sh[4];
    mherm(Sm, sh);
    mmul(R, gq, tmp);
    mmul(tmp, sh, dGp);
    mherm(R, gh);
    mmul(gh, gp, tmp);
    mmul(tmp, Sm, dGq);
}

namespace f32 {
// The phase of eq. 3 in turns, nu tau, reduced to about [-1/2, 1/2] from the
// double-float pairs nu = nu_hi + nu_lo and tau = tau.x + tau.y:
// nu_hi tau_hi = p + e exactly (FMA), p - round(p) is exact (|p| < 2^22),
// and the small products add the rest. The result differs from the FP64
// value nu tau - round(nu tau), rounded to FP32, by at most about one unit in
// the last place of 1/2 (2^-24 turns) plus 2^-47 |nu tau| (the pairs'
// representation and the small products' rounding).
__device__ __forceinline__ float reduced_turns(float2 tau, float nu_hi, float nu_lo) {
    const float p = nu_hi * tau.x;
    const float e = fmaf(nu_hi, tau.x, -p);
    const float r = p - round_int_f(p);
    return r + (e + fmaf(nu_hi, tau.y, nu_lo * tau.x));
}
// Phase factor K = exp(2 pi i nu tau) (eq. 3) from the double-float delay,
// reduced as above; the SFU sine and cosine are accurate to ~2^-21 absolute
// on [-pi, pi].
__device__ __forceinline__ float2 phase_factor(float2 tau, const ChanF &ch) {
    const float f = reduced_turns(tau, ch.nu_hi, ch.nu_lo);
    float sn, cs;
    __sincosf(6.28318530717958648f * f, &sn, &cs);
    return make_float2(cs, sn);
}

// Beam E of eq. 4 (or the Jinc model) at x = C nu[GHz] rho.
__device__ __forceinline__ float beam(float rho, const ChanF &ch) { return beam_E(ch.beam, ch.cnu * rho); }

}  // namespace f32

}  // namespace rime
