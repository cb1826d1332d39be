// rime_beam.cuh -- the primary beam E of eq. 4 as a function of
// x = C nu[GHz] rho (rho the distance of the source from the antenna's
// pointing centre), for the beam models of rime_set_beam:
//   RIME_BEAM_COS3 (eq. 4, WSRT): E = cos^3 x for x < pi/2, zero past the
//                  first null;
//   RIME_BEAM_JINC (the Jinc that Sec. 2.1 names for the VLA): E = 2 J1(x)/x,
//                  the Airy pattern of a uniformly illuminated dish.
// With J1' = J0 - J1/x, d(2 J1(x)/x)/dx = -2 J2(x)/x, J2 = 2 J1/x - J0; near
// x = 0 the power series 2 J1(x)/x = sum_k (-1)^k (x/2)^(2k) / (k! (k+1)!) =
// 1 - x^2/8 + x^4/192 - x^6/9216 ... and its derivative over x,
// -1/4 + x^2/48 - x^4/1536 + x^6/92160 ..., avoid 0/0 and the cancellation
// in 2 J1/x - J0. J0 and J1 are CUDA's j0f / j1f / j0 / j1.
#pragma once
#include "../../include/rime.h"
#include <cuda_runtime.h>

namespace rime {

__device__ __forceinline__ float jinc_f(float x) { return x < 1e-3f ? 1.0f - 0.125f * x * x : 2.0f * j1f(x) / x; }

__device__ __forceinline__ float beam_E(int model, float x) {
    if (model == RIME_BEAM_JINC) return jinc_f(x);
    const float cb = cosf(x);
    return (x < 1.57079632679f) ? cb * cb * cb : 0.0f;
}
__device__ __forceinline__ double jinc_d(double x) {
    if (x < 0.05) {
        const double x2 = x * x;
        return 1.0 - x2 / 8.0 + x2 * x2 / 192.0 - x2 * x2 * x2 / 9216.0;
    }
    return 2.0 * j1(x) / x;
}

__device__ __forceinline__ double beam_E(int model, double x) {
    if (model == RIME_BEAM_JINC) return jinc_d(x);
    const double cb = cos(x);
    return (x < 1.5707963267948966) ? cb * cb * cb : 0.0;
}

__device__ __forceinline__ void jinc_d_f(float x, float &E, float &dEx) {
    if (x < 0.5f) {
        const float x2 = x * x;
        E = x < 1e-3f ? 1.0f - 0.125f * x2 : 2.0f * j1f(x) / x;
        dEx = -0.25f + x2 * (1.0f / 48.0f - x2 * (1.0f / 1536.0f - x2 * (1.0f / 92160.0f)));
    } else {
        const float j1x = j1f(x), j0x = j0f(x);
        E = 2.0f * j1x / x;
        dEx = -2.0f * (2.0f * j1x / x - j0x) / (x * x);
    }
}

__device__ __forceinline__ void jinc_dd(double x, double &E, double &dEx) {
    if (x < 0.05) {
        const double x2 = x * x;
        E = 1.0 - x2 / 8.0 + x2 * x2 / 192.0 - x2 * x2 * x2 / 9216.0;
        dEx = -0.25 + x2 / 48.0 - x2 * x2 / 1536.0 + x2 * x2 * x2 / 92160.0;
    } else {
        const double j1x = j1(x), j0x = j0(x);
        E = 2.0 * j1x / x;
        dEx = -2.0 * (2.0 * j1x / x - j0x) / (x * x);
    }
}

// E and t3 = (dE/dx) / (x E), so that d ln E / dl = t3 (C nu)^2 (l - dl);
// t3 = 0 where E = 0 (a source exactly on a null).
__device__ __forceinline__ void beam_Ed(int model, float x, float &E, float &t3) {
    float dEx;   // (dE/dx) / x
    if (model == RIME_BEAM_JINC) {
        jinc_d_f(x, E, dEx);
    } else {
        if (x >= 1.57079632679f) {
            E = 0.0f;
            t3 = 0.0f;
            return;
        }
        float sn, cs;
        sincosf(x, &sn, &cs);
        E = cs * cs * cs;
        const float sinc = x < 1e-4f ? 1.0f : sn / x;
        dEx = -3.0f * cs * cs * sinc;
    }
    t3 = E != 0.0f ? dEx / E : 0.0f;
}
__device__ __forceinline__ void beam_Ed(int model, double x, double &E, double &t3) {
    double dEx;
    if (model == RIME_BEAM_JINC) {
        jinc_dd(x, E, dEx);
    } else {
        if (x >= 1.5707963267948966) {
            E = 0.0;
            t3 = 0.0;
            return;
        }
        double sn, cs;
        sincos(x, &sn, &cs);
        E = cs * cs * cs;
        const double sinc = x < 1e-8 ? 1.0 : sn / x;
        dEx = -3.0 * cs * cs * sinc;
    }
    t3 = E != 0.0 ? dEx / E : 0.0;
}

}  // namespace rime
