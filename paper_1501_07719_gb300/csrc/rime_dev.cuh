// rime_dev.cuh -- small device helpers shared by the kernels: exact
// rounding to an integer and 2x2 complex matrix arithmetic.
#pragma once

#include <cuda_runtime.h>

namespace rime {

__device__ __forceinline__ float round_int_f(float x) {
    // nearest integer for |x| < 2^22 (1.5 * 2^23 magic constant), ties to even
    const float M = 12582912.0f;
    return __fsub_rn(__fadd_rn(x, M), M);
}
__device__ __forceinline__ double round_int_d(double x) {
    const double M = 6755399441055744.0;   // 1.5 * 2^52
    return __dsub_rn(__dadd_rn(x, M), M);
}

// ---------------------------------------------------------------------------
// 2x2 complex matrices (row-major 00, 01, 10, 11) for the epilogues
// ---------------------------------------------------------------------------
template <typename T2> __device__ __forceinline__ T2 cmk(double x, double y);
template <> __device__ __forceinline__ float2 cmk<float2>(double x, double y) { return make_float2((float)x, (float)y); }
template <> __device__ __forceinline__ double2 cmk<double2>(double x, double y) { return make_double2(x, y); }
template <typename T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b) {
    T2 r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename T2> __device__ __forceinline__ T2 cmulc(T2 a, T2 b) {   // a conj(b)
    T2 r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}
template <typename T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b) { T2 r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) { T2 r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename T2> __device__ __forceinline__ T2 cconj(T2 a) { T2 r; r.x = a.x; r.y = -a.y; return r; }
template <typename T2> __device__ __forceinline__ void mmul(const T2 *a, const T2 *b, T2 *o) {
    T2 r0 = cadd(cmul(a[0], b[0]), cmul(a[1], b[2])), r1 = cadd(cmul(a[0], b[1]), cmul(a[1], b[3]));
    T2 r2 = cadd(cmul(a[2], b[0]), cmul(a[3], b[2])), r3 = cadd(cmul(a[2], b[1]), cmul(a[3], b[3]));
    o[0] = r0; o[1] = r1; o[2] = r2; o[3] = r3;
}
template <typename T2> __device__ __forceinline__ void mherm(const T2 *a, T2 *o) {
    T2 r1 = cconj(a[2]), r2 = cconj(a[1]);
    o[0] = cconj(a[0]); o[1] = r1; o[2] = r2; o[3] = cconj(a[3]);
}

}  // namespace rime
