// Device helpers shared by the librom kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace romk {

// Ricker wavelet of Sec. 3.2 with delay t0 = 1.5 T, sampled at t = step * dt:
//   f = (1 - 2u) exp(-u),  u = pi^2 (t - t0)^2 / T^2.
// The time offset tau = t - t0 is formed in FP64 (step * dt reaches ~1e4 and
// would lose the pulse's position in FP32); the wavelet itself is evaluated
// in the path's precision with CUDA's expf / exp.
__device__ __forceinline__ float ricker_eval(long long step, double dt, float T) {
    const double tau = (double)step * dt - 1.5 * (double)T;
    const float a = (float)(3.14159265358979323846 * tau / (double)T);
    const float u = a * a;
    return (1.0f - 2.0f * u) * expf(-u);
}

__device__ __forceinline__ double ricker_eval(long long step, double dt, double T) {
    const double tau = (double)step * dt - 1.5 * T;
    const double a = 3.14159265358979323846 * tau / T;
    const double u = a * a;
    return (1.0 - 2.0 * u) * exp(-u);
}

// d f / d T at fixed t (t0 = 1.5 T moves with T):
//   df/du = (2u - 3) e^{-u},  du/dT = -pi^2 tau (3T + 2 tau) / T^3.
__device__ __forceinline__ float ricker_dT_eval(long long step, double dt, float T) {
    const double tau = (double)step * dt - 1.5 * (double)T;
    const float a = (float)(3.14159265358979323846 * tau / (double)T);
    const float u = a * a;
    const float dudT = (float)(-9.8696044010893586188 * tau * (3.0 * (double)T + 2.0 * tau) /
                               ((double)T * (double)T * (double)T));
    return (2.0f * u - 3.0f) * expf(-u) * dudT;
}
__device__ __forceinline__ double ricker_dT_eval(long long step, double dt, double T) {
    const double tau = (double)step * dt - 1.5 * T;
    const double a = 3.14159265358979323846 * tau / T;
    const double u = a * a;
    const double dudT = -9.8696044010893586188 * tau * (3.0 * T + 2.0 * tau) / (T * T * T);
    return (2.0 * u - 3.0) * exp(-u) * dudT;
}

// First derivative of a Gaussian (the paper's second source signal, Sec.
// 3.2): the tau-derivative of the Ricker's envelope exp(-pi^2 tau^2 / T^2),
// delay 1.5 T, scaled to unit peak magnitude:
//   f = -sqrt(2e) a exp(-a^2),  a = pi tau / T.
constexpr double kSqrt2e = 2.33164398159712420;

__device__ __forceinline__ float gauss1_eval(long long step, double dt, float T) {
    const double tau = (double)step * dt - 1.5 * (double)T;
    const float a = (float)(3.14159265358979323846 * tau / (double)T);
    return -(float)kSqrt2e * a * expf(-a * a);
}
__device__ __forceinline__ double gauss1_eval(long long step, double dt, double T) {
    const double tau = (double)step * dt - 1.5 * T;
    const double a = 3.14159265358979323846 * tau / T;
    return -kSqrt2e * a * exp(-a * a);
}
// d f / d T at fixed t: df/da = -sqrt(2e) (1 - 2a^2) e^{-a^2}, da/dT = -pi t / T^2.
__device__ __forceinline__ float gauss1_dT_eval(long long step, double dt, float T) {
    const double t = (double)step * dt;
    const double tau = t - 1.5 * (double)T;
    const float a = (float)(3.14159265358979323846 * tau / (double)T);
    const float dadT = (float)(-3.14159265358979323846 * t / ((double)T * (double)T));
    return -(float)kSqrt2e * (1.0f - 2.0f * a * a) * expf(-a * a) * dadT;
}
__device__ __forceinline__ double gauss1_dT_eval(long long step, double dt, double T) {
    const double t = (double)step * dt;
    const double tau = t - 1.5 * T;
    const double a = 3.14159265358979323846 * tau / T;
    const double dadT = -3.14159265358979323846 * t / (T * T);
    return -kSqrt2e * (1.0 - 2.0 * a * a) * exp(-a * a) * dadT;
}

// The FP32 source signal of kind `wavelet` from per-column FP64 constants
// m15T = -1.5 T and piT = pi / T set once per run: a = (t - 1.5 T) pi / T
// takes one FMA and one multiply in FP64 instead of a division per step,
// and the rest is the float expressions of ricker_eval / gauss1_eval.
__device__ __forceinline__ float wavelet_eval_pre(int wavelet, long long step, double dt, double m15T,
                                                  double piT) {
    const float a = (float)(fma((double)step, dt, m15T) * piT);
    if (wavelet == 1) return -(float)kSqrt2e * a * expf(-a * a);
    const float u = a * a;
    return (1.0f - 2.0f * u) * expf(-u);
}

// Source signal of kind `wavelet` (0 Ricker, 1 first derivative of a Gaussian).
template <typename T>
__device__ __forceinline__ T wavelet_eval(int wavelet, long long step, double dt, T period) {
    return wavelet == 1 ? gauss1_eval(step, dt, period) : ricker_eval(step, dt, period);
}
template <typename T>
__device__ __forceinline__ T wavelet_dT_eval(int wavelet, long long step, double dt, T period) {
    return wavelet == 1 ? gauss1_dT_eval(step, dt, period) : ricker_dT_eval(step, dt, period);
}

// Four consecutive elements from shared or global memory (16-byte aligned).
__device__ __forceinline__ void load4(const float* p, float (&x)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
}
__device__ __forceinline__ void load4(const double* p, double (&x)[4]) {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
}
__device__ __forceinline__ void load4_ro(const float* p, float (&x)[4]) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
}
__device__ __forceinline__ void load4_ro(const double* p, double (&x)[4]) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
}

__device__ __forceinline__ bool is_finite(float x) { return isfinite(x); }
__device__ __forceinline__ bool is_finite(double x) { return isfinite(x); }

// Compensated (Kahan) accumulation v += inc with carry c.  The explicit
// round-to-nearest intrinsics keep the compiler from contracting or
// reassociating the compensation away.
__device__ __forceinline__ float kahan_add(float v, float inc, float& c) {
    const float y = __fsub_rn(inc, c);
    const float t = __fadd_rn(v, y);
    c = __fsub_rn(__fsub_rn(t, v), y);
    return t;
}

// Asynchronous global -> shared copy of one 4- or 8-byte element (zero fill
// when src_bytes is 0; gsrc must still be a valid address), and the wait for
// all of this thread's outstanding ones.
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;"
                 ::"r"((uint32_t)__cvta_generic_to_shared(sdst)), "l"(gsrc), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;"
                 ::"r"((uint32_t)__cvta_generic_to_shared(sdst)), "l"(gsrc), "r"(src_bytes) : "memory");
}
// 16 bytes (both addresses 16-byte aligned), bypassing L1; src_bytes = 0
// zero-fills the destination.
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                 ::"r"((uint32_t)__cvta_generic_to_shared(sdst)), "l"(gsrc), "r"(src_bytes) : "memory");
}
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* sdst, const T* gsrc, bool ok) {
    if constexpr (sizeof(T) == 4) cp_async4(sdst, gsrc, ok ? 4 : 0);
    else cp_async8(sdst, gsrc, ok ? 8 : 0);
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

}  // namespace romk
