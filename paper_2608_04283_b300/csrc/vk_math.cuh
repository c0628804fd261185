// Small math helpers shared by the device code (and the host-side checker).
// FP32 on the device uses the SFU intrinsics; FP64 and host code use libm.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#define VK_HD __host__ __device__ __forceinline__

namespace vk {

enum SetKind : int { SET_WEIGHTED = 0, SET_CENTERED = 1, SET_DISCONTINUOUS = 2 };

// FP32 on the device uses the hardware approximations (about 1 ulp): the FP32
// path's tolerance is 1e-5 relative; FP64 and host code stay IEEE.
VK_HD float vsqrt(float x) {
#ifdef __CUDA_ARCH__
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
#else
  return sqrtf(x);
#endif
}
VK_HD double vsqrt(double x) { return sqrt(x); }
VK_HD float vabs(float x) { return fabsf(x); }
VK_HD double vabs(double x) { return fabs(x); }
VK_HD float vmax(float a, float b) { return fmaxf(a, b); }
VK_HD double vmax(double a, double b) { return fmax(a, b); }
VK_HD float vmin(float a, float b) { return fminf(a, b); }
VK_HD double vmin(double a, double b) { return fmin(a, b); }

VK_HD float vexp(float x) {
#ifdef __CUDA_ARCH__
  return __expf(x);
#else
  return expf(x);
#endif
}
VK_HD double vexp(double x) { return exp(x); }
// a * b + c in one rounding
VK_HD float vfma(float a, float b, float c) { return fmaf(a, b, c); }
VK_HD double vfma(double a, double b, double c) { return fma(a, b, c); }
// 1 where a >= 0, else 0 (the discontinuous set's Heaviside weight)
VK_HD float vstep(float a) { return a >= 0.0f ? 1.0f : 0.0f; }
VK_HD double vstep(double a) { return a >= 0.0 ? 1.0 : 0.0; }

// a / b
VK_HD float vdiv(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fdividef(a, b);
#else
  return a / b;
#endif
}
VK_HD double vdiv(double a, double b) { return a / b; }
VK_HD float vrcp(float x) {
#ifdef __CUDA_ARCH__
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
#else
  return 1.0f / x;
#endif
}
VK_HD double vrcp(double x) { return 1.0 / x; }

// Bit patterns of positive doubles order like the doubles, so a max can be
// reduced with an integer atomicMax on these bits.
VK_HD double bits_to_double(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  memcpy(&d, &b, sizeof(d));
  return d;
#endif
}
VK_HD unsigned long long double_to_bits(double d) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(d);
#else
  unsigned long long b;
  memcpy(&b, &d, sizeof(b));
  return b;
#endif
}

// Weight of the "+" part for an eigenvalue lam (Sec. 3.1):
//   weighted      alpha = 1 / (1 + exp(-k lam / max_j |lam_j|))      (Eq. 27)
//   discontinuous alpha = 1 if lam >= 0 else 0                        (Eq. 17)
//   centered      alpha = 1/2                                         (Eqs. 8-10)
template <class R>
VK_HD R alpha_w(R lam, R k_over_lmax, int set) {
  if (set == SET_WEIGHTED) return vrcp(R(1) + vexp(-k_over_lmax * lam));
  if (set == SET_DISCONTINUOUS) return vstep(lam);
  return R(0.5);
}

// (1 - e^{-y}) / y for y >= 0, accurate also for small y.
template <class R>
VK_HD R one_minus_exp_over(R y) {
  if (y < R(1e-3)) return R(1) - y * (R(0.5) - y * (R(1) / R(6) - y * R(1) / R(24)));
  return vdiv(R(1) - vexp(-y), y);
}

// Divided difference (alpha(l1) - alpha(l2)) / (l1 - l2) of the weights.  For the
// sigmoid, with x = k l / lmax, sigma(x1) - sigma(x2) = sigma(x1) (1 - sigma(x2))
// (1 - e^{-(x1 - x2)}), so the quotient needs no subtraction of nearly equal
// numbers and is exact at l1 = l2 (the derivative).
template <class R>
VK_HD R alpha_dd(R a1, R l1, R a2, R l2, R k_over_lmax, R lmax, int set) {
  if (set == SET_WEIGHTED) {
    const R dl = l1 - l2;
    // well separated speeds: the plain quotient loses no more than a few ulp
    // relative to alpha's own rounding
    if (vabs(dl) > R(0.05) * lmax) return (a1 - a2) * vrcp(dl);
    R y = k_over_lmax * dl;
    if (y >= R(0)) return a1 * (R(1) - a2) * k_over_lmax * one_minus_exp_over(y);
    return a2 * (R(1) - a1) * k_over_lmax * one_minus_exp_over(-y);
  }
  if (set == SET_DISCONTINUOUS) {
    R dl = l1 - l2;
    return vabs(dl) > R(1e-12) * lmax ? (a1 - a2) / dl : R(0);
  }
  return R(0);
}

// Storage conversions.
template <class T> struct Store;
// ld_keep: a global load whose line L2 should keep longer (an evict_last cache
// policy), for reads made well before another block reads the same line.
// ld_again: a second read of a value this thread loaded moments before (an L1
// hit, or shared memory where the caller staged the row there), issued as its
// own instruction so that the compiler cannot keep the first load's register
// live in its place; a generic-address load, valid for either state space.
#ifdef __CUDA_ARCH__
__device__ __forceinline__ unsigned long long l2_keep_policy() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
#endif
template <> struct Store<double> {
  typedef double R;
  static VK_HD double ld(const double* p) { return *p; }
  static VK_HD double ld_keep(const double* p) {
#ifdef __CUDA_ARCH__
    double v;
    asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(l2_keep_policy()));
    return v;
#else
    return *p;
#endif
  }
  static VK_HD double ld_again(const double* p) {
#ifdef __CUDA_ARCH__
    double v;
    asm volatile("ld.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
#else
    return *p;
#endif
  }
  static VK_HD void st(double* p, double v) { *p = v; }
};
template <> struct Store<float> {
  typedef float R;
  static VK_HD float ld(const float* p) { return *p; }
  static VK_HD float ld_keep(const float* p) {
#ifdef __CUDA_ARCH__
    float v;
    asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(l2_keep_policy()));
    return v;
#else
    return *p;
#endif
  }
  static VK_HD float ld_again(const float* p) {
#ifdef __CUDA_ARCH__
    float v;
    asm volatile("ld.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
#else
    return *p;
#endif
  }
  static VK_HD void st(float* p, float v) { *p = v; }
};
template <> struct Store<__nv_bfloat16> {
  typedef float R;
  static VK_HD float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  static VK_HD float ld_keep(const __nv_bfloat16* p) {
#ifdef __CUDA_ARCH__
    unsigned short b;
    asm volatile("ld.global.L2::cache_hint.b16 %0, [%1], %2;" : "=h"(b) : "l"(p), "l"(l2_keep_policy()));
    return __bfloat162float(__ushort_as_bfloat16(b));
#else
    return __bfloat162float(*p);
#endif
  }
  static VK_HD float ld_again(const __nv_bfloat16* p) {
#ifdef __CUDA_ARCH__
    unsigned short b;
    asm volatile("ld.b16 %0, [%1];" : "=h"(b) : "l"(p));
    return __bfloat162float(__ushort_as_bfloat16(b));
#else
    return __bfloat162float(*p);
#endif
  }
  static VK_HD void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

}  // namespace vk
