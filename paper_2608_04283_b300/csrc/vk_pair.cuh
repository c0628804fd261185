// Two FP32 lanes per thread: the arithmetic type of the paired step kernel.
//
// A thread of the paired march owns two neighbouring cells of a row and carries
// every quantity of the step as a pair (cell x in .x, cell x + 1 in .y).  On
// sm_100-class parts the FP32 pipes execute packed two-lane add, sub, mul and
// fma (the f32x2 instructions of PTX ISA 8.6), so one instruction advances both
// cells; the special functions (exp, reciprocal, square root) stay one per lane.
// Operators are defined so that the system code written for a scalar compute
// type (vk_systems.cuh) compiles unchanged for pairs; the host build (the CPU
// checker) evaluates the lanes one at a time.
#pragma once
#include "vk_math.cuh"

namespace vk {

struct f2 {
  float x, y;
  f2() = default;
  VK_HD constexpr f2(float a, float b) : x(a), y(b) {}
  VK_HD constexpr f2(double a) : x((float)a), y((float)a) {}   // broadcast (R(0.5) in generic code)
  VK_HD constexpr f2(float a) : x(a), y(a) {}
  VK_HD constexpr f2(int a) : x((float)a), y((float)a) {}
};

#ifdef __CUDA_ARCH__
__device__ __forceinline__ unsigned long long f2_pack(f2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ f2 f2_unpack(unsigned long long r) {
  f2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ f2 operator+(f2 a, f2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(r);
}
__device__ __forceinline__ f2 operator-(f2 a, f2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(r);
}
__device__ __forceinline__ f2 operator*(f2 a, f2 b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(r);
}
// a * b + c in one rounding
__device__ __forceinline__ f2 vfma(f2 a, f2 b, f2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)), "l"(f2_pack(c)));
  return f2_unpack(r);
}
#else
inline f2 operator+(f2 a, f2 b) { return f2(a.x + b.x, a.y + b.y); }
inline f2 operator-(f2 a, f2 b) { return f2(a.x - b.x, a.y - b.y); }
inline f2 operator*(f2 a, f2 b) { return f2(a.x * b.x, a.y * b.y); }
inline f2 vfma(f2 a, f2 b, f2 c) { return f2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y)); }
#endif
VK_HD f2 operator-(f2 a) { return f2(-a.x, -a.y); }
VK_HD f2& operator+=(f2& a, f2 b) { return a = a + b; }
VK_HD f2& operator-=(f2& a, f2 b) { return a = a - b; }
VK_HD f2& operator*=(f2& a, f2 b) { return a = a * b; }
VK_HD f2 operator/(f2 a, f2 b) { return f2(vdiv(a.x, b.x), vdiv(a.y, b.y)); }

// lane by lane
VK_HD f2 vsqrt(f2 a) { return f2(vsqrt(a.x), vsqrt(a.y)); }
VK_HD f2 vrcp(f2 a) { return f2(vrcp(a.x), vrcp(a.y)); }
VK_HD f2 vexp(f2 a) { return f2(vexp(a.x), vexp(a.y)); }
VK_HD f2 vabs(f2 a) { return f2(fabsf(a.x), fabsf(a.y)); }
VK_HD f2 vmax(f2 a, f2 b) { return f2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
VK_HD f2 vmin(f2 a, f2 b) { return f2(fminf(a.x, b.x), fminf(a.y, b.y)); }
VK_HD f2 vdiv(f2 a, f2 b) { return f2(vdiv(a.x, b.x), vdiv(a.y, b.y)); }
// 1 where a >= 0, else 0 (the discontinuous set's Heaviside weight)
VK_HD f2 vstep(f2 a) { return f2(a.x >= 0.0f ? 1.0f : 0.0f, a.y >= 0.0f ? 1.0f : 0.0f); }
// alpha's normaliser: lg is one grid-wide value in both lanes
VK_HD f2 lam_norm(f2 lg, f2 local) { return lg.x > 0.0f ? lg : local; }

}  // namespace vk
