// A pair of FP32 values on Blackwell's packed f32x2 arithmetic (FFMA2, FMUL2, FADD2: two FP32
// operations per instruction and lane), usable as the scalar type R of the flux templates so
// that one instantiation computes both sides of a face at once (one side in each half). A
// product is kept pending (M2) and fused into the addition or subtraction that consumes it,
// since the packed intrinsics are not contracted by the compiler; a pending product used any
// other way is rounded into a P2 first. Division, square root, exp and erfc run per half.
#pragma once
#include <cuda_runtime.h>

namespace gks {

struct M2;
struct P2 {
  float2 v;
  P2() = default;
  __device__ __forceinline__ P2(float2 x) : v(x) {}
  __device__ __forceinline__ P2(float a, float b) : v(make_float2(a, b)) {}
  __device__ __forceinline__ explicit P2(double a) : v(make_float2((float)a, (float)a)) {}
  __device__ __forceinline__ explicit P2(float a) : v(make_float2(a, a)) {}
  __device__ __forceinline__ explicit P2(int a) : v(make_float2((float)a, (float)a)) {}
  __device__ __forceinline__ P2(const M2& m);
  __device__ __forceinline__ float lo() const { return v.x; }
  __device__ __forceinline__ float hi() const { return v.y; }
};
// a pending product a * b
struct M2 {
  float2 a, b;
};
__device__ __forceinline__ P2::P2(const M2& m) : v(__fmul2_rn(m.a, m.b)) {}
__device__ __forceinline__ float2 neg2(float2 x) { return make_float2(-x.x, -x.y); }

__device__ __forceinline__ M2 operator*(const P2& a, const P2& b) { return {a.v, b.v}; }
__device__ __forceinline__ M2 operator*(const M2& a, const P2& b) { return {P2(a).v, b.v}; }
__device__ __forceinline__ M2 operator*(const P2& a, const M2& b) { return {a.v, P2(b).v}; }
__device__ __forceinline__ M2 operator*(const M2& a, const M2& b) { return {P2(a).v, P2(b).v}; }
__device__ __forceinline__ P2 operator+(const P2& a, const P2& b) { return __fadd2_rn(a.v, b.v); }
__device__ __forceinline__ P2 operator+(const M2& m, const P2& c) { return __ffma2_rn(m.a, m.b, c.v); }
__device__ __forceinline__ P2 operator+(const P2& c, const M2& m) { return __ffma2_rn(m.a, m.b, c.v); }
__device__ __forceinline__ P2 operator+(const M2& m, const M2& n) {
  return __ffma2_rn(m.a, m.b, P2(n).v);
}
__device__ __forceinline__ P2 operator-(const P2& a) { return neg2(a.v); }
__device__ __forceinline__ M2 operator-(const M2& m) { return {neg2(m.a), m.b}; }
__device__ __forceinline__ P2 operator-(const P2& a, const P2& b) {
  return __fadd2_rn(a.v, neg2(b.v));
}
__device__ __forceinline__ P2 operator-(const M2& m, const P2& c) {
  return __ffma2_rn(m.a, m.b, neg2(c.v));
}
__device__ __forceinline__ P2 operator-(const P2& c, const M2& m) {
  return __ffma2_rn(neg2(m.a), m.b, c.v);
}
__device__ __forceinline__ P2 operator-(const M2& m, const M2& n) {
  return __ffma2_rn(neg2(n.a), n.b, P2(m).v);
}
__device__ __forceinline__ P2 operator/(const P2& a, const P2& b) {
  return P2(a.v.x / b.v.x, a.v.y / b.v.y);
}
__device__ __forceinline__ P2& operator+=(P2& a, const P2& b) { return a = a + b; }
__device__ __forceinline__ P2& operator+=(P2& a, const M2& b) { return a = a + b; }
__device__ __forceinline__ P2& operator-=(P2& a, const P2& b) { return a = a - b; }
__device__ __forceinline__ P2& operator-=(P2& a, const M2& b) { return a = a - b; }
__device__ __forceinline__ P2& operator*=(P2& a, const P2& b) { return a = P2(a * b); }
// true when it holds in both halves (both sides)
__device__ __forceinline__ bool operator>(const P2& a, const P2& b) {
  return (a.v.x > b.v.x) && (a.v.y > b.v.y);
}
__device__ __forceinline__ bool operator<(const P2& a, const P2& b) { return b > a; }
__device__ __forceinline__ bool operator!=(const P2& a, const P2& b) {
  return (a.v.x != b.v.x) || (a.v.y != b.v.y);
}

__device__ __forceinline__ P2 k_div(const P2& a, const P2& b) {
  return P2(__fdividef(a.v.x, b.v.x), __fdividef(a.v.y, b.v.y));
}
__device__ __forceinline__ P2 k_sqrt(const P2& x) { return P2(sqrtf(x.v.x), sqrtf(x.v.y)); }
__device__ __forceinline__ P2 k_exp(const P2& x) { return P2(expf(x.v.x), expf(x.v.y)); }
__device__ __forceinline__ P2 k_erfc(const P2& x) { return P2(erfcf(x.v.x), erfcf(x.v.y)); }
__device__ __forceinline__ P2 k_abs(const P2& x) { return P2(fabsf(x.v.x), fabsf(x.v.y)); }
__device__ __forceinline__ float hsum(const P2& a) { return a.v.x + a.v.y; }

}  // namespace gks
