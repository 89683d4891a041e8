// Host stand-in for <cuda_runtime.h>, used only by the tests: it lets the
// device routines of the exact passes (csrc/gfs_tangent.cuh and the headers
// built on it) compile as plain C++ so that their traversal logic can be
// checked against the oracle on a CPU.
// The FP64 intrinsics become the plain IEEE operations they name (the
// harness is compiled with -ffp-contract=off, so nothing is fused).
#pragma once
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>
#define __device__
#define __host__
#define __global__
#define __forceinline__ inline
struct float4 {
  float x, y, z, w;
};
struct uint4 {
  unsigned x, y, z, w;
};
inline float4 make_float4(float x, float y, float z, float w) { return float4{x, y, z, w}; }
typedef int cudaError_t;
typedef void* cudaStream_t;
static const int cudaSuccess = 0;
inline double __dadd_rn(double a, double b) { return a + b; }
inline double __dsub_rn(double a, double b) { return a - b; }
inline double __dmul_rn(double a, double b) { return a * b; }
inline double __ddiv_rn(double a, double b) { return a / b; }
inline double __dsqrt_rn(double a) { return std::sqrt(a); }
inline unsigned atomicOr(unsigned* p, unsigned v) {
  const unsigned o = *p;
  *p |= v;
  return o;
}
inline unsigned long long atomicAdd(unsigned long long* p, unsigned long long v) {
  const unsigned long long o = *p;
  *p += v;
  return o;
}
inline unsigned __float_as_uint(float f) {
  unsigned u;
  std::memcpy(&u, &f, sizeof(u));
  return u;
}
inline float __uint_as_float(unsigned u) {
  float f;
  std::memcpy(&f, &u, sizeof(f));
  return f;
}
using std::fabs;
using std::fmax;
using std::fmin;
using std::sqrt;
