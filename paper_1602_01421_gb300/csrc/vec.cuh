// Vectorised load/store of short row fragments (<= 16 bytes per access).
#pragma once
#include <cuda_runtime.h>

namespace fe {

template <typename T, int NE> struct VecT;
template <> struct VecT<float, 1> { using type = float; };
template <> struct VecT<float, 2> { using type = float2; };
template <> struct VecT<float, 4> { using type = float4; };
template <> struct VecT<double, 1> { using type = double; };
template <> struct VecT<double, 2> { using type = double2; };

// elements per 16-byte access for a row of B elements of T
template <typename T, int B>
struct FragOf {
  static constexpr int NE = (B * (int)sizeof(T)) <= 16 ? B : 16 / (int)sizeof(T);
  static constexpr int NCH = B / NE;
};

template <typename T, int NE>
__device__ __forceinline__ void ld_frag(const T* p, T* f) {
  using V = typename VecT<T, NE>::type;
  V x = __ldg(reinterpret_cast<const V*>(p));
  const T* xs = reinterpret_cast<const T*>(&x);
#pragma unroll
  for (int i = 0; i < NE; ++i) f[i] = xs[i];
}

// 32-byte fragments (one 256-bit load per lane; sm_100 and later).  The address must be
// 32-byte aligned.  Read-only (non-coherent) path, like __ldg.
template <>
__device__ __forceinline__ void ld_frag<float, 8>(const float* p, float* f) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(f[0]), "=f"(f[1]), "=f"(f[2]), "=f"(f[3]), "=f"(f[4]), "=f"(f[5]), "=f"(f[6]), "=f"(f[7])
      : "l"(p));
}
template <>
__device__ __forceinline__ void ld_frag<double, 4>(const double* p, double* f) {
  asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];"
      : "=d"(f[0]), "=d"(f[1]), "=d"(f[2]), "=d"(f[3])
      : "l"(p));
}

// plain (coherent) load: for data written earlier in the same kernel or aliasing a store
template <typename T, int NE>
__device__ __forceinline__ void ld_frag_rw(const T* p, T* f) {
  using V = typename VecT<T, NE>::type;
  V x = *reinterpret_cast<const V*>(p);
  const T* xs = reinterpret_cast<const T*>(&x);
#pragma unroll
  for (int i = 0; i < NE; ++i) f[i] = xs[i];
}

template <typename T, int NE>
__device__ __forceinline__ void st_frag(T* p, const T* f) {
  using V = typename VecT<T, NE>::type;
  V x;
  T* xs = reinterpret_cast<T*>(&x);
#pragma unroll
  for (int i = 0; i < NE; ++i) xs[i] = f[i];
  *reinterpret_cast<V*>(p) = x;
}

// Load a whole row of B elements (contiguous, 16-byte aligned when B*sizeof(T) >= 16).
template <typename T, int B>
__device__ __forceinline__ void ld_row(const T* p, T* f) {
  using F = FragOf<T, B>;
#pragma unroll
  for (int c = 0; c < F::NCH; ++c) ld_frag<T, F::NE>(p + c * F::NE, f + c * F::NE);
}
template <typename T, int B>
__device__ __forceinline__ void ld_row_rw(const T* p, T* f) {
  using F = FragOf<T, B>;
#pragma unroll
  for (int c = 0; c < F::NCH; ++c) ld_frag_rw<T, F::NE>(p + c * F::NE, f + c * F::NE);
}
template <typename T, int B>
__device__ __forceinline__ void st_row(T* p, const T* f) {
  using F = FragOf<T, B>;
#pragma unroll
  for (int c = 0; c < F::NCH; ++c) st_frag<T, F::NE>(p + c * F::NE, f + c * F::NE);
}

// FP64 -> FP32 by truncating the significand (IEEE 754 binary64 -> binary32 field by field:
// sign, exponent rebiased from 1023 to 127, top 23 of the 52 fraction bits), on the integer
// units so that the FP64 pipe is not touched.  Relative error below 2^-23; magnitudes below
// 2^-126 become signed zero, above the binary32 range infinity.
__device__ __forceinline__ float f64_to_f32_trunc(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  const unsigned frac = ((hi & 0xfffffu) << 3) | (lo >> 29);
  unsigned bits = sign | ((unsigned)e << 23) | frac;
  if (e <= 0) bits = sign;
  if (e >= 255) bits = sign | 0x7f800000u;
  return __uint_as_float(bits);
}

// FP32 -> FP64 by integer operations (exact for normal values, infinities and NaN; subnormal
// inputs give a signed zero), keeping the conversion off the FP64 pipe.
__device__ __forceinline__ double f32_to_f64_flush(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  unsigned long long bits = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long ef = e == 0xffu ? 0x7ffull : (unsigned long long)(e + 896u);
  if (e != 0) bits |= (ef << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}

// Conversion of a block element to the Gram's arithmetic type: FP64 -> FP32 by integer
// truncation (f64_to_f32_trunc), otherwise a plain cast.
template <typename TC, typename T>
__device__ __forceinline__ TC to_arith(T x) {
  if constexpr (sizeof(T) == 8 && sizeof(TC) == 4) return f64_to_f32_trunc((double)x);
  else return (TC)x;
}

}  // namespace fe
