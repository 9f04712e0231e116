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

}  // namespace fe
