// Element types of Krylov vectors: real or complex, FP64 or FP32.
#pragma once
#include <cuda_runtime.h>
#include <type_traits>

template <typename T> struct CxOf;
template <> struct CxOf<double> { using t = double2; };
template <> struct CxOf<float> { using t = float2; };

template <typename T, bool C>
struct Elem {
  using V = std::conditional_t<C, typename CxOf<T>::t, T>;
  static __device__ __forceinline__ double re(const V& v) {
    if constexpr (C) return (double)v.x; else return (double)v;
  }
  static __device__ __forceinline__ double im(const V& v) {
    if constexpr (C) return (double)v.y; else return 0.0;
  }
  static __device__ __forceinline__ V make(double r, double i) {
    if constexpr (C) { V v; v.x = (T)r; v.y = (T)i; return v; } else { (void)i; return (T)r; }
  }
};
