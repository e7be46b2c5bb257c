// Complex arithmetic for the DDA kernels: one struct for float and double,
// laid out like float2 / double2 so box fields load as 8- or 16-byte words.
#pragma once

#include <cuda_runtime.h>

#include "launch.cuh"

namespace dda {

template <typename R>
struct alignas(2 * sizeof(R)) cx {
  R x, y;
};

template <typename R>
__host__ __device__ __forceinline__ cx<R> mk(R a, R b) {
  cx<R> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) {
  return mk<R>(a.x + b.x, a.y + b.y);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) {
  return mk<R>(a.x - b.x, a.y - b.y);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) {
  return mk<R>(s * a.x, s * a.y);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> conj(cx<R> a) {
  return mk<R>(a.x, -a.y);
}
// a * b with b conjugated when C is true.
template <bool C, typename R>
__host__ __device__ __forceinline__ cx<R> mulc(cx<R> a, cx<R> b) {
  if (C) return mk<R>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
  return a * b;
}
template <typename R>
__host__ __device__ __forceinline__ R norm2(cx<R> a) {
  return a.x * a.x + a.y * a.y;
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> zero() {
  return mk<R>(R(0), R(0));
}
// Convert between precisions.
template <typename R, typename S>
__host__ __device__ __forceinline__ cx<R> cvt(cx<S> a) {
  return mk<R>(R(a.x), R(a.y));
}

}  // namespace dda
