// Double-float ("float-float") arithmetic: a value is the unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi)/2, giving about 48 significant
// bits.  GB300 runs FP32 at 58 times its FP64 rate, so the complex128 FFT
// passes of the operator run in this format: the fields stay complex128 in
// memory and are converted on the way in and out.
//
// The error-free transformations are the classical ones: Knuth's TwoSum
// (s + e = a + b exactly, no branch), Dekker's Fast2Sum for |a| >= |b|, and
// the exact product error fmaf(a, b, -a b).  Addition follows the accurate
// (two TwoSum) scheme, multiplication adds the cross terms into the product
// error before renormalising.  No operation here relies on reassociation, and
// none contains a product that FMA contraction could change.
#pragma once

#include <cuda_runtime.h>

#include "cx.cuh"

namespace dda {

struct df {
  float hi, lo;
  __host__ __device__ constexpr df() : hi(0.f), lo(0.f) {}
  __host__ __device__ constexpr df(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ constexpr df(float h, float l, int) : hi(h), lo(l) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__host__ __device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return df(s, e, 0);
}

__host__ __device__ __forceinline__ df df_fast_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return df(s, b - (s - a), 0);
}

__host__ __device__ __forceinline__ df operator+(df a, df b) {
  df s = df_two_sum(a.hi, b.hi);
  const df t = df_two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = df_fast_sum(s.hi, s.lo);
  s.lo += t.lo;
  return df_fast_sum(s.hi, s.lo);
}

__host__ __device__ constexpr df operator-(df a) { return df(-a.hi, -a.lo, 0); }
__host__ __device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__host__ __device__ __forceinline__ df operator*(df a, df b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast_sum(p, e);
}

__host__ __device__ __forceinline__ bool operator==(df a, df b) {
  return a.hi == b.hi && a.lo == b.lo;
}
__host__ __device__ __forceinline__ bool operator!=(df a, df b) { return !(a == b); }

// Element-wise conversions complex128 <-> double-float complex (in place
// allowed: both are 16 bytes per value).
namespace {
__global__ void k_to_df(const double2* in, cx<df>* out, long n) {
  pdl_entry();
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    const double2 v = in[i];
    out[i] = mk<df>(df(v.x), df(v.y));
  }
}
__global__ void k_from_df(const cx<df>* in, double2* out, long n) {
  pdl_entry();
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    const cx<df> v = in[i];
    out[i] = make_double2((double)v.x, (double)v.y);
  }
}
}  // namespace

}  // namespace dda
