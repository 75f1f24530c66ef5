// FP64-accurate reductions shared by the Krylov kernels.
#pragma once

namespace edk {

// float-float accumulation: TwoSum (Knuth) of the running sum and TwoProd
// (Dekker, with one FMA) of each product
struct FAcc {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float a) {
    float s = hi + a;
    float bp = s - hi;
    float err = (hi - (s - bp)) + (a - bp);
    hi = s;
    lo += err;
  }
  __device__ __forceinline__ void add_prod(float x, float y) {
    float p = x * y;
    float e = fmaf(x, y, -p);
    add(p);
    lo += e;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

template <typename T>
struct DotAcc;
template <>
struct DotAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add_prod(double x, double y) { s = fma(x, y, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct DotAcc<float> {
  FAcc f;
  __device__ __forceinline__ void add_prod(float x, float y) { f.add_prod(x, y); }
  __device__ __forceinline__ double value() const { return f.value(); }
};

// sum over the CTA (blockDim.x a multiple of 32, at most 1024); valid in thread 0
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red_[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red_[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (l < (int)(blockDim.x >> 5)) ? red_[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;
}

}  // namespace edk
