// Pipe-rate microbenchmark of the GPU the kernels run on: FP64 FMA/add, FP32
// FMA/add, 32- and 64-bit integer adds, FP64<->int64/FP32 and int32->FP32
// conversions (independent chains, 8 CTAs of 256 threads per SM), and HBM
// copy/read bandwidth.  Prints one JSON object (rates in 1e12 per second).
// All memory indexes are masked into bounds.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA error %s at %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

constexpr int ITERS = 4096;

template <typename T>
__global__ void k_fma(T* out, T a, T b) {
  T c0 = threadIdx.x, c1 = c0 + 1, c2 = c0 + 2, c3 = c0 + 3, c4 = c0 + 4, c5 = c0 + 5, c6 = c0 + 6, c7 = c0 + 7;
#pragma unroll 16
  for (int i = 0; i < ITERS; ++i) {
    c0 = c0 * a + b; c1 = c1 * a + b; c2 = c2 * a + b; c3 = c3 * a + b;
    c4 = c4 * a + b; c5 = c5 * a + b; c6 = c6 * a + b; c7 = c7 * a + b;
  }
  T s = c0 + c1 + c2 + c3 + c4 + c5 + c6 + c7;
  if (s == (T)12345.678) out[0] = s;
}

template <typename T>
__global__ void k_add(T* out, T b) {
  T c0 = threadIdx.x, c1 = c0 + 1, c2 = c0 + 2, c3 = c0 + 3, c4 = c0 + 4, c5 = c0 + 5, c6 = c0 + 6, c7 = c0 + 7;
#pragma unroll 16
  for (int i = 0; i < ITERS; ++i) {
    c0 = c0 + b; c1 = c1 + b; c2 = c2 + b; c3 = c3 + b;
    c4 = c4 + b; c5 = c5 + b; c6 = c6 + b; c7 = c7 + b;
  }
  T s = c0 + c1 + c2 + c3 + c4 + c5 + c6 + c7;
  if (s == (T)12345) out[0] = s;
}

__global__ void k_iadd32(int* out, int b) {
  int c0 = threadIdx.x, c1 = c0 + 1, c2 = c0 + 2, c3 = c0 + 3, c4 = c0 + 4, c5 = c0 + 5, c6 = c0 + 6, c7 = c0 + 7;
#pragma unroll 16
  for (int i = 0; i < ITERS; ++i) {
    asm volatile("add.s32 %0, %0, %8;\n\tadd.s32 %1, %1, %8;\n\tadd.s32 %2, %2, %8;\n\tadd.s32 %3, %3, %8;\n\t"
                 "add.s32 %4, %4, %8;\n\tadd.s32 %5, %5, %8;\n\tadd.s32 %6, %6, %8;\n\tadd.s32 %7, %7, %8;"
                 : "+r"(c0), "+r"(c1), "+r"(c2), "+r"(c3), "+r"(c4), "+r"(c5), "+r"(c6), "+r"(c7) : "r"(b));
  }
  int s = c0 + c1 + c2 + c3 + c4 + c5 + c6 + c7;
  if (s == 12345) out[0] = s;
}

__global__ void k_iadd64(long long* out, long long b) {
  long long c0 = threadIdx.x, c1 = c0 + 1, c2 = c0 + 2, c3 = c0 + 3, c4 = c0 + 4, c5 = c0 + 5, c6 = c0 + 6, c7 = c0 + 7;
#pragma unroll 16
  for (int i = 0; i < ITERS; ++i) {
    asm volatile("add.s64 %0, %0, %8;\n\tadd.s64 %1, %1, %8;\n\tadd.s64 %2, %2, %8;\n\tadd.s64 %3, %3, %8;\n\t"
                 "add.s64 %4, %4, %8;\n\tadd.s64 %5, %5, %8;\n\tadd.s64 %6, %6, %8;\n\tadd.s64 %7, %7, %8;"
                 : "+l"(c0), "+l"(c1), "+l"(c2), "+l"(c3), "+l"(c4), "+l"(c5), "+l"(c6), "+l"(c7) : "l"(b));
  }
  long long s = c0 + c1 + c2 + c3 + c4 + c5 + c6 + c7;
  if (s == 12345) out[0] = s;
}

__global__ void k_cvt_d2l(long long* out, long long b) {
  long long bits0 = 0x3ff0000000000000ll + threadIdx.x, bits1 = bits0 + 99; long long a0 = 0, a1 = 0;
#pragma unroll 16
  for (int i = 0; i < ITERS; ++i) { a0 ^= __double2ll_rn(__longlong_as_double(bits0)); a1 ^= __double2ll_rn(__longlong_as_double(bits1)); bits0 += b; bits1 += b; }
  if ((a0 ^ a1) == 12345) out[0] = a0;
}
__global__ void k_cvt_l2d(long long* out, long long b) {
  long long c0 = threadIdx.x, c1 = c0 + 7; long long a0 = 0, a1 = 0;
#pragma unroll 16
  for (int i = 0; i < ITERS; ++i) { a0 ^= __double_as_longlong(__ll2double_rn(c0)); a1 ^= __double_as_longlong(__ll2double_rn(c1)); c0 += b; c1 += b; }
  if ((a0 ^ a1) == 12345) out[0] = a0;
}
__global__ void k_cvt_d2f(int* out, long long b) {
  long long bits0 = 0x3ff0000000000000ll + threadIdx.x, bits1 = bits0 + 99; int a0 = 0, a1 = 0;
#pragma unroll 16
  for (int i = 0; i < ITERS; ++i) { a0 ^= __float_as_int(__double2float_rn(__longlong_as_double(bits0))); a1 ^= __float_as_int(__double2float_rn(__longlong_as_double(bits1))); bits0 += b; bits1 += b; }
  if ((a0 ^ a1) == 12345) out[0] = a0;
}
__global__ void k_cvt_i2f(float* out, int b) {
  int c0 = threadIdx.x, c1 = c0 + 7, c2 = c0 + 9, c3 = c0 + 11; float a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll 16
  for (int i = 0; i < ITERS; ++i) { a0 += __int2float_rn(c0); a1 += __int2float_rn(c1); a2 += __int2float_rn(c2); a3 += __int2float_rn(c3); c0 += b; c1 += b; c2 += b; c3 += b; }
  if (a0 + a1 + a2 + a3 == 12345.f) out[0] = a0;
}

__global__ void k_copy(const float4* __restrict__ a, float4* __restrict__ b, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) b[i] = a[i];
}

__global__ void k_read(const float4* __restrict__ a, float* out, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  float s = 0;
  for (; i < n; i += stride) { float4 v = a[i]; s += v.x + v.y + v.z + v.w; }
  if (s == 1.2345f) out[0] = s;
}

int main() {
  int nsm = 0; CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0));
  int clk = 0; CK(cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0));
  printf("{\"sms\": %d, \"clock_khz\": %d", nsm, clk);
  double* dout; float* fout; int* iout; long long* lout;
  CK(cudaMalloc(&dout, 64)); CK(cudaMalloc(&fout, 64)); CK(cudaMalloc(&iout, 64)); CK(cudaMalloc(&lout, 64));
  cudaEvent_t e0, e1; CK(cudaEventCreate(&e0)); CK(cudaEventCreate(&e1));
  int blocks = nsm * 8, threads = 256;
  double nthreads = (double)blocks * threads;
  float ms;
  auto rate = [&](double ops) { return ops / (ms * 1e-3) / 1e12; };
  // warmup
  k_fma<double><<<blocks, threads>>>(dout, 1.0000001, 1e-9);
  CK(cudaDeviceSynchronize());
#define TIME(launch, ops, name) \
  CK(cudaEventRecord(e0)); launch; CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1)); \
  CK(cudaEventElapsedTime(&ms, e0, e1)); printf(", \"%s\": %.4f", name, rate(ops));
  TIME((k_fma<double><<<blocks, threads>>>(dout, 1.0000001, 1e-9)), nthreads * ITERS * 8, "dfma_tinstr_s");
  TIME((k_add<double><<<blocks, threads>>>(dout, 1e-9)), nthreads * ITERS * 8, "dadd_tinstr_s");
  TIME((k_fma<float><<<blocks, threads>>>(fout, 1.0000001f, 1e-9f)), nthreads * ITERS * 8, "ffma_tinstr_s");
  TIME((k_add<float><<<blocks, threads>>>(fout, 1e-9f)), nthreads * ITERS * 8, "fadd_tinstr_s");
  TIME((k_iadd32<<<blocks, threads>>>(iout, 3)), nthreads * ITERS * 8, "iadd32_tops_s");
  TIME((k_iadd64<<<blocks, threads>>>(lout, 3)), nthreads * ITERS * 8, "iadd64_tops_s");
  TIME((k_cvt_d2l<<<blocks, threads>>>(lout, 12345)), nthreads * ITERS * 2, "cvt_f64_to_s64_t_s");
  TIME((k_cvt_l2d<<<blocks, threads>>>(lout, 3)), nthreads * ITERS * 2, "cvt_s64_to_f64_t_s");
  TIME((k_cvt_d2f<<<blocks, threads>>>(iout, 12345)), nthreads * ITERS * 2, "cvt_f64_to_f32_t_s");
  TIME((k_cvt_i2f<<<blocks, threads>>>(fout, 3)), nthreads * ITERS * 4, "cvt_s32_to_f32_t_s");
  size_t n = (size_t)1 << 28;  // 4 GiB of float4
  float4 *a, *b;
  CK(cudaMalloc(&a, n * 16)); CK(cudaMalloc(&b, n * 16));
  CK(cudaMemset(a, 0, n * 16)); CK(cudaMemset(b, 0, n * 16));
  for (int w = 0; w < 3; ++w) k_copy<<<nsm * 16, 512>>>(a, b, n);
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    CK(cudaEventRecord(e0)); k_copy<<<nsm * 16, 512>>>(a, b, n); CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1)); CK(cudaEventElapsedTime(&ms, e0, e1)); if (ms < best) best = ms;
  }
  printf(", \"copy_gbs\": %.1f", 2.0 * n * 16 / (best * 1e-3) / 1e9);
  best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    CK(cudaEventRecord(e0)); k_read<<<nsm * 16, 512>>>(a, fout, n); CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1)); CK(cudaEventElapsedTime(&ms, e0, e1)); if (ms < best) best = ms;
  }
  printf(", \"read_gbs\": %.1f}\n", 1.0 * n * 16 / (best * 1e-3) / 1e9);
  return 0;
}
