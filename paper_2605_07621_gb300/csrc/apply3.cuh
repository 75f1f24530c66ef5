// Device code shared by the class-sorted H|psi> kernels (paper Eq. (2)):
// the kernel parameter block, the arithmetic policies (FP32, FP64, exact
// 64-bit fixed point, fixed-point sums with FP64 weights), the fixed-point
// <-> FP64 conversions done by
// bit manipulation, and the TMA / mbarrier helpers.
#pragma once

#include <cstdint>
#include <cstring>

#include "ed_internal.h"

namespace edk {
struct P3 {
  Dev3 t;
  const DevBlock* blocks;
  const DevCross* cross;
  const long long* row_start;
  int nblk;
  int ncross;
  long long n_rows;
  int keep_fixed;  // row pass leaves every row as a 64-bit partial sum (cross terms added later)
};

// Policy types: S = staged / gathered values (and per-class sums), Y = the
// partial output kept in y between the passes, A = the accumulator, D = the
// diagonal, W = the per-class weights; dmul / wmul combine them.
struct PF32 {
  using S = float;
  using Y = float;
  using A = float;
  using D = float;
  using W = float;
  __device__ static float dmul(float d, float x) { return d * x; }
  __device__ static float wmul(float w, float s) { return w * s; }
  __device__ static float w(const Dev3& t, int c) { return t.w32[c]; }
  __device__ static float bw(const Dev3& t, int k) { return t.bond_w32[k]; }
  __device__ static float diagA(const Dev3& t, long long gA) { return t.A_d32[gA] + t.dc0_32; }
  __device__ static float diagB(const Dev3& t, long long gB) { return t.B_d32[gB]; }
  __device__ static float vab(const Dev3& t, unsigned z) {
    float v = 0.f;
    for (int q = 0; q < t.ncls_d; ++q) v += t.dw32[q] * (float)__popc(z & t.dmask[q]);
    return v;
  }
  __device__ static float diag(const Dev3& t, long long gA, long long gB, unsigned z) {
    float v = t.A_d32[gA] + t.B_d32[gB] + t.dc0_32;
    for (int q = 0; q < t.ncls_d; ++q) v += t.dw32[q] * (float)__popc(z & t.dmask[q]);
    return v;
  }
};
struct PF64 {
  using S = double;
  using Y = double;
  using A = double;
  using D = double;
  using W = double;
  __device__ static double dmul(double d, double x) { return d * x; }
  __device__ static double wmul(double w, double s) { return w * s; }
  __device__ static double w(const Dev3& t, int c) { return t.w64[c]; }
  __device__ static double bw(const Dev3& t, int k) { return t.bond_w64[k]; }
  __device__ static double diagA(const Dev3& t, long long gA) { return t.A_d64[gA] + t.dc0_64; }
  __device__ static double diagB(const Dev3& t, long long gB) { return t.B_d64[gB]; }
  __device__ static double vab(const Dev3& t, unsigned z) {
    double v = 0.0;
    for (int q = 0; q < t.ncls_d; ++q) v += t.dw64[q] * (double)__popc(z & t.dmask[q]);
    return v;
  }
  __device__ static double diag(const Dev3& t, long long gA, long long gB, unsigned z) {
    double v = t.A_d64[gA] + t.B_d64[gB] + t.dc0_64;
    for (int q = 0; q < t.ncls_d; ++q) v += t.dw64[q] * (double)__popc(z & t.dmask[q]);
    return v;
  }
};
struct PI64 {
  using S = long long;
  using Y = long long;
  using A = long long;
  using D = long long;
  using W = long long;
  __device__ static long long dmul(long long d, long long x) { return d * x; }
  __device__ static long long wmul(long long w, long long s) { return w * s; }
  __device__ static long long w(const Dev3& t, int c) { return t.wI[c]; }
  __device__ static long long bw(const Dev3& t, int k) { return t.bond_wI[k]; }
  __device__ static long long diagA(const Dev3& t, long long gA) { return (long long)t.A_dI[gA] + t.dc0_I; }
  __device__ static long long diagB(const Dev3& t, long long gB) { return (long long)t.B_dI[gB]; }
  __device__ static long long vab(const Dev3& t, unsigned z) {
    long long v = 0;
    for (int q = 0; q < t.ncls_d; ++q) v += t.dwI[q] * (long long)__popc(z & t.dmask[q]);
    return v;
  }
  __device__ static long long diag(const Dev3& t, long long gA, long long gB, unsigned z) {
    long long v = (long long)t.A_dI[gA] + (long long)t.B_dI[gB] + t.dc0_I;
    for (int q = 0; q < t.ncls_d; ++q) v += t.dwI[q] * (long long)__popc(z & t.dmask[q]);
    return v;
  }
};

// Fixed-point gathers with FP64 weights (models whose couplings are not
// dyadic): x is summed exactly per value class on the integer pipe as in
// PI64, and each class sum is multiplied by its FP64 weight once per
// element, the diagonal likewise (a few FP64 operations per element instead
// of one per matrix element).  The partial result between the passes is FP64
// in fixed-point units; the last store scales it by one power of two.
struct PC64 {
  using S = long long;
  using Y = double;
  using A = double;
  using D = double;
  using W = double;
  __device__ static double dmul(double d, long long x) { return d * (double)x; }
  __device__ static double wmul(double w, long long s) { return w * (double)s; }
  __device__ static double w(const Dev3& t, int c) { return t.w64[c]; }
  __device__ static double bw(const Dev3& t, int k) { return t.bond_w64[k]; }
  __device__ static double diagA(const Dev3& t, long long gA) { return t.A_d64[gA] + t.dc0_64; }
  __device__ static double diagB(const Dev3& t, long long gB) { return t.B_d64[gB]; }
  __device__ static double vab(const Dev3& t, unsigned z) { return PF64::vab(t, z); }
};

// 128-bit two's-complement integer: sums of products of 64-bit integers
struct I128 {
  unsigned long long lo;
  long long hi;
};
__host__ __device__ __forceinline__ I128 operator+(I128 a, I128 b) {
  I128 r;
  r.lo = a.lo + b.lo;
  r.hi = a.hi + b.hi + (r.lo < a.lo ? 1 : 0);
  return r;
}
__host__ __device__ __forceinline__ I128 mul_wide(long long a, long long b) {
  I128 r;
  r.lo = (unsigned long long)a * (unsigned long long)b;
#ifdef __CUDA_ARCH__
  r.hi = __mul64hi(a, b);
#else
  r.hi = (long long)(((__int128)a * (__int128)b) >> 64);
#endif
  return r;
}

// Wide integer weights (models whose couplings are not dyadic): every
// coupling and diagonal value is an FP64 number, i.e. an integer multiple of
// 2^-q_shift for one q_shift that covers them all; the class sums of the
// fixed-point x are multiplied by these 64-bit integer weights into an exact
// 128-bit sum, rounded once to FP64 per pass by bit manipulation (no FP64
// instruction per matrix element).  The row pass's partial result is kept in
// y as FP64 and the panel pass adds its own rounded sum to it.
struct AccW {
  I128 s;    // exact sum of this pass
  double p;  // partial result of the row pass (panel pass only)
  __device__ AccW() {}
  __device__ AccW(I128 v) : s(v), p(0.0) {}
  __device__ AccW(double v) : p(v) { s.lo = 0ull; s.hi = 0ll; }
  __device__ AccW& operator+=(I128 v) {
    s = s + v;
    return *this;
  }
};
struct PW {
  using S = long long;
  using Y = double;
  using A = AccW;
  using D = long long;
  using W = long long;
  __device__ static I128 dmul(long long d, long long x) { return mul_wide(d, x); }
  __device__ static I128 wmul(long long w, long long s) { return mul_wide(w, s); }
  __device__ static long long w(const Dev3& t, int c) { return t.wI[c]; }
  __device__ static long long bw(const Dev3& t, int k) { return t.bond_wI[k]; }
  __device__ static long long diagA(const Dev3& t, long long gA) { return t.A_dW[gA] + t.dc0_I; }
  __device__ static long long diagB(const Dev3& t, long long gB) { return t.B_dW[gB]; }
  __device__ static long long vab(const Dev3& t, unsigned z) { return PI64::vab(t, z); }
};

// ---------------------------------------------------------------- fixed point <-> FP64 by bit manipulation

__host__ __device__ __forceinline__ unsigned long long f64_bits(double v) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(v);
#else
  unsigned long long u;
  memcpy(&u, &v, 8);
  return u;
#endif
}
__host__ __device__ __forceinline__ double bits_f64(unsigned long long u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double v;
  memcpy(&v, &u, 8);
  return v;
#endif
}
__host__ __device__ __forceinline__ int clz64(unsigned long long u) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)u);
#else
  return __builtin_clzll(u);
#endif
}

// round(v * 2^sh_base) (ties away from zero) for |v| < 2^E, sh_base = P - E
__host__ __device__ __forceinline__ long long to_fixed(double v, int sh_base) {
  const unsigned long long u = f64_bits(v);
  const int s = (int)(u >> 63);
  int e = (int)((u >> 52) & 0x7ffull);
  unsigned long long m = u & 0xFFFFFFFFFFFFFull;
  if (e == 0) {
    if (m == 0) return 0;
    e = 1;
  } else {
    m |= 1ull << 52;
  }
  const int sh = e - 1075 + sh_base;
  long long X;
  if (sh >= 0) X = (long long)(m << sh);
  else if (sh > -64) X = (long long)((m + (1ull << (-sh - 1))) >> (-sh));
  else X = 0;
  return s ? -X : X;
}

// Y * 2^e2 rounded to nearest (ties to even) FP64
__host__ __device__ __forceinline__ double from_fixed(long long Y, int e2) {
  if (Y == 0) return 0.0;
  const unsigned long long s = Y < 0 ? 1ull : 0ull;
  unsigned long long u = s ? (unsigned long long)(-Y) : (unsigned long long)Y;
  int p = 63 - clz64(u);
  unsigned long long mant;
  if (p <= 52) {
    mant = u << (52 - p);
  } else {
    const int sh = p - 52;
    mant = u >> sh;
    const unsigned long long rem = u & ((1ull << sh) - 1);
    const unsigned long long half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (mant & 1ull))) {
      ++mant;
      if (mant >> 53) {
        mant >>= 1;
        ++p;
      }
    }
  }
  const int ex = p + e2 + 1023;
  if (ex <= 0) return s ? -0.0 : 0.0;
  if (ex >= 2047) return bits_f64((s << 63) | (0x7ffull << 52));
  return bits_f64((s << 63) | ((unsigned long long)ex << 52) | (mant & 0xFFFFFFFFFFFFFull));
}

// v * 2^e2 rounded to nearest (ties to even) FP64, v a 128-bit integer
__host__ __device__ __forceinline__ double from_fixed128(I128 v, int e2) {
  const unsigned long long s = v.hi < 0 ? 1ull : 0ull;
  unsigned long long lo = v.lo, hi = (unsigned long long)v.hi;
  if (s) {  // magnitude
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0ull ? 1ull : 0ull);
  }
  if (hi == 0ull && lo == 0ull) return 0.0;
  // normalise: leading one at bit 63 of h, the bits below it in h then l
  int p;
  unsigned long long h, l;
  if (hi != 0ull) {
    const int n = clz64(hi);
    p = 127 - n;
    h = n == 0 ? hi : (hi << n) | (lo >> (64 - n));
    l = lo << n;
  } else {
    const int n = clz64(lo);
    p = 63 - n;
    h = lo << n;
    l = 0ull;
  }
  unsigned long long mant = h >> 11;  // 53 bits
  const unsigned long long rbit = (h >> 10) & 1ull;
  const bool sticky = (h & 0x3FFull) != 0ull || l != 0ull;
  if (rbit && (sticky || (mant & 1ull))) {
    ++mant;
    if (mant >> 53) {
      mant >>= 1;
      ++p;
    }
  }
  const int ex = p + e2 + 1023;
  if (ex <= 0) return s ? -0.0 : 0.0;
  if (ex >= 2047) return bits_f64((s << 63) | (0x7ffull << 52));
  return bits_f64((s << 63) | ((unsigned long long)ex << 52) | (mant & 0xFFFFFFFFFFFFFull));
}

__device__ __forceinline__ int out_exp(const Dev3& t, const int* emax) { return (emax[0] - 1022) - t.P - t.q_shift; }

template <class Pol>
__device__ __forceinline__ void store_out(typename Pol::Y* y, long long i, typename Pol::A v, bool final_,
                                          int e2) {
  y[i] = v;
}
template <>
__device__ __forceinline__ void store_out<PI64>(long long* y, long long i, long long v, bool final_, int e2) {
  if (final_) reinterpret_cast<double*>(y)[i] = from_fixed(v, e2);
  else y[i] = v;
}
template <>
__device__ __forceinline__ void store_out<PC64>(double* y, long long i, double v, bool final_, int e2) {
  y[i] = final_ ? ldexp(v, e2) : v;
}
template <>
__device__ __forceinline__ void store_out<PW>(double* y, long long i, AccW v, bool final_, int e2) {
  y[i] = v.p + from_fixed128(v.s, e2);  // both passes store real values
}

// ---------------------------------------------------------------- TMA / mbarrier

__device__ __forceinline__ unsigned s_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void bar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(bar)) : "memory");
}
__device__ __forceinline__ void bar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bar_expect(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_u32(bar)) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   s_u32(dst)),
               "l"(src), "r"(bytes), "r"(s_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool bar_wait(unsigned long long* bar, unsigned parity) {
  for (long long i = 0; i < (1ll << 22); ++i) {
    unsigned ok;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok)
                 : "r"(s_u32(bar)), "r"(parity)
                 : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ int find_blk(const long long* row_start, int nblk, long long row) {
  int lo = 0, hi = nblk - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (row_start[mid] <= row) lo = mid; else hi = mid - 1;
  }
  return lo;
}

inline int n_sms(int dev) {
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    n = 148;
  }
  return n;
}

}  // namespace edk
