// Eigenvalues of a dense symmetric FP64 matrix (the Gram matrices of the
// entanglement spectrum), in two stages:
//  1. Householder reduction to tridiagonal form on the GPU (Golub and Van
//     Loan, Matrix Computations, Sec. 8.3): step k takes the reflector
//     H_k = I - beta v v^T of column k below the diagonal, and
//     H_k A H_k = A - v w^T - w v^T with w = beta A v - K v,
//     K = beta^2 (v^T A v) / 2.  Only the lower triangle is stored.  Blocked
//     as in LAPACK's dsytrd/dlatrd: the reflectors of a panel of kTriNb
//     columns are formed against the panel's starting matrix with the
//     panel's pending updates applied on the fly (the column c, and
//     A v = A0 v - V (W^T v) - W (V^T v)); after the panel the trailing
//     matrix takes A -= V W^T + W V^T in one FP64-accurate tensor-core
//     product (rank 2 kTriNb, lower-triangle tiles).  Within the panel every
//     step -- the column, the product A0 v (the whole cost of the
//     reduction), the pending terms and the dots -- reads a float-float copy
//     of the panel's starting matrix and runs in float-float arithmetic (48
//     significant bits, error-free products and sums on the FP32 pipe): on
//     this GPU FP64 arithmetic runs about 70 times slower than FP32, and the
//     float-float product is bound by HBM instead.  Per column three kernels:
//     the column and its reflector (k_pcol), the product (k_symv), its sums
//     and the pending terms (k_psum2).
//  2. The eigenvalues of the tridiagonal matrix by implicit QL steps with
//     shifts and deflation, on the host, one thread per matrix.
#include <algorithm>
#include <cmath>
#include <vector>

#include "eigsym.h"
#include "tc.cuh"

namespace edk {
namespace {

// the last 2 x 2 (or 1 x 1) block after every reflector was applied
__global__ void k_tail(const double* __restrict__ A, int m, double* d, double* e) {
  if (threadIdx.x != 0) return;
  const long long ld = m;
  d[m - 1] = A[(long long)(m - 1) * ld + (m - 1)];
  if (m >= 2) {
    d[m - 2] = A[(long long)(m - 2) * ld + (m - 2)];
    e[m - 2] = A[(long long)(m - 1) * ld + (m - 2)];
  }
}

// ---- blocked reduction: panel kernels.  The panel's columns are reduced
// against a float-float copy F of the panel's starting matrix: a = hi + lo
// with two FP32 values (48 significant bits), the whole matrix scaled by a
// power of two sigma = 2^sh that brings its largest entry into [1/2, 1).
// All per-column work runs in float-float arithmetic on the FP32 pipe --
// error-free products (FMA) and sums (Knuth's TwoSum) -- because this GPU's
// FP64 pipe is about 70 times slower; scalars (norms, beta, K) are FP64.  The
// reflectors take LAPACK's normalisation (dlarfg): v = x / (x_1 - alpha), so
// v_1 = 1, |v_i| <= 1 and beta = (|alpha| + |x_1|) / |alpha| lies in [1, 2],
// which keeps every float-float quantity within FP32's exponent range however
// small the column; v is the same for sigma A and A, w scales with sigma.  So
// the panel keeps sigma W (columns 0..nb-1) and V (columns nb..2nb-1) in WVf;
// at the panel's end they become the FP64 operands of the trailing update,
// WV = (W, V) and NVW = (-V, -W).  A column whose norm is below 2^-60 of the
// scaled matrix (below FP64's resolution of it) is taken as already reduced.
constexpr int kNb = kTriNb, kKw = 2 * kTriNb;
constexpr int kU = 64;             // edge of the product's units
constexpr int kSvWarps = 1;        // warps (units in flight) per CTA of the product
constexpr int kSvBuf = 3;          // staging buffers (sub-tiles in flight) per warp
constexpr int kSvCtas = 8;         // resident CTAs of the product per SM (shared memory)
constexpr int kTs = 34;            // row stride (float2) of its staging tiles: 16-byte aligned rows
constexpr int kPcolCtas = 128;     // most CTAs of k_pcol (partial-sum slots)
constexpr int kRowCtas = 4096;     // most CTAs of k_psum2 (partial-sum slots)
constexpr int kAmaxCtas = 1024;    // most CTAs of k_amax
constexpr int kPr = 8;             // rows per warp and step of k_pcol
constexpr int kPsT = 16;           // threads per row of k_psum2
static_assert(kPcolCtas == 128 && kRowCtas == 4096 && kAmaxCtas == 1024 && kU == 64,
              "tridiag_blocked_work_doubles counts these slots");

// a * 2^sh as hi + lo: hi = the leading 24 significant bits (truncated), lo =
// the next 29 rounded to 24, so hi + lo is within 2^-48 |a 2^sh|; built from
// the FP64 bit fields on the integer pipe.  Magnitudes below 2^-126 (after
// scaling) become zero; the caller keeps the scaled magnitude below 2^127.
__device__ __forceinline__ float2 split_scaled(double a, int sh) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(a);
  const unsigned s = (unsigned)(u >> 63) << 31;
  const int E = (int)((u >> 52) & 0x7ffu);
  if (E == 0) return make_float2(0.f, 0.f);  // zero or FP64 subnormal
  const int e = E - 1023 + sh;
  if (e < -126) return make_float2(0.f, 0.f);
  const unsigned long long M = u & 0xFFFFFFFFFFFFFull;
  const float hi = __uint_as_float(s | ((unsigned)(e + 127) << 23) | (unsigned)(M >> 29));
  const unsigned long long R = M & 0x1FFFFFFFull;  // the remaining 29 bits, unit 2^(e - 52)
  if (R == 0) return make_float2(hi, 0.f);
  const int nb = 64 - __clzll((long long)R);  // bit length, 1..29
  int el = e - 53 + nb;                       // exponent of R's leading bit
  unsigned frac;
  if (nb > 24) {
    const int d = nb - 24;
    unsigned long long q = (R + (1ull << (d - 1))) >> d;
    if (q >> 24) {
      q >>= 1;
      ++el;
    }
    frac = (unsigned)q & 0x7FFFFFu;
  } else {
    frac = (unsigned)(R << (24 - nb)) & 0x7FFFFFu;
  }
  if (el < -126) return make_float2(hi, 0.f);
  return make_float2(hi, __uint_as_float(s | ((unsigned)(el + 127) << 23) | frac));
}

// float-float value as FP64 (exact for a normalised pair)
__device__ __forceinline__ double df_to_d(float2 a) { return (double)a.x + (double)a.y; }

// (sh, sl) += (ah + al)(bh + bl): ah bh split exactly into p + e (FMA), p
// added to sh by TwoSum, the rounding error, e and the cross terms into sl
// (al bl, below 2^-48 of the product, is dropped).  The _rn intrinsics keep
// the compiler from contracting or reordering the error-free steps.
__device__ __forceinline__ void df_fma(float& sh, float& sl, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  const float e = fmaf(ah, bh, -p);
  const float s = __fadd_rn(sh, p);
  const float z = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, z)), __fsub_rn(p, z));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, fmaf(ah, bl, fmaf(al, bh, e))));
}
__device__ __forceinline__ void df_fma(float2& s, float2 a, float2 b) { df_fma(s.x, s.y, a.x, a.y, b.x, b.y); }

// (sh, sl) += (bh, bl) for two float-float sums (TwoSum of the leading parts)
__device__ __forceinline__ void df_add(float& sh, float& sl, float bh, float bl) {
  const float s = __fadd_rn(sh, bh);
  const float z = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, z)), __fsub_rn(bh, z));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, bl));
}
__device__ __forceinline__ void df_add(float2& s, float2 b) { df_add(s.x, s.y, b.x, b.y); }
// the pair renormalised (|lo| at most half an ulp of hi)
__device__ __forceinline__ float2 df_norm(float2 a) {
  const float s = __fadd_rn(a.x, a.y);
  return make_float2(s, __fsub_rn(a.y, __fsub_rn(s, a.x)));
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
// a b as a normalised pair
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  float2 s = make_float2(0.f, 0.f);
  df_fma(s, a, b);
  return df_norm(s);
}
// warp-wide float-float sum; lane 0's result is the one to use (the low
// parts of the other lanes may differ in their last bits)
__device__ __forceinline__ float2 df_warp_sum(float2 a) {
  for (int o = 16; o > 0; o >>= 1) {
    const float bh = __shfl_xor_sync(0xffffffffu, a.x, o), bl = __shfl_xor_sync(0xffffffffu, a.y, o);
    df_add(a.x, a.y, bh, bl);
  }
  return a;
}

__device__ inline unsigned long long warp_umax(unsigned long long x) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
    x = y > x ? y : x;
  }
  return x;
}

// programmatic dependent launch: let the stream's next kernel be scheduled
// now (its CTAs wait in pdl_enter), then wait until the previous kernel has
// finished and its writes are visible.  Called before any global access.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// largest |A[r][c]| over the trailing triangle r0 <= c <= r < m, per CTA, as
// FP64 bit patterns without the sign (their unsigned order is the order of
// the magnitudes); one warp per row
__global__ void __launch_bounds__(256) k_amax(const double* __restrict__ A, int m, int r0,
                                              unsigned long long* __restrict__ amx) {
  __shared__ unsigned long long red[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long ld = m;
  unsigned long long x = 0;
  for (int r = r0 + blockIdx.x * 8 + warp; r < m; r += gridDim.x * 8) {
    const double* row = A + (long long)r * ld;
    for (int c = r0 + lane; c <= r; c += 32) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(row[c]) & 0x7FFFFFFFFFFFFFFFull;
      x = b > x ? b : x;
    }
  }
  x = warp_umax(x);
  if (lane == 0) red[warp] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) x = red[w] > x ? red[w] : x;
    amx[blockIdx.x] = x;
  }
}

// the float-float copy F = split(A 2^sh) of the trailing triangle (row
// stride ldF); sh (the same in every CTA, written to *shp by CTA 0) brings
// the largest magnitude into [1/2, 1)
__global__ void __launch_bounds__(256) k_pconv(const double* __restrict__ A, float2* __restrict__ F, long long ldF,
                                               int m, int r0, const unsigned long long* __restrict__ amx, int na,
                                               int* shp) {
  pdl_enter();
  __shared__ int s_sh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) {
    unsigned long long x = 0;
    for (int b = lane; b < na; b += 32) x = amx[b] > x ? amx[b] : x;
    x = warp_umax(x);
    if (lane == 0) {
      s_sh = x == 0 ? 0 : 1022 - (int)(x >> 52);
      if (blockIdx.x == 0) *shp = s_sh;
    }
  }
  __syncthreads();
  const int sh = s_sh;
  const long long ld = m;
  for (int r = r0 + blockIdx.x * 8 + warp; r < m; r += gridDim.x * 8) {
    const double* row = A + (long long)r * ld;
    float2* out = F + (long long)r * ldF;
    for (int c = r0 + lane; c <= r; c += 32) out[c] = split_scaled(row[c], sh);
  }
}

// column c of the scaled matrix with the panel's pending updates, rows
// c+1..m-1: x = F[., c] - V (sigma W)[c]^T - (sigma W) V[c]^T, into vf; one
// warp per kPr rows at a time, lanes over the panel's terms.  Column j - 1
// (the previous reflector) is not stored yet: its w' = beta' p - K' v' (from
// the previous column's pf, vf, beta and K) is formed here row by row and
// stored with v' as it is used.  Per CTA: the partial sums (sigma W)^T x
// (slots 0..nb-1), V^T x (slots nb..2nb-1) over rows c+1.. and the sum of
// squares below row c+1 (slot 2nb); the last CTA to finish (a ticket on
// *ctr) adds them up in a fixed order and forms the reflector of column c:
// beta_c (FP64 and float-float), d_c, e_c (unscaled), vf[c+1], the factor
// tau (*tauf) with v = tau (x - alpha e_{c+1}) -- vf keeps x until k_psum2
// has applied it -- and, for j > 0, tu = ((sigma W)^T v, V^T v).
__global__ void __launch_bounds__(256) k_pcol(const float2* __restrict__ F, long long ldF, int m, int c, int j,
                                              float2* __restrict__ WVf, float2* __restrict__ vf,
                                              const float2* __restrict__ pf, double* beta, float2* betaf,
                                              const float2* Kf, const int* __restrict__ shp, float2* __restrict__ cp,
                                              unsigned* ctr, double* d, double* e, float2* __restrict__ tu,
                                              float2* tauf) {
  pdl_enter();
  __shared__ float2 acc[8][kKw + 1];
  __shared__ float2 tot[kKw + 1];
  __shared__ float2 s_alpha, s_vw, s_tau;
  __shared__ unsigned s_last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float2 z2 = make_float2(0.f, 0.f);
  const int jp = j - 1;  // the pending column formed here (none for j = 0)
  const float2 bq = j > 0 ? betaf[c - 1] : z2, kq = j > 0 ? *Kf : z2;
  // w'_r = beta' p_r - K' v'_r
  auto wprev = [&](float2 pr, float2 vr) {
    float2 s = z2;
    df_fma(s, bq, pr);
    df_fma(s, df_neg(kq), vr);
    return df_norm(s);
  };
  const float2 vpc = j > 0 ? vf[c] : z2, wpc = j > 0 ? wprev(pf[c], vpc) : z2;  // v'_c, w'_c
  const float2* rc = WVf + (long long)c * kKw;
  float2 w0 = lane < jp ? rc[lane] : z2, w1 = lane + 32 < jp ? rc[lane + 32] : z2;
  float2 v0 = lane < jp ? rc[kNb + lane] : z2, v1 = lane + 32 < jp ? rc[kNb + lane + 32] : z2;
  if (lane == jp) {
    w0 = wpc;
    v0 = vpc;
  }
  if (lane + 32 == jp) {
    w1 = wpc;
    v1 = vpc;
  }
  if (j > 0 && blockIdx.x == 0 && threadIdx.x == 0) {
    WVf[(long long)c * kKw + jp] = wpc;
    WVf[(long long)c * kKw + kNb + jp] = vpc;
  }
  float2 s2 = z2, dw0 = z2, dw1 = z2, dv0 = z2, dv1 = z2;
  for (int rb = c + 1 + (blockIdx.x * 8 + warp) * kPr; rb < m; rb += gridDim.x * 8 * kPr) {
    float2 a[kPr], t[kPr], rw0[kPr], rw1[kPr], rv0[kPr], rv1[kPr], wq[kPr], vq[kPr];
#pragma unroll
    for (int q = 0; q < kPr; ++q) {
      const int r = rb + q;
      const bool in = r < m;
      const float2* row = WVf + (long long)(in ? r : c) * kKw;
      a[q] = in ? F[(long long)r * ldF + c] : z2;
      rw0[q] = in && lane < jp ? row[lane] : z2;
      rv0[q] = in && lane < jp ? row[kNb + lane] : z2;
      rw1[q] = in && lane + 32 < jp ? row[lane + 32] : z2;
      rv1[q] = in && lane + 32 < jp ? row[kNb + lane + 32] : z2;
      vq[q] = j > 0 && in ? vf[r] : z2;  // v'_r, read before this kernel overwrites it
      wq[q] = j > 0 && in ? wprev(pf[r], vq[q]) : z2;
      if (lane == jp) {
        rw0[q] = wq[q];
        rv0[q] = vq[q];
      }
      if (lane + 32 == jp) {
        rw1[q] = wq[q];
        rv1[q] = vq[q];
      }
      float2 s = z2;
      df_fma(s, rv0[q], w0);
      df_fma(s, rw0[q], v0);
      df_fma(s, rv1[q], w1);
      df_fma(s, rw1[q], v1);
      t[q] = s;
    }
    if (j > 0) {
      for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int q = 0; q < kPr; ++q) {
          const float bh = __shfl_xor_sync(0xffffffffu, t[q].x, o), bl = __shfl_xor_sync(0xffffffffu, t[q].y, o);
          df_add(t[q].x, t[q].y, bh, bl);
        }
      }
      // TwoSum's low part is not commutative, so the butterfly leaves the
      // lanes with slightly different sums; x is a small difference of large
      // terms and every lane must use the value stored in vf: lane 0's
#pragma unroll
      for (int q = 0; q < kPr; ++q) {
        t[q].x = __shfl_sync(0xffffffffu, t[q].x, 0);
        t[q].y = __shfl_sync(0xffffffffu, t[q].y, 0);
      }
    }
#pragma unroll
    for (int q = 0; q < kPr; ++q) {
      const int r = rb + q;
      if (r >= m) break;
      float2 x = a[q];
      df_add(x, df_neg(t[q]));
      x = df_norm(x);
      if (lane == 0) {
        if (j > 0) {
          WVf[(long long)r * kKw + jp] = wq[q];
          WVf[(long long)r * kKw + kNb + jp] = vq[q];
        }
        vf[r] = x;
        if (r > c + 1) df_fma(s2, x, x);
      }
      df_fma(dw0, rw0[q], x);
      df_fma(dv0, rv0[q], x);
      df_fma(dw1, rw1[q], x);
      df_fma(dv1, rv1[q], x);
    }
  }
  acc[warp][lane] = dw0;
  acc[warp][lane + 32] = dw1;
  acc[warp][kNb + lane] = dv0;
  acc[warp][kNb + lane + 32] = dv1;
  if (lane == 0) acc[warp][kKw] = s2;
  __syncthreads();
  for (int k = threadIdx.x; k <= kKw; k += blockDim.x) {
    float2 s = z2;
    for (int w = 0; w < 8; ++w) df_add(s, acc[w][k]);
    cp[(long long)blockIdx.x * (kKw + 1) + k] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ctr, 1u) == gridDim.x - 1 ? 1u : 0u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the last CTA: the reflector of column c; thread (k, half) adds slot k
  // of every other CTA's partials, then the halves meet
  {
    const int k = threadIdx.x & (kKw - 1), hf = threadIdx.x >> 7;
    float2 s = z2;
#pragma unroll 16
    for (int b = hf; b < (int)gridDim.x; b += 2) df_add(s, cp[(long long)b * (kKw + 1) + k]);
    acc[hf][k] = s;
    if (warp == 0) {  // slot 2 nb (the sum of squares)
      float2 q = z2;
      for (int b = lane; b < (int)gridDim.x; b += 32) df_add(q, cp[(long long)b * (kKw + 1) + kKw]);
      q = df_warp_sum(q);
      if (lane == 0) tot[kKw] = q;
    }
  }
  __syncthreads();
  if (threadIdx.x < kKw) {
    float2 s = acc[0][threadIdx.x];
    df_add(s, acc[1][threadIdx.x]);
    tot[threadIdx.x] = df_norm(s);
  }
  if (warp == 0) {  // sum_i V[c,i] (sigma W)[c,i] (the diagonal's pending update)
    float2 t = z2;
    if (lane < j) df_fma(t, rc[kNb + lane], rc[lane]);
    if (lane + 32 < j) df_fma(t, rc[kNb + lane + 32], rc[lane + 32]);
    t = df_warp_sum(t);
    if (lane == 0) s_vw = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *ctr = 0u;
    const int sh = *shp;
    d[c] = ldexp(df_to_d(F[(long long)c * ldF + c]) - 2.0 * df_to_d(s_vw), -sh);
    const double tail = df_to_d(tot[kKw]);
    const double x0 = df_to_d(vf[c + 1]);
    const double nrm = sqrt(x0 * x0 + tail);
    double alpha = 0.0, tau = 0.0;
    if (tail == 0.0 || nrm < 0x1p-60) {  // nothing to annihilate
      e[c] = ldexp(x0, -sh);
      beta[c] = 0.0;
      betaf[c] = z2;
    } else {
      alpha = x0 >= 0.0 ? -nrm : nrm;
      tau = 1.0 / (x0 - alpha);  // v = tau x, v_{c+1} = tau (x0 - alpha)
      vf[c + 1] = split_scaled(x0 - alpha, 0);
      const double b = (nrm + fabs(x0)) / nrm;
      beta[c] = b;
      betaf[c] = split_scaled(b, 0);
      e[c] = ldexp(alpha, -sh);
    }
    s_alpha = split_scaled(alpha, 0);
    s_tau = split_scaled(tau, 0);
    *tauf = s_tau;
  }
  __syncthreads();
  if (j > 0 && threadIdx.x < kKw && (threadIdx.x & (kNb - 1)) < j) {  // the slots of the panel's columns
    float2 s = tot[threadIdx.x];
    df_fma(s, df_neg(s_alpha), WVf[(long long)(c + 1) * kKw + threadIdx.x]);
    tu[threadIdx.x] = df_mul(df_norm(s), s_tau);
  }
}

// unit t of the triangle, numbered row by row: (I, J), J <= I
__device__ __forceinline__ void unit_ij(long long t, int& I, int& J) {
  long long i = (long long)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
  while (i * (i + 1) / 2 > t) --i;
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  I = (int)i;
  J = (int)(t - i * (i + 1) / 2);
}

constexpr long long kSvSpin = 1LL << 24;  // polls of an mbarrier before k_symv gives up

// partial sums of p = (sigma A) v over the trailing triangle from the
// float-float copy (v = tau vf).  Units of 64 x 64 (I, J), J <= I, start at row and
// column u0 (r0 rounded down to even, so that every box starts on a 16-byte
// boundary; v is zero below r0) and are numbered row by row; one warp per
// unit, as 2 x 2 sub-tiles of 32 x 32, each brought into shared memory by
// one TMA box of 32 rows x 34 columns (the two extra columns give a 272-byte
// row pitch, free of bank conflicts; F streams through L2 once per column,
// marked evict-first), kSvBuf buffers per warp so that the next sub-tiles
// (across units) are in flight while one is summed, and the next unit's v
// values are fetched a unit ahead.  Lane = column for the
// column sums (a_ij v_i, kept in registers over the unit's rows), lane = row
// for the row sums (a_ij v_j); two independent float-float chains each.
// Diagonal entries count once, for their row.  Unit (I, J) writes its row
// sums to slot J and its column sums to slot TU + I of `part` (slot s, row i
// at part[s * m + i]) as float-float pairs.
__global__ void __launch_bounds__(32 * kSvWarps) k_symv(const __grid_constant__ CUtensorMap tmF, int m, int r0,
                                                        int u0, const float2* __restrict__ vf, const float2* tauf,
                                                        float2* __restrict__ part, int TU, long long nunits,
                                                        int* err) {
  __shared__ __align__(128) float2 tile[kSvWarps][kSvBuf][32][kTs];
  __shared__ __align__(16) float2 vs[kSvWarps][2 * kU];  // the unit's row values, then its column values
  __shared__ __align__(8) uint64_t bar[kSvWarps][kSvBuf];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long ld = m;
  const long long t0 = (long long)blockIdx.x * kSvWarps + w, nw = (long long)gridDim.x * kSvWarps;
  if (lane == 0) {
    for (int b = 0; b < kSvBuf; ++b) tc::mbar_init(&bar[w][b], 1);
    tc::fence_mbar_init();
  }
  __syncwarp();
  pdl_enter();
  // sub-tile k of this warp: unit t0 + (k / 4) nw, s = k % 4 -> column half
  // h = s / 2, row half g = s % 2, buffer k % kSvBuf; false if it holds
  // nothing to sum
  auto present = [&](long long k, int& I, int& J) {
    const long long t = t0 + (k >> 2) * nw;
    if (t >= nunits) return false;
    const int s = (int)(k & 3), h = s >> 1, g = s & 1;
    unit_ij(t, I, J);
    return !(I == J && g < h) && u0 + I * kU + 32 * g < m;
  };
  const uint64_t pol = tc::l2_evict_first();
  const float2 tau = *tauf;  // v = tau vf
  auto issue = [&](long long k, int buf) {
    int I, J;
    if (!present(k, I, J) || lane != 0) return;
    const int s = (int)(k & 3), h = s >> 1, g = s & 1;
    uint64_t* b = &bar[w][buf];
    tc::mbar_expect_tx(b, 32 * kTs * (unsigned)sizeof(float2));
    tc::tma_load_2d_hint(tile[w][buf], &tmF, u0 + J * kU + 32 * h, u0 + I * kU + 32 * g, b, pol);
  };
  for (int b = 0; b < kSvBuf; ++b) issue(b, b);
  // the v values of a unit (rows ib + lane, ib + 32 + lane, columns likewise),
  // fetched one unit ahead
  const float2 z2 = make_float2(0.f, 0.f);
  auto fetch_v = [&](long long t, float2* nv) {
    int I2, J2;
    unit_ij(t, I2, J2);
    const int a = u0 + I2 * kU + lane, c2 = u0 + J2 * kU + lane;
    nv[0] = a >= r0 && a < m ? vf[a] : z2;
    nv[1] = a + 32 >= r0 && a + 32 < m ? vf[a + 32] : z2;
    nv[2] = c2 >= r0 && c2 < m ? vf[c2] : z2;
    nv[3] = c2 + 32 >= r0 && c2 + 32 < m ? vf[c2 + 32] : z2;
  };
  float2 nv[4] = {z2, z2, z2, z2};
  if (t0 < nunits) fetch_v(t0, nv);
  unsigned phases = 0u;  // bit b: parity of the next phase of buffer b
  int I = 0, J = 0, ib = 0, jb = 0, bk = 0;
  bool diag = false;
  float rh0 = 0.f, rl0 = 0.f, rh1 = 0.f, rl1 = 0.f;  // row sums of rows ib + lane, ib + 32 + lane
  float ch = 0.f, cl = 0.f;                          // column sums of column jb + 32 h + lane
  for (long long k = 0;; ++k, bk = bk + 1 == kSvBuf ? 0 : bk + 1) {
    const long long t = t0 + (k >> 2) * nw;
    if (t >= nunits) break;
    const int s = (int)(k & 3), h = s >> 1, g = s & 1;
    if (s == 0) {
      unit_ij(t, I, J);
      diag = I == J;
      ib = u0 + I * kU;
      jb = u0 + J * kU;
      __syncwarp();
      vs[w][lane] = df_mul(nv[0], tau);
      vs[w][lane + 32] = df_mul(nv[1], tau);
      vs[w][kU + lane] = df_mul(nv[2], tau);
      vs[w][kU + lane + 32] = df_mul(nv[3], tau);
      if (t + nw < nunits) fetch_v(t + nw, nv);
      rh0 = rl0 = rh1 = rl1 = 0.f;
      __syncwarp();
    }
    if (g == 0) ch = cl = 0.f;
    const int j = jb + 32 * h + lane;
    int Ik, Jk;
    if (present(k, Ik, Jk)) {
      if (!tc::mbar_wait(&bar[w][bk], (phases >> bk) & 1u, kSvSpin)) {
        // give up: record it, let the other buffers' copies land, stop
        if (lane == 0) atomicExch(err, 3);
        for (int i = 1; i < kSvBuf; ++i) {
          int I2, J2;
          const int b2 = (bk + i) % kSvBuf;
          if (present(k + i, I2, J2)) tc::mbar_wait(&bar[w][b2], (phases >> b2) & 1u, kSvSpin);
        }
        return;
      }
      phases ^= 1u << bk;
      const float2(*buf)[kTs] = tile[w][bk];
      const float2* xr = &vs[w][32 * g];
      const float2* xc = &vs[w][kU + 32 * h];
      float c2h = 0.f, c2l = 0.f, r2h = 0.f, r2l = 0.f, r3h = 0.f, r3l = 0.f;
      if (!(diag && g == h)) {
#pragma unroll
        for (int li = 0; li < 32; li += 2) {
          const float2 a0 = buf[li][lane], x0 = xr[li];
          const float2 a1 = buf[li + 1][lane], x1 = xr[li + 1];
          df_fma(ch, cl, a0.x, a0.y, x0.x, x0.y);
          df_fma(c2h, c2l, a1.x, a1.y, x1.x, x1.y);
        }
#pragma unroll
        for (int q = 0; q < 32; q += 2) {
          const float4 a2 = *reinterpret_cast<const float4*>(&buf[lane][q]);
          const float4 x2 = *reinterpret_cast<const float4*>(&xc[q]);
          df_fma(r2h, r2l, a2.x, a2.y, x2.x, x2.y);
          df_fma(r3h, r3l, a2.z, a2.w, x2.z, x2.w);
        }
      } else {  // diagonal sub-tile: entry (li, q) is stored for q <= li only
#pragma unroll 4
        for (int li = 0; li < 32; ++li) {
          if (li > lane) {
            const float2 a0 = buf[li][lane], x0 = xr[li];
            df_fma(ch, cl, a0.x, a0.y, x0.x, x0.y);
          }
        }
#pragma unroll 4
        for (int q = 0; q < 32; ++q) {
          if (q <= lane) {
            const float2 a0 = buf[lane][q], x0 = xc[q];
            df_fma(r2h, r2l, a0.x, a0.y, x0.x, x0.y);
          }
        }
      }
      df_add(ch, cl, c2h, c2l);
      df_add(r2h, r2l, r3h, r3l);
      if (g == 0)
        df_add(rh0, rl0, r2h, r2l);
      else
        df_add(rh1, rl1, r2h, r2l);
    }
    if (g == 1 && j >= r0 && j < m) part[(long long)(TU + I) * ld + j] = make_float2(ch, cl);
    if (s == 3) {
      if (ib + lane >= r0 && ib + lane < m) part[(long long)J * ld + ib + lane] = make_float2(rh0, rl0);
      if (ib + 32 + lane < m) part[(long long)J * ld + ib + 32 + lane] = make_float2(rh1, rl1);
    }
    __syncwarp();
    issue(k + kSvBuf, bk);
  }
}

// p[i] for rows i >= r0 (pf, float-float, in the scaled matrix; vf[i] becomes
// v = tau vf): the unit slots that k_symv wrote (row slots 0..I(i), column
// slots TU + I(i) .. TU + Tn - 1, units from u0), minus the panel's pending
// terms V ((sigma W)^T v) + (sigma W) (V^T v); kPsT threads per row.  Per
// CTA: the partial sum of p.v; the last CTA to finish (a ticket on *ctr)
// adds them in a fixed order into K = beta^2 p.v / 2 (*Kf, float-float),
// which makes w = beta p - K v.
__global__ void __launch_bounds__(256) k_psum2(const float2* __restrict__ part, int m, int r0, int u0, int TU, int Tn,
                                               const float2* __restrict__ WVf, const float2* __restrict__ tu, int j,
                                               float2* __restrict__ vf, const float2* tauf, float2* __restrict__ pf,
                                               float2* __restrict__ pvp, const double* beta, int c, unsigned* ctr,
                                               float2* Kf) {
  pdl_enter();
  __shared__ float2 red[8];
  __shared__ unsigned s_last;
  const int q = threadIdx.x & (kPsT - 1), lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long ld = m;
  const float2 z2 = make_float2(0.f, 0.f);
  const float2 tau = *tauf;
  float2 pv = z2;
  constexpr int rows_cta = 256 / kPsT;
  for (int base = r0 + blockIdx.x * rows_cta; base < m; base += gridDim.x * rows_cta) {
    const int i = base + threadIdx.x / kPsT;
    float2 s = z2, corr = z2;
    if (i < m) {
      const int Ii = (i - u0) / kU;
#pragma unroll 8
      for (int J = q; J <= Ii; J += kPsT) df_add(s, part[(long long)J * ld + i]);
#pragma unroll 8
      for (int I = Ii + q; I < Tn; I += kPsT) df_add(s, part[(long long)(TU + I) * ld + i]);
      const float2* row = WVf + (long long)i * kKw;
#pragma unroll 4
      for (int k = q; k < j; k += kPsT) {
        df_fma(corr, row[kNb + k], tu[k]);
        df_fma(corr, row[k], tu[kNb + k]);
      }
    }
    df_add(s, df_neg(corr));
    for (int o = kPsT / 2; o > 0; o >>= 1) {
      const float bh = __shfl_xor_sync(0xffffffffu, s.x, o), bl = __shfl_xor_sync(0xffffffffu, s.y, o);
      df_add(s.x, s.y, bh, bl);
    }
    if (i < m && q == 0) {
      const float2 pi = df_norm(s), vi = df_mul(vf[i], tau);
      pf[i] = pi;
      vf[i] = vi;  // v itself from here on
      df_fma(pv, pi, vi);
    }
  }
  pv = df_warp_sum(pv);
  if (lane == 0) red[warp] = pv;
  __syncthreads();
  if (threadIdx.x == 0) {
    float2 t = z2;
    for (int w = 0; w < 8; ++w) df_add(t, red[w]);
    pvp[blockIdx.x] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ctr, 1u) == gridDim.x - 1 ? 1u : 0u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  float2 t = z2;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) df_add(t, pvp[b]);
  t = df_warp_sum(t);
  if (lane == 0) red[warp] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    float2 u = z2;
    for (int w = 0; w < 8; ++w) df_add(u, red[w]);
    const double b = beta[c];
    *Kf = split_scaled(0.5 * b * b * df_to_d(u), 0);
    *ctr = 0u;
  }
}

// w = beta p - K v over rows c+1..m-1, stored with v as column j of the
// panel (the panel's last column; the others are stored by the next
// column's k_pcol)
__global__ void __launch_bounds__(256) k_pw(int m, int c, int j, const float2* __restrict__ vf,
                                            const float2* __restrict__ pf, const float2* Kf, const float2* betaf,
                                            float2* __restrict__ WVf) {
  pdl_enter();
  const float2 b = betaf[c], K = df_neg(*Kf);
  for (int r = c + 1 + blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
    const float2 vr = vf[r];
    float2 s = make_float2(0.f, 0.f);
    df_fma(s, b, pf[r]);
    df_fma(s, K, vr);
    WVf[(long long)r * kKw + j] = df_norm(s);
    WVf[(long long)r * kKw + kNb + j] = vr;
  }
}

__device__ inline float block_maxf(float x, float* red) {
  for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = x;
  __syncthreads();
  if (w == 0) {
    x = l < (int)(blockDim.x >> 5) ? red[l] : 0.f;
    for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (l == 0) red[32] = x;
  }
  __syncthreads();
  return red[32];
}

// after the panel: the FP64 operands of the trailing update from WVf, column
// j of v scaled by 2^k and of w (sigma w unscaled) by 2^-k (their product
// unchanged) so that their largest magnitudes meet, and the negated swapped
// copy NVW; the trailing product slices each operand row with one exponent
// across all the panel's v and w, and this keeps either half from losing its
// low digits to the other.  One CTA per column.
__global__ void __launch_bounds__(256) k_pbal(int m, int k0, const float2* __restrict__ WVf, const int* shp,
                                              double* __restrict__ WV, double* __restrict__ NVW) {
  pdl_enter();
  __shared__ float red[33];
  const int j = blockIdx.x, c = k0 + j;
  const int sh = *shp;
  float mv = 0.f, mw = 0.f;
  for (int r = c + 1 + threadIdx.x; r < m; r += blockDim.x) {
    mv = fmaxf(mv, fabsf(WVf[(long long)r * kKw + kNb + j].x));
    mw = fmaxf(mw, fabsf(WVf[(long long)r * kKw + j].x));
  }
  mv = block_maxf(mv, red);
  mw = block_maxf(mw, red);
  int k = 0;
  if (mv > 0.f && mw > 0.f) {
    int ev, ew;
    frexpf(mv, &ev);
    frexpf(mw, &ew);
    k = ((ew - sh) - ev) / 2;  // w = (sigma w) 2^-sh
  }
  for (int r = c + 1 + threadIdx.x; r < m; r += blockDim.x) {
    const float2* row = WVf + (long long)r * kKw;
    const double vi = ldexp(df_to_d(row[kNb + j]), k), wi = ldexp(df_to_d(row[j]), -sh - k);
    WV[(long long)r * kKw + kNb + j] = vi;
    WV[(long long)r * kKw + j] = wi;
    NVW[(long long)r * kKw + j] = -vi;
    NVW[(long long)r * kKw + kNb + j] = -wi;
  }
}

}  // namespace

std::vector<TriPanel> tridiag_panels(int m) {
  std::vector<TriPanel> out;
  for (int k0 = 0; k0 < m - 2; k0 += kTriNb) {
    TriPanel t;
    t.k0 = k0;
    t.jb = std::min(kTriNb, m - 2 - k0);
    t.t0 = k0 + t.jb;
    out.push_back(t);
  }
  return out;
}

// launch with programmatic stream serialization: the kernel may be
// scheduled while the stream's previous kernel runs (each blocked-reduction
// kernel starts with pdl_enter)
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*k)(KArgs...), unsigned grid, unsigned block, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

ed_status tridiag_reduce_blocked(double* A, int m, double* work, double* d_host, double* e_host, cudaStream_t st,
                                 int sms, const TriBlocked& tb) {
  if (m <= 0) return ED_OK;
  auto cdiv = [](long long a, long long b) { return (a + b - 1) / b; };
  const int TU = (int)cdiv(m, kU);
  float2* vf = reinterpret_cast<float2*>(work);          // the latest column's x, then its v
  float2* pf = reinterpret_cast<float2*>(work + m);      // its p (scaled)
  double* beta = work + 2 * m;
  float2* betaf = reinterpret_cast<float2*>(work + 3 * m);
  double* d = work + 4 * m;
  double* e = work + 5 * m;
  float2* part = reinterpret_cast<float2*>(work + 6 * m);  // 2 TU slots of m
  float2* cp = part + 2LL * TU * m;                         // k_pcol partials (kPcolCtas x (2 nb + 1))
  float2* tu = cp + (long long)kPcolCtas * (kKw + 1);       // (sigma W)^T v, V^T v (2 nb)
  float2* pvp = tu + kKw;                                   // p.v partials (kRowCtas)
  auto* amx = reinterpret_cast<unsigned long long*>(pvp + kRowCtas);  // kAmaxCtas
  float2* Kf = reinterpret_cast<float2*>(amx + kAmaxCtas);  // K of the latest column
  int* shp = reinterpret_cast<int*>(Kf + 1);                // the panel's scale exponent
  unsigned* ctr = reinterpret_cast<unsigned*>(Kf + 2);      // tickets of k_pcol and k_psum2
  float2* tauf = Kf + 3;                                    // tau of the latest column
  ED_CUDA_TRY(cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned), st));
  const std::vector<TriPanel> pan = tridiag_panels(m);  // none for m < 3: k_tail alone
  for (size_t q = 0; q < pan.size(); ++q) {
    const TriPanel& P = pan[q];
    ED_CUDA_TRY(cudaMemsetAsync(tb.WV + (long long)P.k0 * kKw, 0, (size_t)(m - P.k0) * kKw * sizeof(double), st));
    ED_CUDA_TRY(cudaMemsetAsync(tb.NVW + (long long)P.k0 * kKw, 0, (size_t)(m - P.k0) * kKw * sizeof(double), st));
    // float-float copy of the panel's trailing triangle (rows and columns >= k0)
    {
      const int ga = (int)std::max(1LL, std::min((long long)kAmaxCtas, cdiv(m - P.k0, 8)));
      k_amax<<<ga, 256, 0, st>>>(A, m, P.k0, amx);
      const int gc = (int)std::max(1LL, std::min((long long)sms * 8, cdiv(m - P.k0, 8)));
      ED_CUDA_TRY(launch_pdl(k_pconv, gc, 256, st, A, tb.F, tb.ldF, m, P.k0, amx, ga, shp));
    }
    for (int j = 0; j < P.jb; ++j) {
      const int c = P.k0 + j;
      const int n = m - c - 1;  // rows and columns of the product, from c + 1
      const int g1 = (int)std::max(1LL, std::min((long long)kPcolCtas, cdiv(n, 8 * kPr)));
      ED_CUDA_TRY(launch_pdl(k_pcol, g1, 256, st, tb.F, tb.ldF, m, c, j, tb.WVf, vf, pf, beta, betaf, Kf, shp, cp, ctr,
                             d, e, tu, tauf));
      const int u0 = (c + 1) & ~1;  // the units' origin: even, so that the boxes start 16-byte aligned
      const long long Tn = cdiv(m - u0, kU), nu = Tn * (Tn + 1) / 2;
      const int gs = (int)std::max(1LL, std::min((long long)sms * kSvCtas, cdiv(nu, kSvWarps)));
      ED_CUDA_TRY(launch_pdl(k_symv, gs, 32 * kSvWarps, st, tb.tmF, m, c + 1, u0, vf, tauf, part, TU, nu, tb.err));
      const int g4 = (int)std::max(1LL, std::min((long long)kRowCtas, cdiv(n, 256 / kPsT)));
      ED_CUDA_TRY(launch_pdl(k_psum2, g4, 256, st, part, m, c + 1, u0, TU, (int)Tn, tb.WVf, tu, j, vf, tauf, pf, pvp,
                             beta, c, ctr + 1, Kf));
    }
    {
      const int c = P.k0 + P.jb - 1;
      const int g5 = (int)std::max(1LL, std::min((long long)sms * 2, cdiv(m - c - 1, 256)));
      ED_CUDA_TRY(launch_pdl(k_pw, g5, 256, st, m, c, P.jb - 1, vf, pf, Kf, betaf, tb.WVf));
    }
    ED_CUDA_TRY(launch_pdl(k_pbal, P.jb, 256, st, m, P.k0, tb.WVf, shp, tb.WV, tb.NVW));
    // trailing matrix (rows and columns >= t0): A -= V W^T + W V^T
    ED_TRY(oz_slice(tb.oz, tb.d_jobs + 2 * q, 2, 2LL * (m - P.t0), false, nullptr, st));
    ED_TRY(oz_gemm(tb.oz, tb.d_probs + q, 1, oz_tiles(m - P.t0, m - P.t0, 1), nullptr, st));
  }
  k_tail<<<1, 32, 0, st>>>(A, m, d, e);
  ED_CUDA_TRY(cudaGetLastError());
  ED_CUDA_TRY(cudaMemcpyAsync(d_host, d, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (m >= 2) ED_CUDA_TRY(cudaMemcpyAsync(e_host, e, (size_t)(m - 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
  return ED_OK;
}

ed_status tridiag_blocked_setup(OzContext* oz, double* A, int m, const OzOperand& opA, const OzOperand& opB,
                                const double* NVW, const double* WV, std::vector<OzSliceJob>& jobs,
                                std::vector<OzProblem>& probs) {
  for (const TriPanel& P : tridiag_panels(m)) {
    const int mm = m - P.t0;
    OzOperand a = opA, b = opB;
    int ma = 0, mb = 0;
    ED_TRY(oz_map(oz, &a, mm, kKw, true, &ma));
    ED_TRY(oz_map(oz, &b, mm, kKw, false, &mb));
    for (int side = 0; side < 2; ++side) {
      OzSliceJob jb{};
      jb.src = (side == 0 ? NVW : WV) + (long long)P.t0 * kKw;
      jb.sbase = 0;
      jb.ld = kKw;
      jb.rows = mm;
      jb.cols = kKw;
      jb.dst = side == 0 ? a.slices : b.slices;
      jb.exps = side == 0 ? a.exps : b.exps;
      jb.Kpad = kKw;
      jb.first = side == 0 ? 0 : mm;
      jobs.push_back(jb);
    }
    OzProblem pr{};
    pr.mapA = ma;
    pr.mapB = mb;
    pr.ea = a.exps;
    pr.eb = b.exps;
    pr.C = A + (long long)P.t0 * m + P.t0;
    pr.cbase = 0;
    pr.ldc = m;
    pr.M = pr.N = mm;
    pr.K = kKw;
    pr.acc = 1;
    pr.tiles_n = (mm + kOzBN - 1) / kOzBN;
    pr.tri = 1;
    pr.tile0 = 0;
    probs.push_back(pr);
  }
  return ED_OK;
}

// All eigenvalues of the symmetric tridiagonal matrix (d, e) by the
// root-free QL iteration (Pal, Walker and Kahan; Reinsch, "A stable,
// rational QR algorithm for the computation of the eigenvalues of an
// Hermitian, tridiagonal matrix", Math. Comp. 25, 1971; Parlett, The
// Symmetric Eigenvalue Problem, Sec. 8.15): the implicitly shifted QL sweep
// written in the squared off-diagonals e_i^2, so a rotation costs one
// reciprocal and one division and no square root.  For the unreduced block
// starting at row l: the shift is the eigenvalue of its leading 2 x 2 nearer
// d[l], the sweep runs from the bottom of the block up.  e[i] couples i and
// i+1; d is overwritten with the eigenvalues (unordered), each within a few
// eps of the matrix norm.  false if a block needs more than 60 sweeps.
bool tridiag_eigenvalues(std::vector<double>& d, std::vector<double>& e) {
  const int n = (int)d.size();
  if (n <= 1) return true;
  const double eps = std::ldexp(1.0, -53), eps2 = eps * eps;
  // an off-diagonal counts as zero below eps times its neighbours or below
  // eps times the norm of the whole matrix (eigenvalues far below the norm,
  // here the many vanishing ones of a Gram matrix, are resolved absolutely)
  double tnorm = 0.0;
  for (int i = 0; i < n; ++i)
    tnorm = std::max(tnorm, std::fabs(d[i]) + (i > 0 ? std::fabs(e[i - 1]) : 0.0) +
                                (i < n - 1 && i < (int)e.size() ? std::fabs(e[i]) : 0.0));
  const double tiny2 = (eps * tnorm) * (eps * tnorm);
  std::vector<double> e2(n, 0.0);
  for (int i = 0; i < n - 1; ++i) e2[i] = e[i] * e[i];
  for (int l = 0; l < n; ++l) {
    for (int iter = 0;; ++iter) {
      int m = l;  // end of the unreduced block that starts at l
      while (m < n - 1) {
        const double s = std::fabs(d[m]) + std::fabs(d[m + 1]);
        if (e2[m] <= eps2 * s * s || e2[m] <= tiny2) break;
        ++m;
      }
      if (m == l) break;
      if (iter == 60) return false;
      // shift: the eigenvalue of the leading 2 x 2 nearer d[l]
      const double rte = std::sqrt(e2[l]);
      double sigma = (d[l + 1] - d[l]) / (2.0 * rte);
      sigma = d[l] - rte / (sigma + std::copysign(std::hypot(sigma, 1.0), sigma));
      // the sweep, bottom up: rotation i carries c, s (as squares) and gamma
      double c = 1.0, s = 0.0, gamma = d[m] - sigma, p = gamma * gamma;
      for (int i = m - 1; i >= l; --i) {
        const double bb = e2[i], r = p + bb;
        if (i != m - 1) e2[i + 1] = s * r;
        const double oldc = c, ri = 1.0 / r;
        c = p * ri;
        s = bb * ri;
        const double oldgam = gamma, alpha = d[i];
        gamma = c * (alpha - sigma) - s * oldgam;
        d[i + 1] = oldgam + (alpha - gamma);
        p = c != 0.0 ? gamma * gamma / c : oldc * bb;
      }
      e2[l] = s * p;
      d[l] = sigma + gamma;
    }
  }
  return true;
}

}  // namespace edk

extern "C" ed_status ed_tridiag_eigenvalues(const double* d, const double* e, int64_t n, double* lambda) {
  if (n < 0 || (n > 0 && (!d || !lambda)) || (n > 1 && !e)) {
    edk::set_error("ed_tridiag_eigenvalues: n < 0 or a NULL array");
    return ED_EINVAL;
  }
  if (n == 0) return ED_OK;
  if (n > (int64_t)1 << 30) {
    edk::set_error("ed_tridiag_eigenvalues: n = %lld is too large", (long long)n);
    return ED_EINVAL;
  }
  std::vector<double> dd(d, d + n), ee(n > 1 ? e : d, n > 1 ? e + (n - 1) : d);
  if (!edk::tridiag_eigenvalues(dd, ee)) {
    edk::set_error("ed_tridiag_eigenvalues: the QL iteration did not converge");
    return ED_ENOCONV;
  }
  std::sort(dd.begin(), dd.end());
  std::copy(dd.begin(), dd.end(), lambda);
  return ED_OK;
}
