// Krylov layer on top of H|psi> (the paper's "core operation in any
// Krylov-based method"): Lanczos vector kernels with FP64 reductions,
// ground-state driver (plain FP64, FP32 storage, and FP32 + FP64 restarted
// refinement), and the continued-fraction Green's function.
#include <cuda_bf16.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "apply3.cuh"
#include "ed_internal.h"
#include "krylov.h"
#include "reduce.cuh"

namespace edk {

constexpr int kRedThreads = 256;

// ---------------------------------------------------------------- reductions

// sum of partials in fixed order -> out[0]; op 1: sqrt of the sum
__global__ void k_finalize(const double* __restrict__ part, int n, double* out, int op) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
  double s = block_sum(v);
  if (threadIdx.x == 0) out[0] = op == 1 ? sqrt(s > 0.0 ? s : 0.0) : s;
}

template <typename T>
__global__ void k_dot(const T* __restrict__ a, const T* __restrict__ b, long long n, double* part) {
  DotAcc<T> acc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc.add_prod(a[i], b[i]);
  double s = block_sum(acc.value());
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// w -= beta * vprev (beta from device memory; skipped when use_beta == 0); alpha partial <v, w>
template <typename T>
__global__ void k_lz_a(T* __restrict__ w, const T* __restrict__ v, const T* __restrict__ vprev, const double* beta,
                       int use_beta, long long n, double* part) {
  const T bt = use_beta ? (T)beta[0] : (T)0;
  DotAcc<T> acc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    T wi = w[i];
    if (use_beta) {
      wi -= bt * vprev[i];
      w[i] = wi;
    }
    acc.add_prod(v[i], wi);
  }
  double s = block_sum(acc.value());
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// w -= alpha * v; partial ||w||^2
template <typename T>
__global__ void k_lz_b(T* __restrict__ w, const T* __restrict__ v, const double* alpha, long long n, double* part) {
  const T al = (T)alpha[0];
  DotAcc<T> acc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    T wi = w[i] - al * v[i];
    w[i] = wi;
    acc.add_prod(wi, wi);
  }
  double s = block_sum(acc.value());
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// FP64 with the exact fixed-point H|psi>: w -= alpha * v, partial ||w||^2,
// and the largest biased exponent of w (atomic max into *ew, zeroed before)
__global__ void k_lz_b_emax(double* __restrict__ w, const double* __restrict__ v, const double* alpha, long long n,
                            double* part, int* ew) {
  const double al = alpha[0];
  DotAcc<double> acc;
  int em = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double wi = w[i] - al * v[i];
    w[i] = wi;
    acc.add_prod(wi, wi);
    em = max(em, (int)(((unsigned long long)__double_as_longlong(wi) >> 52) & 0x7ffull));
  }
  for (int o = 16; o > 0; o >>= 1) em = max(em, __shfl_down_sync(0xffffffffu, em, o));
  if ((threadIdx.x & 31) == 0) atomicMax(ew, em);
  double s = block_sum(acc.value());
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// out = w / beta, and the fixed-point copy X of out that the next H|psi>
// takes: |out| < 2^E with E = E(max|w|) - E(beta) + 1 (E(y): 2^(E-1) <= |y|
// < 2^E), X = round(out * 2^(P - E)); the biased-exponent form of E
// (E + 1022) goes to *ex for the apply's output scale
__global__ void k_lz_c_fixed(const double* __restrict__ w, double* __restrict__ out, long long* __restrict__ X,
                             const double* beta, const int* ew, int* ex, int P, long long n) {
  const double b = beta[0];
  const double inv = b > 0.0 ? 1.0 / b : 0.0;
  const int eb = (int)(((unsigned long long)__double_as_longlong(b) >> 52) & 0x7ffull);
  const int E = (ew[0] - 1022) - (eb - 1022) + 1;
  if (blockIdx.x == 0 && threadIdx.x == 0) ex[0] = E + 1022;
  const int sh = P - E;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double o = w[i] * inv;
    out[i] = o;
    X[i] = to_fixed(o, sh);
  }
}

// out = w / beta
template <typename T>
__global__ void k_lz_c(const T* __restrict__ w, T* __restrict__ out, const double* beta, long long n) {
  const double b = beta[0];
  const T inv = (T)(b > 0.0 ? 1.0 / b : 0.0);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = w[i] * inv;
}

// y[i] = s * x[i] (types may differ); s from host
template <typename TI, typename TO>
__global__ void k_scale_cvt(const TI* x, TO* y, double s, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (TO)((double)x[i] * s);
}

// y[i] += s * x[i]
template <typename TI, typename TO>
__global__ void k_axpy(const TI* __restrict__ x, TO* __restrict__ y, double s, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (TO)((double)y[i] + s * (double)x[i]);
}

// y[i] += s[0] * x[i], s read on the device (reorthogonalisation)
template <typename TI, typename TO>
__global__ void k_axpy_dev(const TI* __restrict__ x, TO* __restrict__ y, const double* s, double sign, long long n) {
  const double c = sign * s[0];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (TO)((double)y[i] + c * (double)x[i]);
}

__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(float v) { return (double)v; }
__device__ __forceinline__ double to_d(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

template <typename TO>
__device__ __forceinline__ TO from_d(double v);
template <>
__device__ __forceinline__ double from_d<double>(double v) { return v; }
template <>
__device__ __forceinline__ float from_d<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_d<__nv_bfloat16>(double v) { return __float2bfloat16((float)v); }

template <typename TI, typename TO>
__global__ void k_cvt(const TI* __restrict__ x, TO* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = from_d<TO>(to_d(x[i]));
}

// x += s * v for a stored basis vector of any storage type
template <typename TB, typename TO>
__global__ void k_axpy_basis(const TB* __restrict__ v, TO* __restrict__ x, double s, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = from_d<TO>(to_d(x[i]) + s * to_d(v[i]));
}

// appends this step's alpha and beta to the device history at the step
// index the device keeps (so the same launch serves every step of a graph)
__global__ void k_hist_push(const double* __restrict__ sl, double* __restrict__ hist, int* counter) {
  const int j = *counter;
  hist[2 * j] = sl[0];
  hist[2 * j + 1] = sl[1];
  *counter = j + 1;
}

// x = sum_j s_j V_j over an FP32 basis (V_j = V + j n).  Each coefficient
// comes as a float pair (hi, lo), s_j = hi + lo to about 48 bits; the
// product hi * v is split exactly by an fma into its rounded value and
// error, and the terms are summed in float-float arithmetic (Knuth's
// TwoSum), so the combination carries about 42 bits without one FP64
// instruction per term.  The explicit _rn operations keep the compiler
// from contracting the error-free transformations.
__device__ __forceinline__ void ff_acc(float& hi, float& lo, float2 c, float v) {
  const float p = __fmul_rn(c.x, v);
  const float pe = fmaf(c.y, v, fmaf(c.x, v, -p));
  const float t = __fadd_rn(hi, p);
  const float bb = __fsub_rn(t, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  hi = t;
  lo = __fadd_rn(lo, __fadd_rn(e, pe));
}

__global__ void k_combine_f32(const float* __restrict__ V, long long n, int m, const float2* __restrict__ s,
                              double* __restrict__ x) {
  extern __shared__ float2 sc[];
  for (int j = threadIdx.x; j < m; j += blockDim.x) sc[j] = s[j];
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float hi = 0.f, lo = 0.f;
    int j = 0;
    for (; j + 4 <= m; j += 4) {
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = __ldg(V + (long long)(j + u) * n + i);
#pragma unroll
      for (int u = 0; u < 4; ++u) ff_acc(hi, lo, sc[j + u], v[u]);
    }
    for (; j < m; ++j) ff_acc(hi, lo, sc[j], __ldg(V + (long long)j * n + i));
    x[i] = (double)hi + (double)lo;
  }
}

// Continued fraction G(w) = CF_p(w + i eta + E0) - CF_h(E0 - w - i eta),
// CF(z) = w0 / (z - a0 - b1^2 / (z - a1 - ...)), one thread per frequency.
__device__ __forceinline__ void cf_eval(double zr, double zi, const double* a, const double* b, int m, double w0,
                                        double* gr, double* gi) {
  double tr = 0.0, ti = 0.0;  // tail g
  for (int n = m - 1; n >= 1; --n) {
    double dr = zr - a[n] - tr, di = zi - ti;
    double den = dr * dr + di * di;
    double b2 = b[n - 1] * b[n - 1];
    tr = b2 * dr / den;
    ti = -b2 * di / den;
  }
  double dr = zr - a[0] - tr, di = zi - ti;
  double den = dr * dr + di * di;
  *gr = w0 * dr / den;
  *gi = -w0 * di / den;
}

__global__ void k_green_cf(const double* omega, int n_omega, double eta, double e0, const double* ap, const double* bp,
                           int mp, double wp, const double* ah, const double* bh, int mh, double wh, double* G) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_omega) return;
  double w = omega[j];
  double gr = 0.0, gi = 0.0, r, i;
  if (mp > 0 && wp > 0.0) {
    cf_eval(w + e0, eta, ap, bp, mp, wp, &r, &i);
    gr += r;
    gi += i;
  }
  if (mh > 0 && wh > 0.0) {
    cf_eval(e0 - w, -eta, ah, bh, mh, wh, &r, &i);
    gr -= r;
    gi -= i;
  }
  G[2 * j] = gr;
  G[2 * j + 1] = gi;
}

// phi[a', b'] = sign * psi[a, b] for a row (side A) or column (side B) remap
__global__ void k_fermion_remap(const double* __restrict__ psi, long long dA_src, long long dB_src,
                                double* __restrict__ phi, long long dA_dst, long long dB_dst, const int* __restrict__ map,
                                const signed char* __restrict__ sgn, int side) {
  long long n = dA_dst * dB_dst;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    long long r = i / dB_dst, cidx = i % dB_dst;
    double v = 0.0;
    if (side == 0) {
      int sr = map[r];
      if (sr >= 0) v = sgn[r] * psi[(long long)sr * dB_src + cidx];
    } else {
      int sc = map[cidx];
      if (sc >= 0) v = sgn[cidx] * psi[r * dB_src + sc];
    }
    phi[i] = v;
  }
}

// out = (w - alpha v - beta vprev) * inv_next  (second pass of a two-pass eigenvector)
template <typename T>
__global__ void k_lz_rerun(const T* __restrict__ w, const T* __restrict__ v, const T* vprev, T alpha, T beta,
                           T inv_next, T* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    T r = w[i] - alpha * v[i];
    if (vprev) r -= beta * vprev[i];
    out[i] = r * inv_next;
  }
}

// Blocked classical Gram-Schmidt against a contiguous basis V[j][i] (row j
// = basis vector j, leading dimension ldv): part[j*chunks + c] = partial
// <V_j, w> over chunk c; then w -= sum_j h_j V_j.
template <typename T>
__global__ void k_basis_dots(const T* __restrict__ V, long long ldv, const T* __restrict__ w, long long n,
                             double* part, int chunks) {
  const int j = blockIdx.y;
  const T* vj = V + (long long)j * ldv;
  DotAcc<T> acc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)chunks * blockDim.x)
    acc.add_prod(vj[i], w[i]);
  double s = block_sum(acc.value());
  if (threadIdx.x == 0) part[(long long)j * chunks + blockIdx.x] = s;
}

__global__ void k_finalize_many(const double* __restrict__ part, int chunks, int m, double* out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += part[(long long)j * chunks + c];
    out[j] = s;
  }
}

template <typename T>
__global__ void k_basis_update(const T* __restrict__ V, long long ldv, int m, const double* __restrict__ h,
                               T* __restrict__ w, long long n) {
  extern __shared__ double hs[];
  for (int j = threadIdx.x; j < m; j += blockDim.x) hs[j] = h[j];
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < m; ++j) acc = fma(hs[j], (double)V[(long long)j * ldv + i], acc);
    w[i] = (T)((double)w[i] - acc);
  }
}

// ---------------------------------------------------------------- host helpers

int grid_for(const ed_ctx* c, long long n) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    cudaGetLastError();
    sms = 148;
  }
  long long g = (n + kRedThreads - 1) / kRedThreads;
  long long cap = (long long)sms * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

ed_status ensure_scratch(ed_ctx* c) {
  if (!c->d_partials) {
    ED_TRY(dev_alloc(c, (void**)&c->d_partials, sizeof(double) * (kMaxPartials + 64 + kMaxBasis)));
  }
  if (!c->h_pinned) {
    if (cudaMallocHost((void**)&c->h_pinned, sizeof(double) * 64) != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMallocHost failed");
      return ED_ENOMEM;
    }
  }
  return ED_OK;
}

// scalar slots in the scratch area after the partials
double* slot(ed_ctx* c, int k) { return c->d_partials + kMaxPartials + k; }
// reorthogonalisation coefficients after the scalar slots
double* hcoef(ed_ctx* c) { return c->d_partials + kMaxPartials + 64; }

template <typename T>
ed_status dot_dev(ed_ctx* c, const T* a, const T* b, long long n, double* out, cudaStream_t st, int op) {
  int g = grid_for(c, n);
  k_dot<T><<<g, kRedThreads, 0, st>>>(a, b, n, c->d_partials);
  k_finalize<<<1, kRedThreads, 0, st>>>(c->d_partials, g, out, op);
  ED_CUDA_TRY(cudaGetLastError());
  return ED_OK;
}
template ed_status dot_dev<double>(ed_ctx*, const double*, const double*, long long, double*, cudaStream_t, int);
template ed_status dot_dev<float>(ed_ctx*, const float*, const float*, long long, double*, cudaStream_t, int);

ed_status read_scalars(ed_ctx* c, int first, int count, double* out, cudaStream_t st) {
  ED_CUDA_TRY(cudaMemcpyAsync(c->h_pinned, slot(c, first), sizeof(double) * count, cudaMemcpyDeviceToHost, st));
  ED_CUDA_TRY(cudaStreamSynchronize(st));
  std::memcpy(out, c->h_pinned, sizeof(double) * count);
  return ED_OK;
}

// ---------------------------------------------------------------- tridiagonal eigensolver

// number of eigenvalues of T (diag a, off b) below x: Sturm sequence count
static int sturm_count(const double* a, const double* b, int m, double x) {
  int cnt = 0;
  double q = 1.0;
  for (int i = 0; i < m; ++i) {
    double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
    q = a[i] - x - (i > 0 ? bb / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

double tridiag_lowest(const double* a, const double* b, int m) {
  if (m == 1) return a[0];
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < m; ++i) {
    double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i < m - 1 ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  double span = hi - lo;
  lo -= 1e-12 * span + 1e-300;
  hi += 1e-12 * span + 1e-300;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(a, b, m, mid) >= 1) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// eigenvector of the lowest eigenvalue theta by inverse iteration with a
// partially pivoted tridiagonal solve of (T - theta) s = r.
void tridiag_vector(const double* a, const double* b, int m, double theta, std::vector<double>& s) {
  s.assign(m, 1.0);
  if (m == 1) { s[0] = 1.0; return; }
  double scale = 0.0;
  for (int i = 0; i < m; ++i) scale = std::max(scale, std::fabs(a[i]) + (i < m - 1 ? std::fabs(b[i]) : 0.0));
  double shift = theta - 1e-14 * (scale > 0 ? scale : 1.0);
  for (int i = 0; i < m; ++i) s[i] = 1.0 / std::sqrt((double)m) * (1.0 + 0.01 * ((i * 7919) % 13));
  std::vector<double> d(m), du(m), du2(m), dl(m), rhs(m);
  std::vector<int> piv(m);
  for (int iter = 0; iter < 3; ++iter) {
    // LU with partial pivoting of the tridiagonal (T - shift)
    for (int i = 0; i < m; ++i) {
      d[i] = a[i] - shift;
      du[i] = i < m - 1 ? b[i] : 0.0;
      dl[i] = i < m - 1 ? b[i] : 0.0;
      du2[i] = 0.0;
    }
    for (int i = 0; i < m - 1; ++i) {
      if (std::fabs(d[i]) >= std::fabs(dl[i])) {
        piv[i] = 0;
        if (d[i] == 0.0) d[i] = 1e-300;
        double f = dl[i] / d[i];
        dl[i] = f;
        d[i + 1] -= f * du[i];
      } else {
        piv[i] = 1;
        double f = d[i] / dl[i];
        d[i] = dl[i];
        dl[i] = f;
        double t = du[i];
        du[i] = d[i + 1];
        d[i + 1] = t - f * d[i + 1];
        if (i < m - 2) {
          du2[i] = du[i + 1];
          du[i + 1] = -f * du[i + 1];
        }
      }
    }
    if (d[m - 1] == 0.0) d[m - 1] = 1e-300;
    rhs = s;
    for (int i = 0; i < m - 1; ++i) {
      if (piv[i] == 0) rhs[i + 1] -= dl[i] * rhs[i];
      else { double t = rhs[i]; rhs[i] = rhs[i + 1]; rhs[i + 1] = t - dl[i] * rhs[i + 1]; }
    }
    rhs[m - 1] /= d[m - 1];
    if (m > 1) rhs[m - 2] = (rhs[m - 2] - du[m - 2] * rhs[m - 1]) / d[m - 2];
    for (int i = m - 3; i >= 0; --i) rhs[i] = (rhs[i] - du[i] * rhs[i + 1] - du2[i] * rhs[i + 2]) / d[i];
    double nrm = 0.0;
    for (int i = 0; i < m; ++i) nrm += rhs[i] * rhs[i];
    nrm = std::sqrt(nrm);
    for (int i = 0; i < m; ++i) s[i] = rhs[i] / nrm;
  }
  if (s[0] < 0) for (auto& v : s) v = -v;
}

// ---------------------------------------------------------------- launchers

template <typename T>
void launch_lz_a(ed_ctx* c, T* w, const T* v, const T* vprev, int use_beta, long long n, cudaStream_t st) {
  int g = grid_for(c, n);
  k_lz_a<T><<<g, kRedThreads, 0, st>>>(w, v, vprev, slot(c, 1), use_beta, n, c->d_partials);
  k_finalize<<<1, kRedThreads, 0, st>>>(c->d_partials, g, slot(c, 0), 0);
}
template <typename T>
void launch_lz_b(ed_ctx* c, T* w, const T* v, long long n, cudaStream_t st) {
  int g = grid_for(c, n);
  k_lz_b<T><<<g, kRedThreads, 0, st>>>(w, v, slot(c, 0), n, c->d_partials);
  k_finalize<<<1, kRedThreads, 0, st>>>(c->d_partials, g, slot(c, 1), 1);
}
template <typename T>
void launch_lz_c(ed_ctx* c, const T* w, T* out, long long n, cudaStream_t st) {
  k_lz_c<T><<<grid_for(c, n), kRedThreads, 0, st>>>(w, out, slot(c, 1), n);
}
void launch_lz_b_emax(ed_ctx* c, double* w, const double* v, long long n, int* ew, cudaStream_t st) {
  int g = grid_for(c, n);
  cudaMemsetAsync(ew, 0, sizeof(int), st);
  k_lz_b_emax<<<g, kRedThreads, 0, st>>>(w, v, slot(c, 0), n, c->d_partials, ew);
  k_finalize<<<1, kRedThreads, 0, st>>>(c->d_partials, g, slot(c, 1), 1);
}
void launch_lz_c_fixed(ed_ctx* c, const double* w, double* out, long long* X, const int* ew, int* ex, long long n,
                       cudaStream_t st) {
  k_lz_c_fixed<<<grid_for(c, n), kRedThreads, 0, st>>>(w, out, X, slot(c, 1), ew, ex, c->t3.P, n);
}
template <typename T>
void launch_lz_rerun(ed_ctx* c, const T* w, const T* v, const T* vprev, double alpha, double beta, double inv_next,
                     T* out, long long n, cudaStream_t st) {
  k_lz_rerun<T><<<grid_for(c, n), kRedThreads, 0, st>>>(w, v, vprev, (T)alpha, (T)beta, (T)inv_next, out, n);
}
template <typename TI, typename TO>
void launch_scale_cvt(ed_ctx* c, const TI* x, TO* y, double s, long long n, cudaStream_t st) {
  k_scale_cvt<TI, TO><<<grid_for(c, n), kRedThreads, 0, st>>>(x, y, s, n);
}
template <typename TB, typename TO>
void launch_axpy_basis(ed_ctx* c, const TB* v, TO* x, double s, long long n, cudaStream_t st) {
  k_axpy_basis<TB, TO><<<grid_for(c, n), kRedThreads, 0, st>>>(v, x, s, n);
}
ed_status launch_combine_f32(ed_ctx* c, const float* V, long long n, const double* s, int m, double* x,
                             cudaStream_t st) {
  if (m < 1 || m > kMaxBasis) {
    set_error("basis combination of %d vectors outside 1..%d", m, kMaxBasis);
    return ED_EINVAL;
  }
  std::vector<float2> h(m);
  for (int j = 0; j < m; ++j) {
    h[j].x = (float)s[j];
    h[j].y = (float)(s[j] - (double)h[j].x);
  }
  // the pairs travel through the reorthogonalisation coefficient buffer
  // (kMaxBasis 8-byte slots)
  float2* d = reinterpret_cast<float2*>(hcoef(c));
  ED_CUDA_TRY(cudaMemcpyAsync(d, h.data(), (size_t)m * sizeof(float2), cudaMemcpyHostToDevice, st));
  k_combine_f32<<<grid_for(c, n), kRedThreads, (size_t)m * sizeof(float2), st>>>(V, n, m, d, x);
  ED_CUDA_TRY(cudaGetLastError());
  return ED_OK;
}
void launch_hist_push(ed_ctx* c, double* hist, int* counter, cudaStream_t st) {
  k_hist_push<<<1, 1, 0, st>>>(slot(c, 0), hist, counter);
}
template <typename TI, typename TO>
void launch_cvt(ed_ctx* c, const TI* x, TO* y, long long n, cudaStream_t st) {
  k_cvt<TI, TO><<<grid_for(c, n), kRedThreads, 0, st>>>(x, y, n);
}
template <typename T>
void launch_axpy_dev(ed_ctx* c, const T* x, T* y, const double* s, double sign, long long n, cudaStream_t st) {
  k_axpy_dev<T, T><<<grid_for(c, n), kRedThreads, 0, st>>>(x, y, s, sign, n);
}
template <typename T>
void launch_reorth(ed_ctx* c, const T* V, long long ldv, int m, T* w, long long n, double* h, cudaStream_t st) {
  if (m <= 0) return;
  int chunks = std::max(1, std::min(kMaxPartials / m, (int)((n + kRedThreads - 1) / kRedThreads)));
  chunks = std::min(chunks, 256);
  dim3 g1(chunks, m);
  k_basis_dots<T><<<g1, kRedThreads, 0, st>>>(V, ldv, w, n, c->d_partials, chunks);
  k_finalize_many<<<(m + 127) / 128, 128, 0, st>>>(c->d_partials, chunks, m, h);
  k_basis_update<T><<<grid_for(c, n), kRedThreads, m * sizeof(double), st>>>(V, ldv, m, h, w, n);
}
template void launch_reorth<double>(ed_ctx*, const double*, long long, int, double*, long long, double*, cudaStream_t);
template void launch_reorth<float>(ed_ctx*, const float*, long long, int, float*, long long, double*, cudaStream_t);

void launch_green_cf(const double* omega, int n_omega, double eta, double e0, const double* ap, const double* bp, int mp,
                     double wp, const double* ah, const double* bh, int mh, double wh, double* G, cudaStream_t st) {
  int th = 128;
  k_green_cf<<<(n_omega + th - 1) / th, th, 0, st>>>(omega, n_omega, eta, e0, ap, bp, mp, wp, ah, bh, mh, wh, G);
}
void launch_fermion_remap(ed_ctx* c, const double* psi, long long dA_src, long long dB_src, double* phi,
                          long long dA_dst, long long dB_dst, const int* map, const signed char* sgn, int side,
                          cudaStream_t st) {
  k_fermion_remap<<<grid_for(c, dA_dst * dB_dst), kRedThreads, 0, st>>>(psi, dA_src, dB_src, phi, dA_dst, dB_dst, map,
                                                                        sgn, side);
}

#define ED_INST(T)                                                                                        \
  template void launch_lz_a<T>(ed_ctx*, T*, const T*, const T*, int, long long, cudaStream_t);          \
  template void launch_lz_b<T>(ed_ctx*, T*, const T*, long long, cudaStream_t);                         \
  template void launch_lz_c<T>(ed_ctx*, const T*, T*, long long, cudaStream_t);                        \
  template void launch_lz_rerun<T>(ed_ctx*, const T*, const T*, const T*, double, double, double, T*,   \
                                   long long, cudaStream_t);                                            \
  template void launch_axpy_dev<T>(ed_ctx*, const T*, T*, const double*, double, long long, cudaStream_t);
ED_INST(double)
ED_INST(float)
template void launch_scale_cvt<double, double>(ed_ctx*, const double*, double*, double, long long, cudaStream_t);
template void launch_scale_cvt<double, float>(ed_ctx*, const double*, float*, double, long long, cudaStream_t);
template void launch_scale_cvt<float, double>(ed_ctx*, const float*, double*, double, long long, cudaStream_t);
template void launch_scale_cvt<float, float>(ed_ctx*, const float*, float*, double, long long, cudaStream_t);
template void launch_axpy_basis<double, double>(ed_ctx*, const double*, double*, double, long long, cudaStream_t);
template void launch_axpy_basis<float, double>(ed_ctx*, const float*, double*, double, long long, cudaStream_t);
template void launch_axpy_basis<__nv_bfloat16, double>(ed_ctx*, const __nv_bfloat16*, double*, double, long long,
                                                       cudaStream_t);
template void launch_cvt<float, __nv_bfloat16>(ed_ctx*, const float*, __nv_bfloat16*, long long, cudaStream_t);
template void launch_cvt<double, float>(ed_ctx*, const double*, float*, long long, cudaStream_t);
template void launch_cvt<float, double>(ed_ctx*, const float*, double*, long long, cudaStream_t);

}  // namespace edk
