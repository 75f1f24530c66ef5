// Matrix-free H|psi> in the entanglement-cut representation (paper Eq. (2)):
//   (H psi)_s[a,b] = V(a,b) psi_s[a,b]                       diagonal
//                  + sum_b' H_B[b,b'] psi_s[a,b']              1 (x) H_R: row-local
//                  + sum_a' H_A[a,a'] psi_s[a',b]              H_L (x) 1: row mixing
//                  + sum_k c_k psi_s'[mapA_k(a), mapB_k(b)]    L_m (x) R_m cross terms
// The paper moves data with its T* transposition so that H_L acts on local
// data; on one GPU the row psi_s[a,:] is staged in shared memory (the
// on-chip transpose) and neighbour rows are read through L2.
#include <cstdio>

#include "ed_internal.h"

namespace edk {

struct ApplyParams {
  DevTables t;
  const DevBlock* blocks;
  const DevCross* cross;
  const long long* row_start;
  DevDiagParams dp;
  int nblk;
  int ncross;
  long long n_rows;
};

template <typename T>
struct Vals;
template <>
struct Vals<double> {
  __device__ static const double* A(const DevTables& t) { return t.A_val64; }
  __device__ static const double* B(const DevTables& t) { return t.B_val64; }
};
template <>
struct Vals<float> {
  __device__ static const float* A(const DevTables& t) { return t.A_val32; }
  __device__ static const float* B(const DevTables& t) { return t.B_val32; }
};

__device__ __forceinline__ int find_block(const long long* row_start, int nblk, long long row) {
  int lo = 0, hi = nblk - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (row_start[mid] <= row) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// V_AB(a,b) from the packed words (weighted popcounts)
template <typename T>
__device__ __forceinline__ T vab(const DevDiagParams& dp, unsigned long long pa, unsigned long long pb);
template <>
__device__ __forceinline__ double vab<double>(const DevDiagParams& dp, unsigned long long pa, unsigned long long pb) {
  unsigned long long z = dp.vab_and ? (pa & pb) : (pa ^ pb);
  double v = dp.c0;
  for (int c = 0; c < dp.ncls; ++c) v += dp.w[c] * (double)__popcll(z & dp.mask[c]);
  return v;
}
template <>
__device__ __forceinline__ float vab<float>(const DevDiagParams& dp, unsigned long long pa, unsigned long long pb) {
  unsigned long long z = dp.vab_and ? (pa & pb) : (pa ^ pb);
  float v = dp.c0_32;
  for (int c = 0; c < dp.ncls; ++c) v += dp.w32[c] * (float)__popcll(z & dp.mask[c]);
  return v;
}

template <typename T>
__device__ __forceinline__ T side_diag(const DevTables& t, long long gA, long long gB);
template <>
__device__ __forceinline__ double side_diag<double>(const DevTables& t, long long gA, long long gB) {
  return t.A_diag[gA] + t.B_diag[gB];
}
template <>
__device__ __forceinline__ float side_diag<float>(const DevTables& t, long long gA, long long gB) {
  return t.A_diag32[gA] + t.B_diag32[gB];
}

// One CTA per (block, row) work item, grid-strided.  kStage: the row of x
// is copied into shared memory and the H_B gathers read it there.
template <typename T, bool kStage>
__global__ void __launch_bounds__(256) k_apply_rows(ApplyParams p, const T* __restrict__ x, T* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);
  __shared__ const T* src_row[kMaxCross];
  __shared__ T src_coef[kMaxCross];
  __shared__ int src_ib[kMaxCross];
  const DevTables& t = p.t;
  const T* Aval = Vals<T>::A(t);
  const T* Bval = Vals<T>::B(t);
  for (long long row = blockIdx.x; row < p.n_rows; row += gridDim.x) {
    const int bi = find_block(p.row_start, p.nblk, row);
    const DevBlock bl = p.blocks[bi];
    const long long a = row - bl.row0;
    const long long gA = bl.gA0 + a;
    const long long dB = bl.dB;
    const T* xrow = x + bl.off + a * dB;
    T* yrow = y + bl.off + a * dB;
    const unsigned long long pa = t.A_pack[gA];
    if (kStage) {
      for (long long b = threadIdx.x; b < dB; b += blockDim.x) xs[b] = xrow[b];
    }
    if (threadIdx.x < p.ncross) {
      const int k = threadIdx.x;
      const DevCross cr = p.cross[k];
      const int abit = (int)((pa >> k) & 1ull);
      const int sb = abit ? bl.nbr_lo : bl.nbr_hi;
      const T* sp = nullptr;
      if (sb >= 0) {
        const DevBlock so = p.blocks[sb];
        const int r = t.mapA[(long long)cr.ia * t.A_total + gA];
        if (r >= 0) sp = x + so.off + (long long)r * so.dB;
      }
      src_row[k] = sp;
      src_coef[k] = (T)cr.coef;
      src_ib[k] = cr.ib;
    }
    __syncthreads();
    const int a0 = t.A_rowptr[gA], a1 = t.A_rowptr[gA + 1];
    const T* xblk = x + bl.off;
    for (long long b = threadIdx.x; b < dB; b += blockDim.x) {
      const long long gB = bl.gB0 + b;
      const T xv = kStage ? xs[b] : xrow[b];
      const unsigned long long pb = t.B_pack[gB];
      T acc = (side_diag<T>(t, gA, gB) + vab<T>(p.dp, pa, pb)) * xv;
      const int b0 = t.B_rowptr[gB], b1 = t.B_rowptr[gB + 1];
      for (int e = b0; e < b1; ++e) {
        const int cb = t.B_col[e];
        acc += Bval[e] * (kStage ? xs[cb] : xrow[cb]);
      }
      for (int e = a0; e < a1; ++e) acc += Aval[e] * xblk[(long long)t.A_col[e] * dB + b];
      if (p.ncross) {
        unsigned long long diff = pa ^ pb;
        while (diff) {
          const int k = __ffsll((long long)diff) - 1;
          diff &= diff - 1;
          const T* sp = src_row[k];
          if (sp) acc += src_coef[k] * sp[t.mapB[(long long)src_ib[k] * t.B_total + gB]];
        }
      }
      yrow[b] = acc;
    }
    __syncthreads();
  }
}

// Key-indexed SplitMix64 start values (Steele, Lea, Flood 2014): the first
// output of a SplitMix64 stream with state seed ^ key, top 53 bits -> [-1, 1).
__device__ __forceinline__ double splitmix_value(unsigned long long seed, unsigned long long key) {
  unsigned long long z = (seed ^ key) + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
}

template <typename T>
__global__ void k_random_vector(ApplyParams p, unsigned long long seed, T* __restrict__ x) {
  const DevTables& t = p.t;
  for (long long row = blockIdx.x; row < p.n_rows; row += gridDim.x) {
    const int bi = find_block(p.row_start, p.nblk, row);
    const DevBlock bl = p.blocks[bi];
    const long long a = row - bl.row0;
    const unsigned long long ka = t.A_key[bl.gA0 + a];
    T* xrow = x + bl.off + a * bl.dB;
    for (long long b = threadIdx.x; b < bl.dB; b += blockDim.x)
      xrow[b] = (T)splitmix_value(seed, ka | t.B_key[bl.gB0 + b]);
  }
}

static ApplyParams make_params(const ed_ctx* c) {
  ApplyParams p;
  p.t = c->tab;
  p.blocks = c->d_blocks;
  p.cross = c->d_cross;
  p.row_start = c->d_row_start;
  p.dp = c->diag;
  p.nblk = (int)c->blocks.size();
  p.ncross = c->kind == ED_SPIN ? (int)c->cross.size() : 0;
  p.n_rows = c->n_rows;
  return p;
}

static int64_t max_dB(const ed_ctx* c) {
  int64_t m = 1;
  for (const auto& b : c->blocks) m = std::max<int64_t>(m, b.dB);
  return m;
}

static int sm_count(int dev) {
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    n = 148;
  }
  return n;
}

template <typename T>
static ed_status launch_apply_rows(const ed_ctx* c, const T* x, T* y, cudaStream_t st) {
  ApplyParams p = make_params(c);
  if (p.n_rows == 0) return ED_OK;
  const int64_t mdb = max_dB(c);
  const size_t smem = (size_t)mdb * sizeof(T);
  int threads = (int)std::min<int64_t>(256, ((mdb + 31) / 32) * 32);
  threads = std::max(threads, 64);
  const long long grid = std::min<long long>(p.n_rows, (long long)sm_count(c->device) * 16);
  if (smem <= 200 * 1024) {
    auto kern = k_apply_rows<T, true>;
    ED_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)grid, threads, smem, st>>>(p, x, y);
  } else {
    k_apply_rows<T, false><<<(unsigned)grid, threads, 0, st>>>(p, x, y);
  }
  ED_CUDA_TRY(cudaGetLastError());
  return ED_OK;
}

ed_status apply_H_impl(const ed_ctx* c, const void* x, void* y, ed_dtype dt, cudaStream_t st) {
  if (dt == ED_F64) return launch_apply_rows<double>(c, (const double*)x, (double*)y, st);
  return launch_apply_rows<float>(c, (const float*)x, (float*)y, st);
}

ed_status random_vector_impl(const ed_ctx* c, uint64_t seed, void* x, ed_dtype dt, cudaStream_t st) {
  ApplyParams p = make_params(c);
  if (p.n_rows == 0) return ED_OK;
  const long long grid = std::min<long long>(p.n_rows, (long long)sm_count(c->device) * 16);
  if (dt == ED_F64)
    k_random_vector<double><<<(unsigned)grid, 256, 0, st>>>(p, seed, (double*)x);
  else
    k_random_vector<float><<<(unsigned)grid, 256, 0, st>>>(p, seed, (float*)x);
  ED_CUDA_TRY(cudaGetLastError());
  return ED_OK;
}

}  // namespace edk

using namespace edk;

static ed_status check_ready(const ed_ctx* c) {
  if (!c) { set_error("ctx is NULL"); return ED_EINVAL; }
  if (!c->ops_built) { set_error("ed_build_local_ops has not been called"); return ED_EINVAL; }
  return ED_OK;
}

extern "C" ed_status ed_apply_H(ed_ctx* c, const void* x, void* y, ed_dtype dt, void* stream) {
  ED_TRY(check_ready(c));
  if (dt != ED_F64 && dt != ED_F32) { set_error("bad dtype %d", (int)dt); return ED_EINVAL; }
  if (c->D > 0 && (!x || !y)) { set_error("x or y is NULL"); return ED_EINVAL; }
  const size_t es = dt == ED_F64 ? 8 : 4;
  const char* xb = (const char*)x;
  const char* yb = (const char*)y;
  if (c->D > 0 && xb < yb + c->D * es && yb < xb + c->D * es) { set_error("x and y overlap"); return ED_EINVAL; }
  ED_CUDA_TRY(cudaSetDevice(c->device));
  return apply_H_impl(c, x, y, dt, (cudaStream_t)stream);
}

extern "C" ed_status ed_random_vector(ed_ctx* c, uint64_t seed, void* x, ed_dtype dt, void* stream) {
  ED_TRY(check_ready(c));
  if (dt != ED_F64 && dt != ED_F32) { set_error("bad dtype %d", (int)dt); return ED_EINVAL; }
  if (c->D > 0 && !x) { set_error("x is NULL"); return ED_EINVAL; }
  ED_CUDA_TRY(cudaSetDevice(c->device));
  return random_vector_impl(c, seed, x, dt, (cudaStream_t)stream);
}
