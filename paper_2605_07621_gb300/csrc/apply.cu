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
#include "splitmix.cuh"

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


// ---------------------------------------------------------------- TMA / mbarrier helpers

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// 1-D bulk copy global -> shared (plain, no multicast), completion on `bar`
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false after kWaitLimit polls (each poll already suspends for a while)
constexpr long long kWaitLimit = 1ll << 22;
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  for (long long i = 0; i < kWaitLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Row pass: per (block, row a), the row psi_s[a,:] is brought into shared
// memory by a bulk TMA copy (double-buffered: the next row streams in while
// this one is computed); then for every column b
//   y[a,b] = V(a,b) x[a,b] + sum_b' H_B[b,b'] x[a,b'] + cross-cut gathers.
// The H_A (row-mixing) term is added afterwards by k_hA_panel.
template <typename T>
__global__ void __launch_bounds__(256, 1) k_rowpass(ApplyParams p, const T* __restrict__ x, T* __restrict__ y,
                                                    long long stage_elems, int* err) {
  extern __shared__ __align__(16) unsigned char smem_rp[];
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_rp);
  T* bufs = reinterpret_cast<T*>(smem_rp + 128);
  __shared__ const T* src_row[kMaxCross];
  __shared__ T src_coef[kMaxCross];
  __shared__ int src_ib[kMaxCross];
  constexpr int V = 16 / (int)sizeof(T);
  const DevTables& t = p.t;
  const T* Bval = Vals<T>::B(t);
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // thread 0: start the bulk copy of row r into stage st
  auto issue = [&](long long r, int st) {
    const int bi = find_block(p.row_start, p.nblk, r);
    const DevBlock bl = p.blocks[bi];
    const long long g0 = bl.off + (r - bl.row0) * bl.dB;
    const long long gend = g0 + bl.dB;
    const long long gal = (g0 + V - 1) / V * V;
    const long long galend = gend / V * V;
    T* buf = bufs + (long long)st * stage_elems;
    if (galend > gal) {
      const unsigned bytes = (unsigned)((galend - gal) * (long long)sizeof(T));
      mbar_arrive_expect_tx(&bar[st], bytes);
      tma_load_1d(buf + (g0 % V) + (gal - g0), x + gal, bytes, &bar[st]);
    } else {
      mbar_arrive(&bar[st]);
    }
  };
  unsigned phase0 = 0, phase1 = 0;
  long long row = blockIdx.x;
  if (threadIdx.x == 0 && row < p.n_rows) issue(row, 0);
  for (int it = 0; row < p.n_rows; row += gridDim.x, ++it) {
    const int st = it & 1;
    T* buf = bufs + (long long)st * stage_elems;
    const long long nrow = row + gridDim.x;
    if (threadIdx.x == 0 && nrow < p.n_rows) {
      fence_proxy_async();
      issue(nrow, st ^ 1);
    }
    const int bi = find_block(p.row_start, p.nblk, row);
    const DevBlock bl = p.blocks[bi];
    const long long a = row - bl.row0;
    const long long gA = bl.gA0 + a;
    const long long dB = bl.dB;
    const long long g0 = bl.off + a * dB;
    const long long gend = g0 + dB;
    const long long gal = (g0 + V - 1) / V * V;
    const long long galend = gend / V * V;
    const int pad = (int)(g0 % V);
    // ragged ends that the 16-byte-aligned bulk copy leaves out
    if (galend > gal) {
      for (long long g = g0 + threadIdx.x; g < gal; g += blockDim.x) buf[pad + (g - g0)] = x[g];
      for (long long g = galend + threadIdx.x; g < gend; g += blockDim.x) buf[pad + (g - g0)] = x[g];
    } else {
      for (long long g = g0 + threadIdx.x; g < gend; g += blockDim.x) buf[pad + (g - g0)] = x[g];
    }
    const unsigned par = st ? phase1 : phase0;
    const bool ok = mbar_wait_bounded(&bar[st], par);
    if (__syncthreads_or(!ok)) {
      // a copy never completed: report, give copies in flight a last bounded
      // chance to land in this CTA's shared memory, and leave uniformly
      if (threadIdx.x == 0) atomicExch(err, 1);
      mbar_wait_bounded(&bar[st], par);
      if (nrow < p.n_rows) mbar_wait_bounded(&bar[st ^ 1], st ? phase0 : phase1);
      return;
    }
    if (st) phase1 ^= 1; else phase0 ^= 1;
    const unsigned long long pa = t.A_pack[gA];
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
    const T* xs = buf + pad;
    for (long long b = threadIdx.x; b < dB; b += blockDim.x) {
      const long long gB = bl.gB0 + b;
      const unsigned long long pb = t.B_pack[gB];
      T acc = (side_diag<T>(t, gA, gB) + vab<T>(p.dp, pa, pb)) * xs[b];
      const int b0 = t.B_rowptr[gB], b1 = t.B_rowptr[gB + 1];
      for (int e = b0; e < b1; ++e) acc += Bval[e] * xs[t.B_col[e]];
      if (p.ncross) {
        unsigned long long diff = pa ^ pb;
        while (diff) {
          const int k = __ffsll((long long)diff) - 1;
          diff &= diff - 1;
          const T* sp = src_row[k];
          if (sp) acc += src_coef[k] * __ldg(sp + t.mapB[(long long)src_ib[k] * t.B_total + gB]);
        }
      }
      y[g0 + b] = acc;
    }
    __syncthreads();
  }
}

// H_A term, y[a, b] += sum_a' H_A[a,a'] x[a', b], over work items (block,
// column panel of kPanelCols columns, 8 rows) ordered panel by panel so that
// the panel x[:, b0:b0+kPanelCols] of a block stays resident in L2 while all
// its rows are processed.  One warp per output row, lanes over columns.
constexpr int kPanelColsPerLane = 8;  // panel = 256 columns (host builds the items to match)

template <typename T>
__global__ void __launch_bounds__(256) k_hA_panel(ApplyParams p, const int4* __restrict__ items, long long n_items,
                                                  const T* __restrict__ x, T* __restrict__ y) {
  const DevTables& t = p.t;
  const T* Aval = Vals<T>::A(t);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (long long w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int4 it = items[w];  // block, first column, first row, rows
    if (warp >= it.w) continue;
    const DevBlock bl = p.blocks[it.x];
    const long long a = it.z + warp;
    const long long gA = bl.gA0 + a;
    const long long dB = bl.dB;
    const T* xb = x + bl.off;
    T* yrow = y + bl.off + a * dB;
    T acc[kPanelColsPerLane];
#pragma unroll
    for (int c = 0; c < kPanelColsPerLane; ++c) {
      const long long b = it.y + lane + 32 * c;
      acc[c] = b < dB ? yrow[b] : (T)0;
    }
    const int e0 = t.A_rowptr[gA], e1 = t.A_rowptr[gA + 1];
    for (int e = e0; e < e1; ++e) {
      const T v = Aval[e];
      const T* xr = xb + (long long)t.A_col[e] * dB;
#pragma unroll
      for (int c = 0; c < kPanelColsPerLane; ++c) {
        const long long b = it.y + lane + 32 * c;
        if (b < dB) acc[c] += v * __ldg(xr + b);
      }
    }
#pragma unroll
    for (int c = 0; c < kPanelColsPerLane; ++c) {
      const long long b = it.y + lane + 32 * c;
      if (b < dB) yrow[b] = acc[c];
    }
  }
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
  const int sms = sm_count(c->device);
  // two row buffers, each padded so that any row start can be 16-byte aligned
  const long long stage_elems = ((mdb + 16 / (long long)sizeof(T) + 15) / 16) * 16;
  const size_t smem2 = 128 + 2 * (size_t)stage_elems * sizeof(T);
  const bool aligned = ((uintptr_t)x % 16) == 0;
  if (aligned && smem2 <= 220 * 1024) {
    auto kern = k_rowpass<T>;
    ED_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
    const long long grid = std::min<long long>(p.n_rows, (long long)sms);
    kern<<<(unsigned)grid, 256, smem2, st>>>(p, x, y, stage_elems, c->d_err);
    ED_CUDA_TRY(cudaGetLastError());
    if (c->n_panel_items > 0) {
      const long long g2 = std::min<long long>(c->n_panel_items, (long long)sms * 8);
      k_hA_panel<T><<<(unsigned)g2, 256, 0, st>>>(p, c->d_panel_items, c->n_panel_items, x, y);
      ED_CUDA_TRY(cudaGetLastError());
    }
    return ED_OK;
  }
  // rows too wide for two shared-memory buffers (or an unaligned vector):
  // single fused pass reading x through the cache hierarchy
  const size_t smem = (size_t)mdb * sizeof(T);
  int threads = (int)std::min<int64_t>(256, ((mdb + 31) / 32) * 32);
  threads = std::max(threads, 64);
  const long long grid = std::min<long long>(p.n_rows, (long long)sms * 16);
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

bool v3_usable(const ed_ctx* c, ed_dtype dt, const void* x);
ed_status apply_v3(ed_ctx* c, const void* x, void* y, ed_dtype dt, cudaStream_t st);

ed_status apply_H_impl(ed_ctx* c, const void* x, void* y, ed_dtype dt, cudaStream_t st) {
  if (v3_usable(c, dt, x)) return apply_v3(c, x, y, dt, st);
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
  ED_DEVICE_SCOPE(c->device);
  return apply_H_impl(c, x, y, dt, (cudaStream_t)stream);
}

extern "C" ed_status ed_random_vector(ed_ctx* c, uint64_t seed, void* x, ed_dtype dt, void* stream) {
  ED_TRY(check_ready(c));
  if (dt != ED_F64 && dt != ED_F32) { set_error("bad dtype %d", (int)dt); return ED_EINVAL; }
  if (c->D > 0 && !x) { set_error("x is NULL"); return ED_EINVAL; }
  ED_DEVICE_SCOPE(c->device);
  return random_vector_impl(c, seed, x, dt, (cudaStream_t)stream);
}
