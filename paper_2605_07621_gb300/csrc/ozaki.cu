// FP64-accurate GEMM on the BF16 tensor cores (Ozaki-style digit
// splitting, see ozaki.h): digit planes formed on the host or by the slicing
// kernels here, tiles staged by TMA with 128-byte swizzle, products issued
// by one thread with tcgen05.mma into FP32 accumulators in TMEM (one per
// digit order), drained by four warps and combined in FP64.
#include <atomic>

#include "ozaki.h"

#include <cmath>
#include <cstring>

#include "apply3.cuh"  // I128, from_fixed128
#include "tc.cuh"

namespace edk {

// ---------------------------------------------------------------- digits

// exponent E with maxabs < 2^E (0 for an all-zero row)
int oz_row_exponent(double maxabs) {
  if (!(maxabs > 0.0)) return 0;
  int e;
  std::frexp(maxabs, &e);  // maxabs = f 2^e, f in [0.5, 1)
  return e;
}

// U = round(v 2^(47 - E)) (|U| <= 2^47), then 8 balanced base-64 digits,
// most significant first: U = sum_p d_p 64^(7 - p), |d_p| <= 32
void oz_digits_host(double v, int E, int* d) {
  long long U = std::llrint(std::ldexp(v, kOzFrac - E));
  for (int p = kOzDigits - 1; p > 0; --p) {
    const long long r = ((U + 32) & 63) - 32;
    d[p] = (int)r;
    U = (U - r) >> kOzBits;
  }
  d[0] = (int)U;
}

__host__ __device__ inline uint16_t bf16_of_small_int(int v) {
  // |v| <= 32: the BF16 bit pattern of (float)v (8 significant bits suffice)
  const float f = (float)v;
  uint32_t u;
#ifdef __CUDA_ARCH__
  u = __float_as_uint(f);
#else
  std::memcpy(&u, &f, 4);
#endif
  return (uint16_t)(u >> 16);
}

__device__ inline double pow2(int k) {  // 2^k for -1022 <= k <= 1023
  return __longlong_as_double((long long)(k + 1023) << 52);
}

__device__ inline int exp_of(double maxabs) {  // maxabs < 2^E
  if (!(maxabs > 0.0)) return 0;
  const int b = (int)((__double_as_longlong(maxabs) >> 52) & 0x7ff);
  if (b == 0) return -1021;  // subnormal: below 2^-1022
  return b - 1022;
}

__device__ inline void digits_dev(double v, int E, int* d) {
  long long U = __double2ll_rn(v * pow2(kOzFrac - E));
#pragma unroll
  for (int p = kOzDigits - 1; p > 0; --p) {
    const long long r = ((U + 32) & 63) - 32;
    d[p] = (int)r;
    U = (U - r) >> kOzBits;
  }
  d[0] = (int)U;
}

// ---------------------------------------------------------------- context

OzContext::~OzContext() {
  for (void* p : allocs) cudaFree(p);
}

ed_status oz_alloc(OzContext* o, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes < 16 ? 16 : bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc(%zu) for tensor-core operands failed: %s", bytes, cudaGetErrorString(e));
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? ED_ENOMEM : ED_ECUDA;
  }
  o->allocs.push_back(*p);
  return ED_OK;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      cudaGetLastError();
  }
  return fn;
}

ed_status tmap_8b_2d(CUtensorMap* m, const void* base, long long cols, long long rows, long long ld, int box_cols,
                     int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return ED_ECUDA;
  }
  cudaFree(nullptr);  // a current context for the driver call (see tmap_bf16_planes)
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 8};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d) for a %lld x %lld matrix", (int)r, rows, cols);
    return ED_ECUDA;
  }
  return ED_OK;
}

ed_status oz_status(OzContext* o, cudaStream_t st) {
  if (!o->d_err) return ED_OK;
  int h = 0;
  ED_CUDA_TRY(cudaMemcpyAsync(&h, o->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  ED_CUDA_TRY(cudaStreamSynchronize(st));
  if (h != 0) {
    ED_CUDA_TRY(cudaMemsetAsync(o->d_err, 0, sizeof(int), st));
    set_error("a tensor-core kernel's wait for its operands ran out (code %d)", h);
    return ED_ECUDA;
  }
  return ED_OK;
}

ed_status tmap_bf16_planes(CUtensorMap* m, const void* base, int K, int R, int planes, long long Kpad, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return ED_ECUDA;
  }
  // a driver call: the calling thread needs a current context, which the
  // runtime binds on its first call that needs one (cudaFree(0) is such a call)
  cudaFree(nullptr);
  const cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)R, (cuuint64_t)planes};
  const cuuint64_t strides[2] = {(cuuint64_t)Kpad * 2, (cuuint64_t)Kpad * 2 * (cuuint64_t)R};
  const cuuint32_t box[3] = {(cuuint32_t)kOzBK, (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d) for a %d x %d operand", (int)r, R, K);
    return ED_ECUDA;
  }
  return ED_OK;
}

// 3-D map over the digit planes: (K, R, 8) BF16, box (64, box_rows, 1),
// 128-byte swizzle, out-of-range elements read as zero
static ed_status make_map(OzContext* o, OzOperand* op, int box_rows) {
  CUtensorMap m;
  ED_TRY(tmap_bf16_planes(&m, op->slices, op->K, op->R, kOzDigits, op->Kpad, box_rows));
  op->map = (int)o->maps.size();
  o->maps.push_back(m);
  return ED_OK;
}

static ed_status alloc_operand(OzContext* o, int R, int K, OzOperand* op) {
  op->R = R;
  op->K = K;
  op->Kpad = (K + 7) / 8 * 8;  // 16-byte row stride
  ED_TRY(oz_alloc(o, (void**)&op->slices, (size_t)kOzDigits * R * op->Kpad * 2));
  ED_TRY(oz_alloc(o, (void**)&op->exps, (size_t)R * sizeof(int)));
  return ED_OK;
}

ed_status oz_operand_host(OzContext* o, const double* h, int R, int K, bool a_role, OzOperand* out) {
  ED_TRY(alloc_operand(o, R, K, out));
  const int Kp = out->Kpad;
  std::vector<uint16_t> s((size_t)kOzDigits * R * Kp, 0);
  std::vector<int> ex(R);
  int d[kOzDigits];
  for (int i = 0; i < R; ++i) {
    double mx = 0.0;
    for (int k = 0; k < K; ++k) mx = std::max(mx, std::fabs(h[(size_t)i * K + k]));
    const int E = oz_row_exponent(mx);
    ex[i] = E;
    for (int k = 0; k < K; ++k) {
      oz_digits_host(h[(size_t)i * K + k], E, d);
      for (int p = 0; p < kOzDigits; ++p) s[((size_t)p * R + i) * Kp + k] = bf16_of_small_int(d[p]);
    }
  }
  ED_CUDA_TRY(cudaMemcpy(out->slices, s.data(), s.size() * 2, cudaMemcpyHostToDevice));
  ED_CUDA_TRY(cudaMemcpy(out->exps, ex.data(), ex.size() * sizeof(int), cudaMemcpyHostToDevice));
  return make_map(o, out, a_role ? kOzBM : kOzBN);
}

ed_status oz_operand_device(OzContext* o, int R, int K, bool a_role, OzOperand* out) {
  ED_TRY(alloc_operand(o, R, K, out));
  ED_CUDA_TRY(cudaMemset(out->slices, 0, (size_t)kOzDigits * R * out->Kpad * 2));
  return make_map(o, out, a_role ? kOzBM : kOzBN);
}

ed_status oz_finish(OzContext* o) {
  if (o->maps.empty()) return ED_OK;
  ED_TRY(oz_alloc(o, (void**)&o->d_maps, o->maps.size() * sizeof(CUtensorMap)));
  ED_CUDA_TRY(cudaMemcpy(o->d_maps, o->maps.data(), o->maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
  if (!o->d_err) {
    ED_TRY(oz_alloc(o, (void**)&o->d_err, 16));
    ED_CUDA_TRY(cudaMemset(o->d_err, 0, 16));
  }
  return ED_OK;
}

// tile rows of a triangular problem hold min(tiles_n, 2 (tm + 1)) tiles (BM = 2 BN)
long long oz_tiles(int M, int N, int tri) {
  const long long tm = (M + kOzBM - 1) / kOzBM, tn = (N + kOzBN - 1) / kOzBN;
  if (!tri) return tm * tn;
  long long t = 0;
  for (long long i = 0; i < tm; ++i) t += std::min(tn, 2 * (i + 1));
  return t;
}

ed_status oz_operand_buffer(OzContext* o, long long max_elems, long long max_rows, OzOperand* out) {
  ED_TRY(oz_alloc(o, (void**)&out->slices, (size_t)kOzDigits * (size_t)max_elems * 2));
  ED_TRY(oz_alloc(o, (void**)&out->exps, (size_t)max_rows * sizeof(int)));
  return ED_OK;
}

ed_status oz_map(OzContext* o, OzOperand* op, int R, int K, bool a_role, int* map) {
  op->R = R;
  op->K = K;
  op->Kpad = (K + 7) / 8 * 8;
  ED_TRY(make_map(o, op, a_role ? kOzBM : kOzBN));
  *map = op->map;
  return ED_OK;
}

// ---------------------------------------------------------------- slicing kernels

__device__ inline int find_job(const OzSliceJob* jobs, int n, long long u) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].first <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// operand rows = source rows: one warp per row (exponent by a warp max, then
// the digits of every element, one BF16 plane store per digit)
__global__ void __launch_bounds__(256) k_oz_slice_rows(const OzSliceJob* __restrict__ jobs, int njobs, long long units,
                                                       const double* __restrict__ x) {
  const long long u = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (u >= units) return;
  const OzSliceJob J = jobs[find_job(jobs, njobs, u)];
  const int i = (int)(u - J.first);
  const double* src = (J.sbase == 1 ? x + J.soff : J.src) + (long long)i * J.ld;
  double mx = 0.0;
  for (int k = lane; k < J.cols; k += 32) mx = fmax(mx, fabs(src[k]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const int E = exp_of(mx);
  if (lane == 0) J.exps[i] = E;
  const long long plane = (long long)J.rows * J.Kpad;
  uint16_t* row = J.dst + (long long)i * J.Kpad;
  for (int k = lane; k < J.Kpad; k += 32) {
    int d[kOzDigits];
    digits_dev(k < J.cols ? src[k] : 0.0, E, d);
#pragma unroll
    for (int p = 0; p < kOzDigits; ++p) row[p * plane + k] = bf16_of_small_int(d[p]);
  }
}

// operand rows = source columns (the transpose): one CTA per strip of 32
// source columns -- per-column exponent over all rows, then 32 x 32 tiles
// transposed through shared memory so both reads and digit stores coalesce
__global__ void __launch_bounds__(256) k_oz_slice_cols(const OzSliceJob* __restrict__ jobs, int njobs,
                                                       long long units, const double* __restrict__ x) {
  __shared__ double tile[32][33];
  __shared__ double cmax[8][32];
  __shared__ int cexp[32];
  const long long u = blockIdx.x;
  if (u >= units) return;
  const OzSliceJob J = jobs[find_job(jobs, njobs, u)];
  const int c0 = (int)(u - J.first) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const double* src = J.sbase == 1 ? x + J.soff : J.src;
  double mx = 0.0;
  if (c0 + tx < J.cols)
    for (int r = ty; r < J.rows; r += 8) mx = fmax(mx, fabs(src[(long long)r * J.ld + c0 + tx]));
  cmax[ty][tx] = mx;
  __syncthreads();
  if (ty == 0) {
    double m = 0.0;
    for (int q = 0; q < 8; ++q) m = fmax(m, cmax[q][tx]);
    const int E = exp_of(m);
    cexp[tx] = E;
    if (c0 + tx < J.cols) J.exps[c0 + tx] = E;
  }
  __syncthreads();
  const long long plane = (long long)J.cols * J.Kpad;  // operand rows = source columns
  for (int r0 = 0; r0 < J.Kpad; r0 += 32) {
    for (int q = ty; q < 32; q += 8) {
      const int r = r0 + q, c = c0 + tx;
      tile[q][tx] = (r < J.rows && c < J.cols) ? src[(long long)r * J.ld + c] : 0.0;
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {
      const int c = c0 + q, k = r0 + tx;  // operand row c, column k
      if (c < J.cols && k < J.Kpad) {
        int d[kOzDigits];
        digits_dev(tile[tx][q], cexp[q], d);
        uint16_t* row = J.dst + (long long)c * J.Kpad;
#pragma unroll
        for (int p = 0; p < kOzDigits; ++p) row[p * plane + k] = bf16_of_small_int(d[p]);
      }
    }
    __syncthreads();
  }
}

ed_status oz_slice(OzContext* o, const OzSliceJob* d_jobs, int njobs, long long units, bool transpose,
                   const double* x, cudaStream_t st) {
  if (units <= 0) return ED_OK;
  if (transpose)
    k_oz_slice_cols<<<(unsigned)units, 256, 0, st>>>(d_jobs, njobs, units, x);
  else
    k_oz_slice_rows<<<(unsigned)((units + 7) / 8), 256, 0, st>>>(d_jobs, njobs, units, x);
  ED_CUDA_TRY(cudaGetLastError());
  return ED_OK;
}

// ---------------------------------------------------------------- the GEMM

constexpr int kOzThreads = 192;          // warps 0-3 epilogue, 4 TMA producer, 5 MMA issuer
constexpr int kOzAStages = 3;
constexpr int kOzATile = kOzBM * kOzBK * 2;   // 16 KB
constexpr int kOzBTile = kOzBN * kOzBK * 2;   // 8 KB
constexpr int kOzBBuf = kOzDigits * kOzBTile; // the 8 digit planes of one K step: 64 KB
constexpr int kOzTmemCols = 512;              // 8 accumulators of 64 columns
constexpr long long kOzSpin = 1ll << 26;      // bounded waits (about a second)
constexpr size_t kOzSmem = 1024 + 2 * kOzBBuf + kOzAStages * kOzATile + 256;

__device__ inline int find_prob(const OzProblem* probs, int n, long long tile) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (probs[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kOzThreads, 1)
    k_oz_gemm(const OzProblem* __restrict__ probs, int nprob, const CUtensorMap* __restrict__ maps, double* y,
              int* err) {
  extern __shared__ unsigned char sm_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sB = sm;                       // [2][8 planes][64 rows][128 B]
  unsigned char* sA = sm + 2 * kOzBBuf;         // [3][128 rows][128 B]
  uint64_t* bar = (uint64_t*)(sA + kOzAStages * kOzATile);
  uint64_t* b_full = bar;          // 2
  uint64_t* b_empty = bar + 2;     // 2
  uint64_t* a_full = bar + 4;      // 3
  uint64_t* a_empty = bar + 7;     // 3
  uint64_t* acc_full = bar + 10;
  uint64_t* acc_empty = bar + 11;
  uint64_t* mma_done = bar + 12;
  __shared__ unsigned s_tmem;
  __shared__ volatile int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  const OzProblem P = probs[find_prob(probs, nprob, (long long)blockIdx.x)];
  long long t = (long long)blockIdx.x - P.tile0;
  int m0, n0;
  if (!P.tri) {
    m0 = (int)(t / P.tiles_n) * kOzBM;
    n0 = (int)(t % P.tiles_n) * kOzBN;
  } else {  // tile row tm holds the column tiles 0 .. min(tiles_n, 2 tm + 2) - 1
    int tm = 0;
    while (t >= min((long long)P.tiles_n, 2ll * (tm + 1))) {
      t -= min((long long)P.tiles_n, 2ll * (tm + 1));
      ++tm;
    }
    m0 = tm * kOzBM;
    n0 = (int)t * kOzBN;
  }
  const int nkb = (P.K + kOzBK - 1) / kOzBK;
  const int kb_per_chunk = kOzKChunk / kOzBK;
  const int nchunk = (nkb + kb_per_chunk - 1) / kb_per_chunk;

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&b_full[i], 1);
      tc::mbar_init(&b_empty[i], 1);
    }
    for (int i = 0; i < kOzAStages; ++i) {
      tc::mbar_init(&a_full[i], 1);
      tc::mbar_init(&a_empty[i], 1);
    }
    tc::mbar_init(acc_full, 1);
    tc::mbar_init(acc_empty, 128);
    tc::mbar_init(mma_done, 1);
    tc::fence_mbar_init();
    s_abort = 0;
  }
  if (warp == 0) tc::tmem_alloc(&s_tmem, kOzTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const unsigned tmem = s_tmem;

  if (warp == 4) {
    // ---- TMA producer: per K step the 8 digit planes of B^T, then A's planes one by one
    if (lane == 0) {
      const CUtensorMap* ma = maps + P.mapA;
      const CUtensorMap* mb = maps + P.mapB;
      long long na = 0;
      for (int kb = 0; kb < nkb && !s_abort; ++kb) {
        const int b = kb & 1, ub = kb >> 1;
        if (ub > 0 && !tc::mbar_wait(&b_empty[b], (ub - 1) & 1, kOzSpin)) { s_abort = 1; break; }
        tc::mbar_expect_tx(&b_full[b], kOzBBuf);
        for (int q = 0; q < kOzDigits; ++q)
          tc::tma_load_3d(sB + b * kOzBBuf + q * kOzBTile, mb, kb * kOzBK, n0, q, &b_full[b]);
        for (int p = 0; p < kOzDigits; ++p, ++na) {
          const int s = (int)(na % kOzAStages);
          const long long ua = na / kOzAStages;
          if (ua > 0 && !tc::mbar_wait(&a_empty[s], (unsigned)((ua - 1) & 1), kOzSpin)) { s_abort = 1; break; }
          tc::mbar_expect_tx(&a_full[s], kOzATile);
          tc::tma_load_3d(sA + s * kOzATile, ma, kb * kOzBK, m0, p, &a_full[s]);
        }
      }
      if (s_abort) atomicExch(err, 1);
    }
  } else if (warp == 5) {
    // ---- MMA issuer: accumulator g (TMEM columns 64 g) sums the digit pairs p + q = g
    if (lane == 0) {
      const unsigned idesc = tc::idesc_bf16_f32(kOzBM, kOzBN);
      long long na = 0;
      for (int c = 0; c < nchunk && !s_abort; ++c) {
        if (c > 0 && !tc::mbar_wait(acc_empty, (c - 1) & 1, kOzSpin)) { s_abort = 1; break; }
        tc::tc_fence_after();
        const int kb_end = min(nkb, (c + 1) * kb_per_chunk);
        for (int kb = c * kb_per_chunk; kb < kb_end && !s_abort; ++kb) {
          const int b = kb & 1, ub = kb >> 1;
          if (!tc::mbar_wait(&b_full[b], ub & 1, kOzSpin)) { s_abort = 1; break; }
          tc::tc_fence_after();
          const bool first_kb = kb == c * kb_per_chunk;
          for (int p = 0; p < kOzDigits; ++p, ++na) {
            const int s = (int)(na % kOzAStages);
            if (!tc::mbar_wait(&a_full[s], (unsigned)((na / kOzAStages) & 1), kOzSpin)) { s_abort = 1; break; }
            tc::tc_fence_after();
            const uint64_t da = tc::sdesc_kmajor_sw128(sA + s * kOzATile);
            for (int q = 0; q + p < kOzDigits; ++q) {
              const uint64_t db = tc::sdesc_kmajor_sw128(sB + b * kOzBBuf + q * kOzBTile);
              const unsigned dt = tmem + (unsigned)((p + q) * kOzBN);
#pragma unroll
              for (int kk = 0; kk < kOzBK / 16; ++kk)  // 32 bytes of K per instruction
                tc::mma_bf16(dt, da + 2 * kk, db + 2 * kk, idesc, !(first_kb && p == 0 && kk == 0));
            }
            tc::mma_commit(&a_empty[s]);
          }
          tc::mma_commit(&b_empty[b]);
        }
        tc::mma_commit(acc_full);
      }
      // every issued MMA finishes before the accumulators are released
      tc::mma_commit(mma_done);
      if (!tc::mbar_wait(mma_done, 0, kOzSpin)) s_abort = 1;
      if (s_abort) atomicExch(err, 1);
    }
  } else {
    // ---- epilogue: thread = one output row.  The 8 digit-order sums S_g of
    // a chunk are exact integers below 2^24 held in FP32; per column they
    // become one 128-bit integer T = sum_g S_g 2^(42 - 6g) (orders 0-3 and
    // 4-7 summed in two 64-bit integers first) on the integer pipe, rounded
    // once to FP64 by bit manipulation (C = T 2^(E_A + E_B - 52)).  With
    // more than one K chunk the chunks' rounded values add in FP64.
    const int row = warp * 32 + lane;
    const int i = m0 + row;
    const bool rv = i < P.M;
    const int ea = rv ? P.ea[i] : 0;
    double* crow = rv ? (P.cbase == 1 ? y + P.coff : P.C) + (long long)i * P.ldc : nullptr;
    const unsigned tl = tmem + ((unsigned)(warp * 32) << 16);
    // T of the 8 columns 8q .. 8q + 7 of the tile
    auto group = [&](int q, I128* T) {
      long long H[8], L[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) H[j] = L[j] = 0;
#pragma unroll
      for (int g = 0; g < kOzDigits; ++g) {
        float v[8];
        tc::tmem_ld8(tl + (unsigned)(g * kOzBN + 8 * q), v);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const long long sg = (long long)__float2int_rn(v[j]);
          if (g < 4) H[j] += sg << (6 * (3 - g));
          else L[j] += sg << (6 * (7 - g));
        }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        I128 h, l;
        h.lo = (unsigned long long)H[j] << 24;
        h.hi = H[j] >> 40;
        l.lo = (unsigned long long)L[j];
        l.hi = L[j] >> 63;
        T[j] = h + l;
      }
    };
    // an accumulating product reads its C tile after the products: bring the
    // tile's rows into L2 now, while the tensor cores run
    if (P.acc && rv) {
#pragma unroll
      for (int q = 0; q < kOzBN * 8 / 128; ++q) {
        const int col = n0 + q * 16;
        if (col < P.N) asm volatile("prefetch.global.L2 [%0];" ::"l"(crow + col));
      }
    }
    auto wait_chunk = [&](int c) -> bool {
      bool ok = false;
      for (long long it = 0; it < kOzSpin && !ok; ++it) {
        ok = tc::mbar_try(acc_full, c & 1);
        if (!ok && s_abort) break;
      }
      if (!ok) s_abort = 1;
      return ok;
    };
    if (nchunk == 1) {
      if (wait_chunk(0)) {
        tc::tc_fence_after();
#pragma unroll 1
        for (int q = 0; q < kOzBN / 8; ++q) {
          I128 T[8];
          group(q, T);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int col = n0 + 8 * q + j;
            if (rv && col < P.N) {
              const double v = from_fixed128(T[j], ea + P.eb[col] - 52);
              crow[col] = P.acc ? crow[col] + v : v;
            }
          }
        }
        tc::tc_fence_before();
        tc::mbar_arrive(acc_empty);
      }
    } else {
      double acc[kOzBN];
#pragma unroll
      for (int j = 0; j < kOzBN; ++j) acc[j] = 0.0;
      for (int c = 0; c < nchunk; ++c) {
        if (!wait_chunk(c)) break;
        tc::tc_fence_after();
#pragma unroll
        for (int q = 0; q < kOzBN / 8; ++q) {
          I128 T[8];
          group(q, T);
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[8 * q + j] += from_fixed128(T[j], -42);
        }
        tc::tc_fence_before();
        tc::mbar_arrive(acc_empty);
      }
      if (!s_abort && rv) {
#pragma unroll
        for (int j = 0; j < kOzBN; ++j) {
          const int col = n0 + j;
          if (col < P.N) {
            const double v = acc[j] * pow2(ea + P.eb[col] - 10);
            crow[col] = P.acc ? crow[col] + v : v;
          }
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, kOzTmemCols);
  }
}

ed_status oz_gemm(OzContext* o, const OzProblem* d_probs, int nprob, long long tiles, double* y, cudaStream_t st) {
  if (tiles <= 0) return ED_OK;
  // the shared-memory opt-in, once per device (calls may come from several host threads)
  static std::atomic<unsigned long long> attr_set{0};
  const unsigned long long bit = 1ull << (o->device & 63);
  if (!(attr_set.load() & bit)) {
    ED_CUDA_TRY(cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzSmem));
    attr_set.fetch_or(bit);
  }
  k_oz_gemm<<<(unsigned)tiles, kOzThreads, kOzSmem, st>>>(d_probs, nprob, o->d_maps, y, o->d_err);
  ED_CUDA_TRY(cudaGetLastError());
  return ED_OK;
}

}  // namespace edk
