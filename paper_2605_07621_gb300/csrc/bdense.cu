// Dense H|psi> of small batched instances on the tensor cores.
//
// An instance is one block Psi (d_A x d_B, row-major) of a Hubbard model
// with the spin cut, which leaves no cross terms, so Eq. (2) reads
//   H psi = H_A Psi + Psi H_B^T + V o Psi
// with the side operators H_A, H_B (hopping of the up and of the down
// electrons) and the diagonal V.  Both products run as BF16 tcgen05 MMAs with
// FP32 accumulation in TMEM.  Every FP32 value v (of H_A, H_B and Psi) is
// split into three BF16 pieces v = h0 + h1 + h2 (8 significant bits each,
// 24 in all, each piece the rounding of what the previous ones leave); the
// piece products h_p(H) h_q(Psi) with p + q <= 2 are accumulated in FP32,
// the dropped ones (p + q >= 3) being below 2^-24 of the leading product.
// The leading products (p = q = 0) and the corrections (p + q = 1, 2) go into
// two accumulators, so the rounding of the many small correction sums does
// not fall on the large leading sum; both products of an output tile (they
// add) share them, and the epilogue adds the two and the diagonal.
//
// Per output tile (128 rows a x BN columns b): the K steps of H_A Psi
// (A operand: H_A's pieces, rows a; B operand: Psi^T's pieces, rows b, both
// K = a' contiguous) and then those of Psi H_B^T (A: Psi's pieces, rows a;
// B: H_B's pieces, rows b, K = b' contiguous).  Tiles staged by TMA with
// 128-byte swizzle, one thread issues the MMAs, four warps drain the
// accumulators (those of two tiles alternate, so the epilogue of one tile
// overlaps the products of the next).  Persistent: each CTA walks the tile
// list of the active instances, read from device memory.
#include <cuda_bf16.h>

#include <cstring>

#include "batch.h"
#include "batch_dev.cuh"
#include "tc.cuh"

namespace edk {

constexpr int kBdEpiWarps = 8;   // two per TMEM lane quarter, splitting the columns
constexpr int kBdThreads = 32 * (kBdEpiWarps + 2);  // warps 0-7 epilogue, 8 TMA producer, 9 MMA issuer
constexpr int kBdWarpTma = kBdEpiWarps, kBdWarpMma = kBdEpiWarps + 1;
constexpr int kBdTrans = 32 * 33;  // floats of one warp's transpose buffer
constexpr int kBdBM = 128;       // output rows per tile (UMMA M)
constexpr int kBdBK = 64;        // K per pipeline step: one 128-byte swizzle row of BF16
constexpr int kBdPieces = 3;
constexpr long long kBdSpin = 1ll << 26;  // bounded waits (about a second)

// tensor maps of one slot: the A-role maps have 128-row boxes, the B-role
// maps BN-row boxes
enum { kMapHA = 0, kMapXN = 1, kMapXT64 = 2, kMapHB64 = 3, kMapXT128 = 4, kMapHB128 = 5 };

template <int BN>
struct BdCfg {
  static constexpr int kStages = 2;
  static constexpr int kATile = kBdBM * kBdBK * 2;  // one piece: 16 KB
  static constexpr int kBTile = BN * kBdBK * 2;
  static constexpr int kStage = kBdPieces * (kATile + kBTile);
  static constexpr int kTmemCols = 4 * BN;  // two tiles in flight x (leading, corrections)
  static constexpr size_t kSmem = 1024 + (size_t)kStages * kStage + 256 + (size_t)kBdEpiWarps * kBdTrans * 4;
};

// ---------------------------------------------------------------- pieces

__device__ __forceinline__ void split3_dev(float v, uint16_t& h0, uint16_t& h1, uint16_t& h2) {
  const __nv_bfloat16 a = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(a);
  const __nv_bfloat16 b = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(b);
  const __nv_bfloat16 c = __float2bfloat16_rn(r2);
  h0 = __bfloat16_as_ushort(a);
  h1 = __bfloat16_as_ushort(b);
  h2 = __bfloat16_as_ushort(c);
}

// Pieces of Psi (rows a, K = b) and of Psi^T (rows b, K = a) for every dense
// instance: 64 x 64 tiles of Psi through shared memory; every warp store
// writes 32 pairs of BF16 (128 bytes) along a row of either layout.  The
// piece rows start on multiples of 64 elements, so pairs at even columns
// are 4-byte aligned.
__global__ void __launch_bounds__(256) k_bslice(BDenseArgs g) {
  __shared__ float tile[64][65];
  const int n = g.cnt[1];
  if (n <= 0) return;
  const long long total = g.dspref[n];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (long long u = blockIdx.x; u < total; u += gridDim.x) {
    const int ai = find_pref(g.dspref, n, u);
    const BInst& I = g.insts[g.didx[ai]];
    const int dA = I.dA, dB = I.dB;
    const long long t = u - g.dspref[ai];
    const int tnb = (dB + 63) >> 6;
    const int a0 = (int)(t / tnb) * 64, b0 = (int)(t % tnb) * 64;
    const float* __restrict__ x = g.user_mode ? g.ux + I.uoff : g.arena + I.voff + I.D;
    uint16_t* __restrict__ XN = I.XN;
    uint16_t* __restrict__ XT = I.XT;
    const long long pn = (long long)dA * I.KpB, pt = (long long)dB * I.KpA;
    for (int i = threadIdx.x; i < 64 * 64; i += 256) {
      const int r = i >> 6, c = i & 63;
      const int a = a0 + r, b = b0 + c;
      tile[r][c] = (a < dA && b < dB) ? x[(long long)a * dB + b] : 0.f;
    }
    __syncthreads();
    const int c = 2 * lane;
    for (int r = warp; r < 64; r += 8) {
      const int a = a0 + r, b = b0 + c;  // Psi row a, columns b, b + 1
      if (a < dA && b < dB) {
        uint16_t h0, h1, h2, k0, k1, k2;
        split3_dev(tile[r][c], h0, h1, h2);
        split3_dev(tile[r][c + 1], k0, k1, k2);  // zero past d_B: the padding of the row
        uint32_t* d = reinterpret_cast<uint32_t*>(XN + (long long)a * I.KpB + b);
        d[0] = h0 | ((uint32_t)k0 << 16);
        d[pn / 2] = h1 | ((uint32_t)k1 << 16);
        d[pn] = h2 | ((uint32_t)k2 << 16);
      }
    }
    for (int r = warp; r < 64; r += 8) {
      const int b = b0 + r, a = a0 + c;  // Psi^T row b, columns a, a + 1
      if (a < dA && b < dB) {
        uint16_t h0, h1, h2, k0, k1, k2;
        split3_dev(tile[c][r], h0, h1, h2);
        split3_dev(tile[c + 1][r], k0, k1, k2);
        uint32_t* d = reinterpret_cast<uint32_t*>(XT + (long long)b * I.KpA + a);
        d[0] = h0 | ((uint32_t)k0 << 16);
        d[pt / 2] = h1 | ((uint32_t)k1 << 16);
        d[pt] = h2 | ((uint32_t)k2 << 16);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- tables

// Dense H_A, H_B pieces and their nonzero-K-block masks from the instance's
// CSR rows (zeroed beforehand): one thread per row of either side; entries
// with the same column are summed before the split.
__global__ void k_btables(BInst I) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool onA = r < I.dA;
  if (r >= (long long)I.dA + I.dB) return;
  const long long row = onA ? r : r - I.dA;
  const int d = onA ? I.dA : I.dB;
  const int* rp = onA ? I.A_rp : I.B_rp;
  const int* col = onA ? I.A_col : I.B_col;
  const float* val = onA ? I.A_val : I.B_val;
  uint16_t* P = const_cast<uint16_t*>(onA ? I.HA : I.HB);
  const int kp = onA ? I.KpA : I.KpB;
  const long long plane = (long long)d * kp;
  uint32_t* km = const_cast<uint32_t*>(I.kmask);
  const int tmA = (I.dA + kBdBM - 1) / kBdBM, tn64 = (I.dB + 63) / 64;
  for (int e = rp[row]; e < rp[row + 1]; ++e) {
    const int c = col[e];
    bool seen = false;
    for (int f = rp[row]; f < e; ++f) seen = seen || col[f] == c;
    if (seen) continue;
    float v = 0.f;
    for (int f = e; f < rp[row + 1]; ++f)
      if (col[f] == c) v += val[f];
    uint16_t h0, h1, h2;
    split3_dev(v, h0, h1, h2);
    P[row * kp + c] = h0;
    P[plane + row * kp + c] = h1;
    P[2 * plane + row * kp + c] = h2;
    const uint32_t bit = 1u << (c / kBdBK);
    if (onA) {
      atomicOr(&km[row / kBdBM], bit);
    } else {
      atomicOr(&km[tmA + row / 64], bit);
      atomicOr(&km[tmA + tn64 + row / 128], bit);
    }
  }
}

ed_status bdense_tables(const BInst& I, cudaStream_t st) {
  const long long n = (long long)I.dA + I.dB;
  k_btables<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(I);
  ED_CUDA_TRY(cudaGetLastError());
  return ED_OK;
}

// ---------------------------------------------------------------- products

// K steps of one output tile: the nonzero 64-wide K blocks of H_A's row
// tile (H_A Psi), then those of H_B's row tile (Psi H_B^T); entry = kb, plus
// 32 for the second product (kb < 16 as d <= 1024).  A tile with none gets
// one zero block (which clears its accumulators).
template <int BN>
__device__ __forceinline__ int tile_steps(const BInst& I, int m0, int n0, unsigned char* ks) {
  const int tmA = (I.dA + kBdBM - 1) / kBdBM, tn64 = (I.dB + 63) / 64;
  const uint32_t ma = I.kmask[m0 / kBdBM];
  const uint32_t mb = BN == 64 ? I.kmask[tmA + n0 / 64] : I.kmask[tmA + tn64 + n0 / 128];
  int n = 0;
  for (uint32_t m = ma; m; m &= m - 1) ks[n++] = (unsigned char)__ffs(m) - 1;
  for (uint32_t m = mb; m; m &= m - 1) ks[n++] = (unsigned char)(32 + __ffs(m) - 1);
  if (n == 0) ks[n++] = 0;
  return n;
}

template <int BN>
__global__ void __launch_bounds__(kBdThreads, 1) k_bgemm(BDenseArgs g, int which) {
  using C = BdCfg<BN>;
  const int n = g.cnt[which];
  if (n <= 0) return;
  const int* vidx = BN == 64 ? g.idx64 : g.idx128;
  const long long* tpref = BN == 64 ? g.tpref64 : g.tpref128;
  const long long total = tpref[n];
  if ((long long)blockIdx.x >= total) return;

  extern __shared__ unsigned char sm_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bar = (uint64_t*)(sm + C::kStages * C::kStage);
  uint64_t* full = bar;                      // kStages
  uint64_t* empty = bar + C::kStages;        // kStages
  uint64_t* acc_full = bar + 2 * C::kStages; // 2
  uint64_t* acc_empty = acc_full + 2;        // 2
  uint64_t* mma_done = acc_empty + 2;
  float* trans = (float*)(sm + C::kStages * C::kStage + 256);  // kBdEpiWarps x [32][33]
  __shared__ unsigned s_tmem;
  __shared__ volatile int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int i = 0; i < C::kStages; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&acc_full[i], 1);
      tc::mbar_init(&acc_empty[i], 32 * kBdEpiWarps);
    }
    tc::mbar_init(mma_done, 1);
    tc::fence_mbar_init();
    s_abort = 0;
  }
  if (warp == 0) tc::tmem_alloc(&s_tmem, C::kTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const unsigned tmem = s_tmem;

  // tile -> (slot, first row, first column)
  auto decode = [&](long long tile, int& slot, int& m0, int& n0) {
    const int ai = find_pref(tpref, n, tile);
    slot = vidx[ai];
    const int tn = (g.insts[slot].dB + BN - 1) / BN;
    const long long t = tile - tpref[ai];
    m0 = (int)(t / tn) * kBdBM;
    n0 = (int)(t % tn) * BN;
  };

  if (warp == kBdWarpTma) {
    // ---- TMA producer: per K step the three pieces of the A tile and of the B tile
    if (lane == 0) {
      long long it = 0;
      unsigned char kst[32];
      constexpr int kAhead = 3;  // K steps prefetched into L2 ahead of their loads
      for (long long tile = blockIdx.x; tile < total && !s_abort; tile += gridDim.x) {
        int slot, m0, n0;
        decode(tile, slot, m0, n0);
        const int nk = tile_steps<BN>(g.insts[slot], m0, n0, kst);
        const CUtensorMap* mp = g.maps + (long long)slot * kBMaps;
        const CUtensorMap* mXT = mp + (BN == 64 ? kMapXT64 : kMapXT128);
        const CUtensorMap* mHB = mp + (BN == 64 ? kMapHB64 : kMapHB128);
        auto prefetch = [&](int k) {
          const bool first = kst[k] < 32;  // H_A Psi, then Psi H_B^T
          const int kc = (kst[k] & 31) * kBdBK;
#pragma unroll
          for (int p = 0; p < kBdPieces; ++p) {
            tc::tma_prefetch_3d(first ? mp + kMapHA : mp + kMapXN, kc, m0, p);
            tc::tma_prefetch_3d(first ? mXT : mHB, kc, n0, p);
          }
        };
        for (int k = 0; k < kAhead && k < nk; ++k) prefetch(k);
        for (int ks = 0; ks < nk; ++ks, ++it) {
          if (ks + kAhead < nk) prefetch(ks + kAhead);
          const int s = (int)(it % C::kStages);
          const long long u = it / C::kStages;
          if (u > 0 && !tc::mbar_wait(&empty[s], (unsigned)((u - 1) & 1), kBdSpin)) {
            s_abort = 1;
            break;
          }
          unsigned char* sa = sm + s * C::kStage;
          unsigned char* sb = sa + kBdPieces * C::kATile;
          const bool first = kst[ks] < 32;
          const int kc = (kst[ks] & 31) * kBdBK;
          const CUtensorMap* ma = first ? mp + kMapHA : mp + kMapXN;
          const CUtensorMap* mb = first ? mXT : mHB;
          tc::mbar_expect_tx(&full[s], C::kStage);
#pragma unroll
          for (int p = 0; p < kBdPieces; ++p) tc::tma_load_3d(sa + p * C::kATile, ma, kc, m0, p, &full[s]);
#pragma unroll
          for (int q = 0; q < kBdPieces; ++q) tc::tma_load_3d(sb + q * C::kBTile, mb, kc, n0, q, &full[s]);
        }
      }
      if (s_abort) atomicExch(g.err, 1);
    }
  } else if (warp == kBdWarpMma) {
    // ---- MMA issuer: piece pairs p + q <= 2 into the tile's accumulator
    if (lane == 0) {
      const unsigned idesc = tc::idesc_bf16_f32(kBdBM, BN);
      long long it = 0;
      int tl = 0;
      for (long long tile = blockIdx.x; tile < total && !s_abort; tile += gridDim.x, ++tl) {
        int slot, m0, n0;
        decode(tile, slot, m0, n0);
        unsigned char kst[32];
        const int nk = tile_steps<BN>(g.insts[slot], m0, n0, kst);
        const int buf = tl & 1, use = tl >> 1;
        if (use > 0 && !tc::mbar_wait(&acc_empty[buf], (unsigned)((use - 1) & 1), kBdSpin)) {
          s_abort = 1;
          break;
        }
        tc::tc_fence_after();
        const unsigned dt = tmem + (unsigned)(2 * buf * BN);  // leading; corrections at + BN
        for (int ks = 0; ks < nk; ++ks, ++it) {
          const int s = (int)(it % C::kStages);
          if (!tc::mbar_wait(&full[s], (unsigned)((it / C::kStages) & 1), kBdSpin)) {
            s_abort = 1;
            break;
          }
          tc::tc_fence_after();
          unsigned char* sa = sm + s * C::kStage;
          unsigned char* sb = sa + kBdPieces * C::kATile;
#pragma unroll
          for (int p = 0; p < kBdPieces; ++p) {
            const uint64_t da = tc::sdesc_kmajor_sw128(sa + p * C::kATile);
#pragma unroll
            for (int q = 0; q + p < kBdPieces; ++q) {
              const uint64_t db = tc::sdesc_kmajor_sw128(sb + q * C::kBTile);
#pragma unroll
              for (int kk = 0; kk < kBdBK / 16; ++kk)  // 32 bytes of K per instruction
                tc::mma_bf16(dt + (p + q > 0 ? BN : 0), da + 2 * kk, db + 2 * kk, idesc,
                             !(ks == 0 && p == 0 && q <= 1 && kk == 0));
            }
          }
          tc::mma_commit(&empty[s]);
        }
        if (s_abort) break;
        tc::mma_commit(&acc_full[buf]);
      }
      // every issued MMA finishes before the accumulators are released
      tc::mma_commit(mma_done);
      if (!tc::mbar_wait(mma_done, 0, kBdSpin)) s_abort = 1;
      if (s_abort) atomicExch(g.err, 1);
    }
  } else {
    // ---- epilogue: warp w drains TMEM lanes 32 (w % 4) .. + 31 (tile rows)
    // for every other 32-column chunk; each 32 x 32 chunk is transposed
    // through shared memory so the loads of x and the stores of
    // y = accumulators + V x run along rows (lane = column)
    const int quarter = warp & 3, half = warp >> 2;
    float* tr = trans + warp * kBdTrans;
    int tl = 0;
    for (long long tile = blockIdx.x; tile < total; tile += gridDim.x, ++tl) {
      int slot, m0, n0;
      decode(tile, slot, m0, n0);
      const BInst& I = g.insts[slot];
      const int buf = tl & 1, use = tl >> 1;
      bool ok = false;
      for (long long i = 0; i < kBdSpin && !ok; ++i) {
        ok = tc::mbar_try(&acc_full[buf], (unsigned)(use & 1));
        if (!ok && s_abort) break;
      }
      if (!ok) {
        s_abort = 1;
        break;
      }
      tc::tc_fence_after();
      // the instance's fields in registers (y stores could alias them otherwise)
      const int dA = I.dA, dB = I.dB;
      const int r0 = m0 + quarter * 32;  // this warp's first row
      const float* __restrict__ x = g.user_mode ? g.ux + I.uoff : g.arena + I.voff + I.D;
      float* __restrict__ y = g.user_mode ? g.uy + I.uoff : g.arena + I.voff + 2 * I.D;
      const uint32_t* __restrict__ Bs = I.B_str;
      const float* __restrict__ Bd = I.B_diag;
      const int ncls = I.ncls, vand = I.vab_and;
      float w[kMaxClasses];
      unsigned mk[kMaxClasses];
#pragma unroll
      for (int q = 0; q < kMaxClasses; ++q) {
        w[q] = I.w[q];
        mk[q] = I.mask[q];
      }
      // lane r holds row r0 + r's side-A string and diagonal
      const int nr = min(32, dA - r0);  // rows of this warp inside the block (may be <= 0)
      float dal = 0.f;
      uint32_t sal = 0;
      if (lane < nr) {
        dal = I.A_diag[r0 + lane] + I.c0;
        sal = I.A_str[r0 + lane];
      }
#pragma unroll 1
      for (int c = half; c < BN / 32; c += 2) {
        float v[32], u[32];
        const unsigned ta = tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)(2 * buf * BN + c * 32);
        tc::tmem_ld32(ta, v);
        tc::tmem_ld32(ta + BN, u);
#pragma unroll
        for (int j = 0; j < 32; ++j) tr[lane * 33 + j] = v[j] + u[j];
        __syncwarp();
        const int col = n0 + c * 32 + lane;
        const bool cv = col < dB;
        const uint32_t sb = cv ? Bs[col] : 0u;
        const float bd = cv ? Bd[col] : 0.f;
        const float* __restrict__ xc = x + (long long)r0 * dB + col;
        float* __restrict__ yc = y + (long long)r0 * dB + col;
        // all 32 rows' x loads in flight before any is used (x is read from
        // DRAM here: one load at a time per warp would leave the epilogue
        // bound by memory latency)
        float xv[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) xv[r] = (r < nr && cv) ? xc[(long long)r * dB] : 0.f;
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const uint32_t sa = __shfl_sync(0xffffffffu, sal, r);
          const float da = __shfl_sync(0xffffffffu, dal, r);
          if (r < nr && cv) {
            const uint32_t z = vand ? (sa & sb) : (sa ^ sb);
            float dg = da + bd;
#pragma unroll
            for (int q = 0; q < kMaxClasses; ++q)  // unrolled: w, mk stay in registers
              if (q < ncls) dg += w[q] * (float)__popc(z & mk[q]);
            yc[(long long)r * dB] = fmaf(dg, xv[r], tr[r * 33 + lane]);
          }
        }
        __syncwarp();
      }
      tc::tc_fence_before();
      tc::mbar_arrive(&acc_empty[buf]);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, C::kTmemCols);
  }
}

ed_status bdense_prepare() {
  ED_CUDA_TRY(cudaFuncSetAttribute(k_bgemm<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BdCfg<64>::kSmem));
  ED_CUDA_TRY(cudaFuncSetAttribute(k_bgemm<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BdCfg<128>::kSmem));
  return ED_OK;
}

ed_status bdense_apply(const BDenseArgs& a, cudaStream_t st) {
  k_bslice<<<a.sms * 8, 256, 0, st>>>(a);
  k_bgemm<64><<<a.sms, kBdThreads, BdCfg<64>::kSmem, st>>>(a, 2);
  k_bgemm<128><<<a.sms, kBdThreads, BdCfg<128>::kSmem, st>>>(a, 3);
  ED_CUDA_TRY(cudaGetLastError());
  return ED_OK;
}

}  // namespace edk
