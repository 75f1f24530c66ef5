// Staged-source row pass (kernel template and launch helper).  Each
// element type is instantiated in its own translation unit (rowx_*.cu) so
// the unrolled variants compile in parallel.
#pragma once

#include "apply3.cuh"

namespace edk {

// ---------------------------------------------------------------- staged-source row pass
//
// Row pass for models with cross-cut bonds.  One CTA per SM; warp 0 is the
// producer, the other warps consume.  A row (s, a) of the output takes
// several phases, each one row of x staged whole in shared memory by a bulk
// TMA copy into a ring of buffers:
//   own phase     x_s[a,:]                    diagonal and H_B (Eq. (2));
//   source phase  x_s'[mapA_ia(a),:], one per A cross site ia whose flip
//                 leads to an existing row: the cross terms of all bonds
//                 (ia, ib) gather x_s'[., mapB_ib(b)] from shared memory.
// Every consumer thread owns the columns b = t + (NT - 32) * j, j < NCOL, of the current row and keeps their sums in registers across the
// phases, so y is written once per row.  Rows are taken from a dynamic work
// counter in an order where source rows are L2-resident (see the work-list
// builder).  Producer and consumers meet at per-buffer "full" (TMA
// complete) and "empty" (all consumer warps done) mbarriers; every wait is
// bounded and sets *err when it runs out.
// threads per CTA: 1024 for 4-byte types; 512 for 8-byte types, whose
// register sums need the larger per-thread register budget (128)
template <class S>
constexpr int rx_threads() { return sizeof(S) == 4 ? 1024 : 512; }
constexpr int kRxMaxBuf = 4;
constexpr int kRxMaxBondsPerSite = 4;

struct RxDesc {
  int kind;  // -2 done, -1 own row, >= 0 A cross site of a source row
  int pad;   // offset of the row's first element in the buffer
  int blk;   // block of the output row
  int a;     // row of the output row within its block
  int last;  // last phase of the output row
  int pad_[3];
};

// Per-row phase list, computed by the 32 lanes of the producer warp: lane 0
// the own row, lane 1 + ia the source row of A cross site ia.
struct RxRow {
  int r;              // work-list index (>= n_rows: no more work)
  int blk, a;
  unsigned valid;     // lanes with a phase
  long long e0;       // this lane's source row: first element, length
  int n;
};

template <class S>
__device__ __forceinline__ RxRow rx_fetch(const P3& p, const int2* __restrict__ rows, int n_rows, int* sched,
                                          int lane) {
  const Dev3& t = p.t;
  RxRow R;
  int r = 0;
  if (lane == 0) r = atomicAdd(sched, 1);
  R.r = __shfl_sync(0xffffffffu, r, 0);
  R.valid = 0;
  R.e0 = 0;
  R.n = 0;
  R.blk = 0;
  R.a = 0;
  if (R.r >= n_rows) return R;
  const int2 w = rows[R.r];
  R.blk = w.x;
  R.a = w.y;
  const DevBlock bl = p.blocks[w.x];
  const long long gA = bl.gA0 + w.y;
  bool ok = false;
  if (lane == 0) {
    R.e0 = bl.off + (long long)w.y * bl.dB;
    R.n = (int)bl.dB;
    ok = true;
  } else if (lane - 1 < t.n_ia) {
    const int ia = lane - 1;
    const unsigned km = t.ia_mask[ia];
    if (km) {
      const int k = __ffs(km) - 1;
      const unsigned pa = t.A_pack[gA];
      const int sb = ((pa >> k) & 1u) ? bl.nbr_lo : bl.nbr_hi;
      if (sb >= 0) {
        const unsigned rr = t.mapA[(long long)ia * t.A_total + gA];
        if (rr != 0xFFFFu) {
          const DevBlock so = p.blocks[sb];
          R.e0 = so.off + (long long)rr * so.dB;
          R.n = (int)so.dB;
          ok = true;
        }
      }
    }
  }
  R.valid = __ballot_sync(0xffffffffu, ok);
  return R;
}

template <class Pol, int NCOL, int NT = rx_threads<typename Pol::S>()>
__global__ void __launch_bounds__(NT, 1)
    k_rowx(P3 p, const int2* __restrict__ rows, int n_rows, const typename Pol::S* __restrict__ x,
           typename Pol::S* __restrict__ y, const int* __restrict__ emax, long long stage_elems, int nbuf, int* sched,
           int* err) {
  using S = typename Pol::S;
  constexpr int kRxConsumers = NT - 32;
  extern __shared__ __align__(16) unsigned char smemx[];
  unsigned long long* full = reinterpret_cast<unsigned long long*>(smemx);
  unsigned long long* empty = full + kRxMaxBuf;
  RxDesc* desc = reinterpret_cast<RxDesc*>(smemx + 64);
  S* bufs = reinterpret_cast<S*>(smemx + 64 + kRxMaxBuf * sizeof(RxDesc));
  constexpr int V = 16 / (int)sizeof(S);
  const Dev3& t = p.t;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < nbuf; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(&full[i])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_u32(&empty[i])), "r"(kRxConsumers / 32)
                   : "memory");
    }
    bar_fence_init();
  }
  __syncthreads();

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    long long ph = 0;
    RxRow nxt = rx_fetch<S>(p, rows, n_rows, sched, lane);
    for (;;) {
      const RxRow cur = nxt;
      const bool done = cur.r >= n_rows;
      unsigned vm = done ? 1u : cur.valid;
      bool first = true;
      while (vm) {
        const int l = __ffs(vm) - 1;
        vm &= vm - 1;
        const long long e0 = __shfl_sync(0xffffffffu, cur.e0, l);
        const int n = __shfl_sync(0xffffffffu, cur.n, l);
        const int buf = (int)(ph % nbuf);
        if (ph >= nbuf) {
          const bool ok = bar_wait(&empty[buf], (unsigned)(((ph / nbuf) - 1) & 1));
          if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) atomicExch(err, 1);
            return;
          }
        }
        if (lane == 0) {
          RxDesc d;
          d.kind = done ? -2 : (l == 0 ? -1 : l - 1);
          d.blk = cur.blk;
          d.a = cur.a;
          d.last = vm == 0;
          unsigned bytes = 0;
          long long gal = 0;
          if (!done) {
            S* b = bufs + (long long)buf * stage_elems;
            gal = e0 / V * V;
            const long long galend = (e0 + n) / V * V;
            d.pad = (int)(e0 - gal);
            if (galend > gal) bytes = (unsigned)((galend - gal) * (long long)sizeof(S));
            for (long long q = galend > e0 ? galend : e0; q < e0 + n; ++q) b[q - gal] = x[q];
            if (l == 0) b[d.pad + n] = (S)0;  // zero slot of the padded H_B index groups
          } else {
            d.pad = 0;
          }
          desc[buf] = d;
          proxy_fence();
          if (bytes) {
            bar_expect(&full[buf], bytes);
            bulk_g2s(bufs + (long long)buf * stage_elems, x + gal, bytes, &full[buf]);
          } else {
            bar_arrive(&full[buf]);
          }
        }
        __syncwarp();
        ++ph;
        if (first && !done) {
          first = false;
          nxt = rx_fetch<S>(p, rows, n_rows, sched, lane);  // overlaps the wait for the next buffer
        }
      }
      if (done) break;
    }
    // the consumers have waited on every copy this warp issued before they
    // read the final descriptor, so none is in flight here
    return;
  }

  // -------------------------------------------------------------- consumers
  const int ct = threadIdx.x - 32;
  const int e2 = emax ? out_exp(t, emax) : 0;
  S acc[NCOL];
  long long ph = 0;
  DevBlock bl{};
  unsigned pa = 0;
  S da = 0;
  for (;;) {
    const int buf = (int)(ph % nbuf);
    const bool ok = bar_wait(&full[buf], (unsigned)((ph / nbuf) & 1));
    if (!ok) {
      atomicExch(err, 1);
      return;
    }
    const RxDesc d = desc[buf];
    if (d.kind == -2) break;
    const S* xs = bufs + (long long)buf * stage_elems + d.pad;
    const int dB = (int)bl.dB;
    if (d.kind == -1) {
      // own phase: diagonal and H_B of a new output row
      bl = p.blocks[d.blk];
      const long long gA = bl.gA0 + d.a;
      pa = t.A_pack[gA];
      da = Pol::diagA(t, gA);
      const int dBn = (int)bl.dB;
      const long long gB0 = bl.gB0;
#pragma unroll
      for (int j = 0; j < NCOL; ++j) {
        const int b = ct + kRxConsumers * j;
        S v = 0;
        if (b < dBn) {
          const long long gB = gB0 + b;
          const uint2 m = t.B_meta4[gB];
          const unsigned pb = t.B_pack[gB];
          const unsigned z = t.vab_and ? (pa & pb) : (pa ^ pb);
          v = (da + Pol::diagB(t, gB) + Pol::vab(t, z)) * xs[b];
          const uint2* cp = t.B_col4 + m.x;
#pragma unroll
          for (int c = 0; c < kMaxCls; ++c) {
            const unsigned n4 = (m.y >> (8 * c)) & 255u;
            if (!n4) continue;
            S sum = 0;
            for (unsigned i = 0; i < n4; ++i) {
              const uint2 q = __ldg(cp + i);
              sum += (xs[q.x & 0xFFFFu] + xs[q.x >> 16]) + (xs[q.y & 0xFFFFu] + xs[q.y >> 16]);
            }
            cp += n4;
            v += Pol::w(t, c) * sum;
          }
        }
        acc[j] = v;
      }
    } else {
      // source phase of A cross site ia: bonds (ia, ib_q), valid where the
      // B bit differs from the row's A bit
      const int ia = d.kind;
      unsigned km = t.ia_mask[ia];
      int kq[kRxMaxBondsPerSite];
      int nb = 0;
#pragma unroll
      for (int q = 0; q < kRxMaxBondsPerSite; ++q) {
        kq[q] = km ? __ffs(km) - 1 : 0;
        if (km) ++nb;
        km &= km - 1;
      }
      const unsigned abit = (pa >> kq[0]) & 1u;
      const long long gB0 = bl.gB0;
      // validity bits: bit j of vq[q] says bond q is valid for column j
      unsigned vq[kRxMaxBondsPerSite] = {0u, 0u, 0u, 0u};
#pragma unroll
      for (int j = 0; j < NCOL; ++j) {
        const int b = ct + kRxConsumers * j;
        if (b < dB) {
          const unsigned pb = t.B_pack[gB0 + b] ^ (abit ? 0xFFFFFFFFu : 0u);
#pragma unroll
          for (int q = 0; q < kRxMaxBondsPerSite; ++q) vq[q] |= ((pb >> kq[q]) & 1u) << j;
        }
      }
#pragma unroll
      for (int q = 0; q < kRxMaxBondsPerSite; ++q) {
        if (q >= nb) break;
        const int k = kq[q];
        const S wk = Pol::bw(t, k);
        const uint16_t* mb = t.mapB + (long long)t.bond_ib[k] * t.B_total + gB0 + ct;
        const unsigned vm = vq[q];
#pragma unroll
        for (int j = 0; j < NCOL; ++j) {
          if ((vm >> j) & 1u) acc[j] += wk * xs[__ldg(mb + kRxConsumers * j)];
        }
      }
    }
    __syncwarp();
    if (lane == 0) bar_arrive(&empty[buf]);
    ++ph;
    if (d.last) {
      const bool final_ = !bl.has_hA;
      S* yr = y + bl.off + (long long)d.a * bl.dB;
      const int dBn = (int)bl.dB;
#pragma unroll
      for (int j = 0; j < NCOL; ++j) {
        const int b = ct + kRxConsumers * j;
        if (b < dBn) store_out<Pol>(yr, b, acc[j], final_, e2);
      }
    }
  }
}

// Launch plan of the staged-source row pass: columns per consumer thread
// (NCOL), ring depth, shared-memory bytes.  Used for spin models with
// cross-cut bonds when ED_OPS_ROW_STAGED asks for it.
// instantiated columns per consumer thread: at most 13 x 992 = 12,896
// columns per row for 4-byte types (more would spill registers) and
// 27 x 480 = 12,960 for 8-byte types
constexpr int kRxCols[4] = {4, 8, 13, 27};

struct RxPlan {
  int ncol = 0, nbuf = 0;
  long long stage = 0;
  size_t smem = 0;
};

template <class Pol, int NCOL>
ed_status rx_launch_n(ed_ctx* c, const P3& p, const RxPlan& rx, const typename Pol::S* x, typename Pol::S* y,
                             const int* emax, cudaStream_t st) {
  auto kern = k_rowx<Pol, NCOL>;
  ED_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rx.smem));
  const int grid = (int)std::min<long long>(c->n_rowx, (long long)n_sms(c->device));
  kern<<<grid, rx_threads<typename Pol::S>(), rx.smem, st>>>(p, c->d_rowx, (int)c->n_rowx, x, y, emax, rx.stage, rx.nbuf, c->d_sched,
                                          c->d_err);
  ED_CUDA_TRY(cudaGetLastError());
  return ED_OK;
}

// one overload per element type: float -> FP32, double -> FP64,
// long long -> exact fixed point
ed_status rx_launch(ed_ctx* c, const P3& p, const RxPlan& rx, const float* x, float* y, const int* emax,
                    cudaStream_t st);
ed_status rx_launch(ed_ctx* c, const P3& p, const RxPlan& rx, const double* x, double* y, const int* emax,
                    cudaStream_t st);
ed_status rx_launch(ed_ctx* c, const P3& p, const RxPlan& rx, const long long* x, long long* y, const int* emax,
                    cudaStream_t st);

}  // namespace edk
