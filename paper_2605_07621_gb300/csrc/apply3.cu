// Class-sorted H|psi> (paper Eq. (2)) in these arithmetic flavours:
//   FP32  storage and accumulation;
//   FP64  storage and accumulation (fallback);
//   I64   FP64 storage, exact 64-bit fixed-point accumulation: when every
//         matrix element is a small integer multiple of 2^-q_shift, x is
//         scaled by one power of two per vector, summed exactly on the
//         integer pipe and rounded once back to FP64.  FP64 adds and FP64
//         conversions run at about 0.5 T/s on this GPU, the integer pipe at
//         tens of T/s, so no FP64 instruction is issued per matrix element;
//   W128  the same for couplings that are not dyadic: FP64 values are
//         integer multiples of 2^-q_shift with up to 53-bit integers, so the
//         class sums are weighted by 64-bit integers into exact 128-bit sums,
//         rounded to FP64 once per pass;
//   C64   fixed-point class sums weighted in FP64 (value ranges too wide
//         for 64-bit integer weights).
// Row pass (k_row5): the diagonal, the H_B (column-mixing) term and the
// cross-cut terms of whole rows.  psi_s[a,:] is staged in shared memory by
// bulk TMA copies, then each column b sums, class by class, its H_B
// neighbours (16-bit column indices) and the cross-cut gathers from x in
// global memory, plus the diagonal.
// Panel pass: the H_A (row-mixing) term over column panels that stay
// resident in L2.
#include <mutex>
#include <type_traits>

#include "apply3.cuh"

namespace edk {

// host entry points of the two conversions (used by the CPU tests)
long long host_to_fixed(double v, int sh_base) { return to_fixed(v, sh_base); }
double host_from_fixed(long long Y, int e2) { return from_fixed(Y, e2); }
double host_from_fixed128(long long hi, unsigned long long lo, int e2) {
  I128 v;
  v.hi = hi;
  v.lo = lo;
  return from_fixed128(v, e2);
}
void host_mul_wide(long long a, long long b, long long* hi, unsigned long long* lo) {
  const I128 v = mul_wide(a, b);
  *hi = v.hi;
  *lo = v.lo;
}

// largest biased exponent of x (atomic max into out[0]; out must start at 0)
__global__ void k_exp_max(const double* __restrict__ x, long long n, int* out) {
  int m = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = max(m, (int)(((unsigned long long)__double_as_longlong(x[i]) >> 52) & 0x7ffull));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// |x| < 2^E with E = emax - 1022; X = round(x * 2^(P - E))
__global__ void k_to_fixed(const double* __restrict__ x, long long* __restrict__ X, long long n,
                           const int* __restrict__ emax, int P) {
  const int E = emax[0] - 1022;
  const int sh = P - E;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    X[i] = to_fixed(x[i], sh);
}

constexpr int kRowThreads = 512;
// valid-bond lists for the cross terms also for 4-byte types (off: the
// four-row FP32 pass measured slower with them, 17.2 vs 15.5 ms)
constexpr bool kListsF32 = false;

// Row pass: work unit = R consecutive rows of one block ("row group"),
// brought into shared memory by bulk TMA copies; one 1024-thread CTA per SM
// whose R staged rows (4 for 4-byte, 2 for 8-byte types) share every B-side
// load.  Per column b:
//  * H_B: the class segments of the column's index list are padded to
//    groups of four 16-bit indices, read with one 8-byte load per group
//    (several groups loaded ahead) and gathered from all R staged rows
//    (padding points at a zero slot);
//  * cross terms: one B-side map load per B cross site, shared by the R
//    rows, then one gather per valid bond from the neighbouring block (8-byte
//    types: from per-row lists of the valid bonds for each column bit and
//    value class, summed per class and weighted once per column);
//  * the diagonal from per-row constants and popcounts of packed words.
template <class Pol, int R, int NT = kRowThreads, int MINB = 2>
__global__ void __launch_bounds__(NT, MINB)
    k_row5(P3 p, const long long* __restrict__ grp_start, long long n_groups, const typename Pol::S* __restrict__ x,
           typename Pol::Y* __restrict__ y, const int* __restrict__ emax, long long stage_elems, int* err) {
  using S = typename Pol::S;
  extern __shared__ __align__(16) unsigned char smem5[];
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem5);
  S* bufs = reinterpret_cast<S*>(smem5 + 128);
  __shared__ const S* src_row[R][32];  // per row, per A cross site
  // per row, B cross site, value beta of the column's bit at that site and
  // value class (of at most two): the site's bonds that are valid there
  // (their A bit differs from beta), as source-row lists of at most kXL
  // entries; a column sums each class's gathers and multiplies once
  constexpr int kXL = 2;
  __shared__ const S* xl_ptr[R][32][2][2][kXL];
  __shared__ unsigned char xl_n[R][32][2][2];
  __shared__ int xl_mx[32][2];  // per B cross site and class: longest list over rows and beta
  constexpr bool kLists = sizeof(S) == 8 || kListsF32;
  __shared__ int s_pad[R];
  constexpr int V = 16 / (int)sizeof(S);
  const Dev3& t = p.t;
  if (threadIdx.x == 0) {
    bar_init(&bar[0]);
    bar_fence_init();
  }
  __syncthreads();
  const int e2 = emax ? out_exp(t, emax) : 0;
  unsigned phase = 0;
  for (long long g = blockIdx.x; g < n_groups; g += gridDim.x) {
    const int bi = find_blk(grp_start, p.nblk, g);
    const DevBlock bl = p.blocks[bi];
    const long long a0 = (g - grp_start[bi]) * R;
    const int nr = (int)min((long long)R, bl.dA - a0);
    const int dB = (int)bl.dB;
    if (threadIdx.x == 0) {
      proxy_fence();
      unsigned bytes = 0;
      for (int r = 0; r < nr; ++r) {
        const long long g0 = bl.off + (a0 + r) * dB;
        const long long gal = (g0 + V - 1) / V * V, galend = (g0 + dB) / V * V;
        if (galend > gal) bytes += (unsigned)((galend - gal) * (long long)sizeof(S));
      }
      if (bytes) {
        bar_expect(&bar[0], bytes);
        for (int r = 0; r < nr; ++r) {
          const long long g0 = bl.off + (a0 + r) * dB;
          const long long gal = (g0 + V - 1) / V * V, galend = (g0 + dB) / V * V;
          if (galend > gal)
            bulk_g2s(bufs + r * stage_elems + (g0 % V) + (gal - g0), x + gal,
                     (unsigned)((galend - gal) * (long long)sizeof(S)), &bar[0]);
        }
      } else {
        bar_arrive(&bar[0]);
      }
    }
    for (int r = 0; r < nr; ++r) {
      const long long g0 = bl.off + (a0 + r) * dB;
      const long long gend = g0 + dB;
      const long long gal = (g0 + V - 1) / V * V, galend = gend / V * V;
      const int pad = (int)(g0 % V);
      S* buf = bufs + r * stage_elems;
      if (threadIdx.x == 0) {
        s_pad[r] = pad;
        buf[pad + dB] = (S)0;  // zero slot addressed by the padding indices
      }
      if (galend > gal) {
        for (long long q = g0 + threadIdx.x; q < gal; q += blockDim.x) buf[pad + (q - g0)] = x[q];
        for (long long q = galend + threadIdx.x; q < gend; q += blockDim.x) buf[pad + (q - g0)] = x[q];
      } else {
        for (long long q = g0 + threadIdx.x; q < gend; q += blockDim.x) buf[pad + (q - g0)] = x[q];
      }
    }
    // neighbouring-block source row of each (row, A cross site)
    if (threadIdx.x < 32 * R) {
      const int r = threadIdx.x >> 5, ia = threadIdx.x & 31;
      const S* sp = nullptr;
      if (r < nr && ia < 32 && p.ncross) {
        const long long gA = bl.gA0 + a0 + r;
        // which bond touches site ia: any bond k with bond_ia[k] == ia gives its A bit
        int k = -1;
        for (int q = 0; q < p.ncross; ++q)
          if (t.bond_ia[q] == ia) { k = q; break; }
        if (k >= 0) {
          const unsigned pa = t.A_pack[gA];
          const int sb = ((pa >> k) & 1u) ? bl.nbr_lo : bl.nbr_hi;
          if (sb >= 0) {
            const DevBlock so = p.blocks[sb];
            const unsigned rr = t.mapA[(long long)ia * t.A_total + gA];
            if (rr != 0xFFFFu) sp = x + so.off + (long long)rr * so.dB;
          }
        }
      }
      src_row[r][ia] = sp;
    }
    if (kLists && p.ncross && t.xl_ok) {
      __syncthreads();  // src_row complete
      if (threadIdx.x < 64) xl_mx[threadIdx.x >> 1][threadIdx.x & 1] = 0;
      __syncthreads();
      if (threadIdx.x < R * 64) {
        const int r = threadIdx.x >> 6, ib = (threadIdx.x >> 1) & 31, beta = threadIdx.x & 1;
        int n0 = 0, n1 = 0;
        if (ib < t.n_ib && r < nr) {
          const unsigned par = t.A_pack[bl.gA0 + a0 + r];
          unsigned km = t.ib_mask[ib];
          while (km) {
            const int k = __ffs(km) - 1;
            km &= km - 1;
            const S* sp = src_row[r][t.bond_ia[k]];
            if ((((par >> k) & 1u) != (unsigned)beta) && sp) {  // at most kXL per class (xl_ok)
              if ((t.xl_c1_mask >> k) & 1u) {
                if (n1 < kXL) xl_ptr[r][ib][beta][1][n1++] = sp;
              } else {
                if (n0 < kXL) xl_ptr[r][ib][beta][0][n0++] = sp;
              }
            }
          }
        }
        xl_n[r][ib][beta][0] = (unsigned char)n0;
        xl_n[r][ib][beta][1] = (unsigned char)n1;
        atomicMax(&xl_mx[ib][0], n0);
        atomicMax(&xl_mx[ib][1], n1);
      }
    }
    const bool ok = bar_wait(&bar[0], phase);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicExch(err, 1);
      bar_wait(&bar[0], phase);
      return;
    }
    phase ^= 1;
    unsigned pa[R];
    const S* xs[R];
    typename Pol::D da[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int rr = r < nr ? r : 0;
      const long long gA = bl.gA0 + a0 + rr;
      pa[r] = t.A_pack[gA];
      xs[r] = bufs + rr * stage_elems + s_pad[rr];
      da[r] = Pol::diagA(t, gA);
    }
    const bool final_ = !bl.has_hA && !p.keep_fixed;
    const long long gB0 = bl.gB0;
    for (int b = threadIdx.x; b < dB; b += blockDim.x) {
      const long long gB = gB0 + b;
      const uint2 m = t.B_meta4[gB];
      const unsigned pb = t.B_pack[gB];
      const typename Pol::D dbv = Pol::diagB(t, gB);
      typename Pol::A acc[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const unsigned z = t.vab_and ? (pa[r] & pb) : (pa[r] ^ pb);
        acc[r] = Pol::dmul(da[r] + dbv + Pol::vab(t, z), xs[r][b]);
      }
      const uint2* cp = t.B_col4 + m.x;
      // index groups in flight per class step (measured best: 4 for 8-byte
      // types, 2 for 4-byte types, whose four rows per pass need registers)
      constexpr int HBU = sizeof(S) == 8 ? 4 : 2;
      const unsigned zz = (unsigned)dB | ((unsigned)dB << 16);  // four zero-slot indices
#pragma unroll
      for (int c = 0; c < kMaxCls; ++c) {
        const unsigned n4 = (m.y >> (8 * c)) & 255u;
        if (!n4) continue;
        S sum[R];
#pragma unroll
        for (int r = 0; r < R; ++r) sum[r] = 0;
        // HBU index groups are loaded before any is used, so their L2
        // latencies overlap; groups past the class end read the zero slot
        for (unsigned i = 0; i < n4; i += HBU) {
          uint2 q[HBU];
#pragma unroll
          for (int u = 0; u < HBU; ++u) q[u] = i + u < n4 ? __ldg(cp + i + u) : make_uint2(zz, zz);
#pragma unroll
          for (int u = 0; u < HBU; ++u) {
            const unsigned i0 = q[u].x & 0xFFFFu, i1 = q[u].x >> 16, i2 = q[u].y & 0xFFFFu, i3 = q[u].y >> 16;
#pragma unroll
            for (int r = 0; r < R; ++r) sum[r] += (xs[r][i0] + xs[r][i1]) + (xs[r][i2] + xs[r][i3]);
          }
        }
        cp += n4;
        const typename Pol::W wc = Pol::w(t, c);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] += Pol::wmul(wc, sum[r]);
      }
      if (p.ncross) {
        unsigned dr[R];
#pragma unroll
        for (int r = 0; r < R; ++r) dr[r] = r < nr ? (pa[r] ^ pb) : 0u;
        if (kLists && t.xl_ok) {
          // per B cross site, the column's bit there picks each row's lists of
          // valid bonds (one per value class); the gathers of all rows' lists are
          // issued before any is summed (invalid slots read nothing and add zero),
          // the next site's map entry is loaded one site ahead, and each class's
          // sum is multiplied by its weight once per column
          unsigned mq_next = t.n_ib > 0 ? __ldg(t.mapB + gB) : 0u;
          S s0[R], s1[R];
#pragma unroll
          for (int r = 0; r < R; ++r) s0[r] = s1[r] = 0;
          for (int ib = 0; ib < t.n_ib; ++ib) {
            const unsigned mq = mq_next;
            if (ib + 1 < t.n_ib) mq_next = __ldg(t.mapB + (long long)(ib + 1) * t.B_total + gB);
            const int mx0 = xl_mx[ib][0], mx1 = xl_mx[ib][1];
            if (!(mx0 | mx1)) continue;
            const int beta = (int)((pb >> (__ffs(t.ib_mask[ib]) - 1)) & 1u);
            int n0[R], n1[R];
            S v0[R][kXL], v1[R][kXL];
#pragma unroll
            for (int r = 0; r < R; ++r) {
              n0[r] = xl_n[r][ib][beta][0];
              n1[r] = xl_n[r][ib][beta][1];
            }
#pragma unroll
            for (int i = 0; i < kXL; ++i) {
#pragma unroll
              for (int r = 0; r < R; ++r) {
                v0[r][i] = (i < mx0 && i < n0[r]) ? __ldg(xl_ptr[r][ib][beta][0][i] + mq) : (S)0;
                v1[r][i] = (i < mx1 && i < n1[r]) ? __ldg(xl_ptr[r][ib][beta][1][i] + mq) : (S)0;
              }
            }
#pragma unroll
            for (int i = 0; i < kXL; ++i)
#pragma unroll
              for (int r = 0; r < R; ++r) {
                s0[r] += v0[r][i];
                s1[r] += v1[r][i];
              }
          }
          {
            const typename Pol::W w0 = Pol::w(t, t.xl_c[0]), w1 = Pol::w(t, t.xl_c[1]);
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] += Pol::wmul(w0, s0[r]) + Pol::wmul(w1, s1[r]);
          }
        } else if constexpr (sizeof(S) == 4) {
          // 4-byte types (four rows per pass): loop over every bond with
          // warp-uniform table indices (B site, bond, weight); only the
          // validity predicate and the gather address vary across lanes
          unsigned mq_next = t.n_ib > 0 ? __ldg(t.mapB + gB) : 0u;  // map entries one site ahead
          for (int ib = 0; ib < t.n_ib; ++ib) {
            const unsigned mq = mq_next;
            if (ib + 1 < t.n_ib) mq_next = __ldg(t.mapB + (long long)(ib + 1) * t.B_total + gB);
            unsigned km = t.ib_mask[ib];
            while (km) {
              const int k = __ffs(km) - 1;
              km &= km - 1;
              const typename Pol::W wk = Pol::bw(t, k);
              const int ia = t.bond_ia[k];
#pragma unroll
              for (int r = 0; r < R; ++r) {
                const S* sp = src_row[r][ia];
                if (((dr[r] >> k) & 1u) && sp) acc[r] += Pol::wmul(wk, __ldg(sp + mq));
              }
            }
          }
        } else {
          // 8-byte types with more than kXL bonds at some B cross site: the
          // gathers of a site's first kXB bonds (warp-uniform bond indices)
          // for both rows are issued before any is summed; bonds beyond kXB
          // take a plain loop
          constexpr int kXB = 4;
          unsigned mq_next = t.n_ib > 0 ? __ldg(t.mapB + gB) : 0u;
          for (int ib = 0; ib < t.n_ib; ++ib) {
            const unsigned mq = mq_next;
            if (ib + 1 < t.n_ib) mq_next = __ldg(t.mapB + (long long)(ib + 1) * t.B_total + gB);
            unsigned rm = t.ib_mask[ib];
            int kq[kXB];
#pragma unroll
            for (int q = 0; q < kXB; ++q) {
              kq[q] = rm ? __ffs(rm) - 1 : -1;
              rm &= rm - 1;
            }
            S v[R][kXB];
#pragma unroll
            for (int q = 0; q < kXB; ++q)
#pragma unroll
              for (int r = 0; r < R; ++r) {
                v[r][q] = 0;
                if (kq[q] >= 0 && ((dr[r] >> kq[q]) & 1u)) {
                  const S* sp = src_row[r][t.bond_ia[kq[q]]];
                  if (sp) v[r][q] = __ldg(sp + mq);
                }
              }
#pragma unroll
            for (int q = 0; q < kXB; ++q)
              if (kq[q] >= 0) {
                const typename Pol::W w = Pol::bw(t, kq[q]);
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] += Pol::wmul(w, v[r][q]);
              }
            while (rm) {
              const int k = __ffs(rm) - 1;
              rm &= rm - 1;
#pragma unroll
              for (int r = 0; r < R; ++r) {
                const S* sp = src_row[r][t.bond_ia[k]];
                if (((dr[r] >> k) & 1u) && sp) acc[r] += Pol::wmul(Pol::bw(t, k), __ldg(sp + mq));
              }
            }
          }
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (r < nr) store_out<Pol>(y, bl.off + (a0 + r) * dB + b, acc[r], final_, e2);
    }
    __syncthreads();
  }
}

// 32 x NC zeros read by k_panel4 in place of missing neighbour rows
static __device__ __align__(16) long long g_zero_row[256];

// H_A panel pass with U neighbour rows in flight per class step: each warp
// owns one output row of a 256-column panel, processed as sub-panels of
// 32 * NC columns; the column indices of U consecutive H_A entries are read
// first (warp-uniform), then all U x NC neighbour values are loaded before
// any is summed, so U x NC independent loads per lane overlap their
// latency instead of one neighbour row at a time.  Full sub-panels need no
// per-column checks, and entries past a class's end read the zero row, so
// their loads carry no predicates.
template <class Pol, int NC, int U>
__global__ void __launch_bounds__(256) k_panel4(P3 p, const int4* __restrict__ items, long long n_items,
                                                const typename Pol::S* __restrict__ x, typename Pol::Y* __restrict__ y,
                                                const int* __restrict__ emax) {
  using S = typename Pol::S;
  constexpr int W = 32 * NC;
  static_assert(256 % W == 0, "sub-panels must tile the 256-column panel");
  const Dev3& t = p.t;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e2 = emax ? out_exp(t, emax) : 0;
  for (long long w = blockIdx.x; w < n_items; w += gridDim.x) {
    const int4 it = items[w];
    if (warp >= it.w) continue;
    const DevBlock bl = p.blocks[it.x];
    const long long a = it.z + warp;
    const long long gA = bl.gA0 + a;
    const long long dB = bl.dB;
    const S* xb = x + bl.off;
    typename Pol::Y* yrow = y + bl.off + a * dB;
    const uint2 m = t.A_meta[gA];
    for (int sp = 0; sp < 256; sp += W) {
      const long long b0 = it.y + sp + lane;
      if (it.y + sp >= dB) break;
      const bool full = it.y + sp + W <= dB;
      const S* xb0 = xb + b0;                                              // column b0 of row 0
      const S* zr = reinterpret_cast<const S*>(g_zero_row) + lane;         // zeros at +32c
      typename Pol::A acc[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const long long b = b0 + 32 * c;
        acc[c] = typename Pol::A(b < dB ? yrow[b] : (typename Pol::Y)0);
      }
      unsigned e = m.x;
#pragma unroll
      for (int cl = 0; cl < kMaxCls; ++cl) {
        const int n = (int)((m.y >> (8 * cl)) & 255u);
        if (!n) continue;
        S sum[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) sum[c] = 0;
        if (full) {
          // full sub-panel: no per-column checks; entries past the class end
          // read a zero row
          for (int i0 = 0; i0 < n; i0 += U) {
            const S* rp[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
              rp[u] = i0 + u < n ? xb0 + (long long)t.A_col[e + i0 + u] * dB : zr;
            S v[U][NC];
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
              for (int c = 0; c < NC; ++c) v[u][c] = __ldg(rp[u] + 32 * c);
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
              for (int c = 0; c < NC; ++c) sum[c] += v[u][c];
          }
        } else {
        for (int i0 = 0; i0 < n; i0 += U) {
          long long rowoff[U];
#pragma unroll
          for (int u = 0; u < U; ++u) rowoff[u] = i0 + u < n ? (long long)t.A_col[e + i0 + u] * dB : -1;
          S v[U][NC];
#pragma unroll
          for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
              const long long b = b0 + 32 * c;
              v[u][c] = (rowoff[u] >= 0 && b < dB) ? __ldg(xb + rowoff[u] + b) : (S)0;
            }
#pragma unroll
          for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < NC; ++c) sum[c] += v[u][c];
        }
        }
        e += n;
        const typename Pol::W wc = Pol::w(t, cl);
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] += Pol::wmul(wc, sum[c]);
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const long long b = b0 + 32 * c;
        if (b < dB) store_out<Pol>(yrow, b, acc[c], true, e2);
      }
    }
  }
}


static P3 make_p3(const ed_ctx* c) {
  P3 p;
  p.t = c->t3;
  p.blocks = c->d_blocks;
  p.cross = c->d_cross;
  p.row_start = c->d_row_start;
  p.nblk = (int)c->blocks.size();
  p.ncross = c->kind == ED_SPIN ? (int)c->cross.size() : 0;
  p.n_rows = c->n_rows;
  p.keep_fixed = 0;
  return p;
}

// Row-pass shapes: one 1024-thread CTA per SM whose staged rows fill the
// shared memory and share the B-side index and map loads: four rows per
// pass for 4-byte types, two for 8-byte types.  On the J1-J2 4x8 workload
// this measured 15.7 ms (FP32) and 35.3 ms (FP64) against 23.3 and 40.9 ms
// for two (FP32) or one (FP64) row per pass in two 512-thread CTAs per SM
// (kRow4Quad / kRow8Pair = false).
constexpr bool kRow8Pair = true;
constexpr bool kRow4Quad = true;
static int rows_per_pass(size_t es) { return es == 4 ? (kRow4Quad ? 4 : 2) : (kRow8Pair ? 2 : 1); }

static size_t v3_smem(const ed_ctx* c, size_t es, long long* stage_elems) {
  long long mdb = 1;
  for (const auto& b : c->blocks) mdb = std::max<long long>(mdb, b.dB);
  *stage_elems = ((mdb + 1 + 16 / (long long)es + 15) / 16) * 16;  // row, zero slot, alignment pad
  return 128 + (size_t)rows_per_pass(es) * (size_t)(*stage_elems) * es;
}

bool v3_usable(const ed_ctx* c, ed_dtype dt, const void* x) {
  if (!c->v3_ok || ((uintptr_t)x % 16) != 0) return false;
  long long se;
  const size_t es = dt == ED_F64 ? 8 : 4;
  const bool one_cta = (es == 8 && kRow8Pair) || (es == 4 && kRow4Quad);
  return v3_smem(c, es, &se) <= (one_cta ? 220 : 110) * 1024;
}

// events bracketing the stages of one apply when profiling is on
struct ProfMarks {
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  bool on = false;
  void begin(ed_ctx* c) {
    on = c->prof;
    if (!on) return;
    for (auto& e : ev) cudaEventCreate(&e);
  }
  void mark(int i, cudaStream_t st) {
    if (on) cudaEventRecord(ev[i], st);
  }
  void end(ed_ctx* c) {
    if (!on) return;
    for (auto& e : ev) c->prof_ev.push_back(e);
  }
};

template <class Pol>
static ed_status run_v3(ed_ctx* c, const typename Pol::S* x, typename Pol::Y* y, const int* emax, cudaStream_t st,
                        ProfMarks& pm) {
  P3 p = make_p3(c);
  if (p.n_rows == 0) return ED_OK;
  long long se;
  constexpr bool pair8 = sizeof(typename Pol::S) == 8 && kRow8Pair;
  constexpr bool quad4 = sizeof(typename Pol::S) == 4 && kRow4Quad;
  constexpr int R = quad4 ? 4 : (sizeof(typename Pol::S) == 4 || pair8) ? 2 : 1;
  constexpr int NT = (pair8 || quad4) ? 1024 : kRowThreads;
  constexpr int CPS = (pair8 || quad4) ? 1 : 2;  // CTAs per SM
  const size_t smem = v3_smem(c, sizeof(typename Pol::S), &se);
  const int sms = n_sms(c->device);
  pm.mark(2, st);
  {
    auto kern = k_row5<Pol, R, NT, CPS>;
    ED_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long* gs = R == 4 ? c->d_grp4_start : R == 2 ? c->d_grp2_start : c->d_row_start;
    const long long ng = R == 4 ? c->n_grp4 : R == 2 ? c->n_grp2 : c->n_rows;
    const long long grid = std::min<long long>(ng, (long long)sms * CPS);
    kern<<<(unsigned)grid, NT, smem, st>>>(p, gs, ng, x, y, emax, se, c->d_err);
  }
  ED_CUDA_TRY(cudaGetLastError());
  pm.mark(3, st);
  if (c->n_panel_items > 0) {
    const long long g2 = std::min<long long>(c->n_panel_items, (long long)sms * 8);
    // measured on the 4x8 J1-J2 and 4x4 Hubbard workloads: 8-byte types
    // gain from four neighbour rows in flight on 128-column sub-panels
    // (one row at a time: 24.5 / 5.1 ms; four: 9.9 / 2.0 ms), FP32 from two
    // rows in flight on full 256-column panels (6.2 -> 5.4 ms on J1-J2 4x8)
    if constexpr (sizeof(typename Pol::S) == 4)
      k_panel4<Pol, 8, 2><<<(unsigned)g2, 256, 0, st>>>(p, c->d_panel_items, c->n_panel_items, x, y, emax);
    else
      k_panel4<Pol, 4, 4><<<(unsigned)g2, 256, 0, st>>>(p, c->d_panel_items, c->n_panel_items, x, y, emax);
    ED_CUDA_TRY(cudaGetLastError());
  }
  return ED_OK;
}

// exact fixed-point FP64 apply with explicit scratch: `fixed` holds D
// 64-bit integers, `emax` one int (cleared here before use)
// y += V x in FP64 after the integer passes of a split diagonal: per
// element the side diagonals, the constant and the weighted popcounts of
// the packed cut words (PF64::diag), one CTA per row, grid-stride
__global__ void __launch_bounds__(256) k_diag_add(P3 p, const double* __restrict__ x, double* __restrict__ y) {
  const Dev3& t = p.t;
  for (long long r = blockIdx.x; r < p.n_rows; r += gridDim.x) {
    const int bi = find_blk(p.row_start, p.nblk, r);
    const DevBlock bl = p.blocks[bi];
    const long long a = r - p.row_start[bi];
    const long long gA = bl.gA0 + a;
    const unsigned pa = t.A_pack[gA];
    const long long base = bl.off + a * bl.dB;
    for (long long b = threadIdx.x; b < bl.dB; b += blockDim.x) {
      const long long gB = bl.gB0 + b;
      const unsigned pb = t.B_pack[gB];
      const unsigned z = t.vab_and ? (pa & pb) : (pa ^ pb);
      y[base + b] = fma(PF64::diag(t, gA, gB, z), x[base + b], y[base + b]);
    }
  }
}

static ed_status diag_add(ed_ctx* c, const double* x, double* y, cudaStream_t st) {
  if (!c->diag_split || c->n_rows < 1) return ED_OK;
  const long long g = std::min<long long>(c->n_rows, (long long)n_sms(c->device) * 16);
  k_diag_add<<<(unsigned)g, 256, 0, st>>>(make_p3(c), x, y);
  ED_CUDA_TRY(cudaGetLastError());
  return ED_OK;
}

static ed_status apply_fixed(ed_ctx* c, const double* x, double* y, long long* fixed, int* emax, cudaStream_t st,
                             ProfMarks& pm) {
  const long long n = c->D;
  ED_CUDA_TRY(cudaMemsetAsync(emax, 0, sizeof(int), st));
  const int sms = n_sms(c->device);
  const long long g = std::min<long long>((n + 255) / 256, (long long)sms * 8);
  pm.mark(0, st);
  k_exp_max<<<(unsigned)std::max<long long>(g, 1), 256, 0, st>>>(x, n, emax);
  pm.mark(1, st);
  k_to_fixed<<<(unsigned)std::max<long long>(g, 1), 256, 0, st>>>(x, fixed, n, emax, c->t3.P);
  ED_CUDA_TRY(cudaGetLastError());
  if (c->dyadic) {
    ED_TRY(run_v3<PI64>(c, fixed, (long long*)y, emax, st, pm));
    return diag_add(c, x, y, st);
  }
  return c->wide ? run_v3<PW>(c, fixed, y, emax, st, pm) : run_v3<PC64>(c, fixed, y, emax, st, pm);
}

// fixed-point input: exact integer sums, with small integer weights (dyadic
// couplings), with 64-bit integer weights into 128-bit sums (other couplings)
// or, when their range is too wide for that, with FP64 weights per value class
static bool fixed_mode(const ed_ctx* c) { return c->dyadic || c->classed; }

bool fixed_path(const ed_ctx* c, const void* x) { return fixed_mode(c) && v3_usable(c, ED_F64, x); }

ed_status apply_prepared_fixed(ed_ctx* c, const double* x, double* y, cudaStream_t st) {
  if (!c->d_fixed) {
    set_error("fixed-point input was not prepared");
    return ED_EINVAL;
  }
  ProfMarks pm;
  pm.begin(c);
  pm.mark(0, st);
  pm.mark(1, st);
  ed_status r;
  if (c->dyadic) {
    r = run_v3<PI64>(c, c->d_fixed, (long long*)y, c->d_exp, st, pm);
    if (r == ED_OK) r = diag_add(c, x, y, st);
  } else {
    r = c->wide ? run_v3<PW>(c, c->d_fixed, y, c->d_exp, st, pm) : run_v3<PC64>(c, c->d_fixed, y, c->d_exp, st, pm);
  }
  pm.mark(4, st);
  pm.end(c);
  return r;
}

ed_status apply_v3(ed_ctx* c, const void* x, void* y, ed_dtype dt, cudaStream_t st) {
  ProfMarks pm;
  pm.begin(c);
  ed_status r;
  if (dt == ED_F32 || !fixed_mode(c)) {
    pm.mark(0, st);
    pm.mark(1, st);
    r = dt == ED_F32 ? run_v3<PF32>(c, (const float*)x, (float*)y, nullptr, st, pm)
                     : run_v3<PF64>(c, (const double*)x, (double*)y, nullptr, st, pm);
  } else {
    // exact fixed point: exponent of max|x|, scaled copy, integer passes
    if (!c->d_fixed) ED_TRY(dev_alloc(c, (void**)&c->d_fixed, (size_t)std::max<long long>(c->D, 2) * 8));
    r = apply_fixed(c, (const double*)x, (double*)y, c->d_fixed, c->d_exp, st, pm);
  }
  pm.mark(4, st);
  pm.end(c);
  return r;
}

// ---------------------------------------------------------------- apply without allocation

// Scratch of ed_apply_H_noalloc: a file-scope device array (one int for the
// exponent of max|x|, then the 64-bit fixed-point copy of x).  Every GPU
// that loads this library holds it until the process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;
constexpr size_t kNoAllocHeader = 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// device address of the scratch on the current device; the first call on a
// device looks it up (cudaGetSymbolAddress) and caches it
static ed_status noalloc_scratch(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    set_error("device %d outside the %d devices the scratch table covers", dev, kNoAllocMaxDevices);
    return ED_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      set_error("cudaGetSymbolAddress of the static scratch failed on device %d: %s", dev, cudaGetErrorString(e));
      return ED_ECUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = (unsigned char*)g_noalloc_ptr[dev];
  return ED_OK;
}

}  // namespace edk

using namespace edk;

extern "C" ed_status ed_apply_H_noalloc(ed_ctx* c, const void* x, void* y, void* stream) {
  if (!c) { set_error("ctx is NULL"); return ED_EINVAL; }
  if (!c->ops_built) { set_error("ed_build_local_ops has not been called"); return ED_EINVAL; }
  if (c->D > 0 && (!x || !y)) { set_error("x or y is NULL"); return ED_EINVAL; }
  const size_t need = kNoAllocHeader + (size_t)c->D * sizeof(long long);
  if (fixed_mode(c) && need > kNoAllocScratchBytes) {
    set_error("ed_apply_H_noalloc: %lld states need %zu bytes of scratch, the static scratch holds %zu "
              "(at most %zu states)", (long long)c->D, need, kNoAllocScratchBytes,
              (kNoAllocScratchBytes - kNoAllocHeader) / sizeof(long long));
    return ED_EINVAL;
  }
  const char* xb = (const char*)x;
  const char* yb = (const char*)y;
  if (c->D > 0 && xb < yb + c->D * 8 && yb < xb + c->D * 8) { set_error("x and y overlap"); return ED_EINVAL; }
  if (!v3_usable(c, ED_F64, x)) {
    set_error("ed_apply_H_noalloc needs the class-sorted kernels (16-byte aligned x, at most 4 value classes, "
              "32 cross bonds and 65534 states per side charge)");
    return ED_EUNSUPPORTED;
  }
  ED_DEVICE_SCOPE(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  ProfMarks pm;  // no profiling events here
  if (!fixed_mode(c)) return run_v3<PF64>(c, (const double*)x, (double*)y, nullptr, st, pm);
  unsigned char* base = nullptr;
  ED_TRY(noalloc_scratch(c->device, &base));
  return apply_fixed(c, (const double*)x, (double*)y, (long long*)(base + kNoAllocHeader), (int*)base, st, pm);
}



extern "C" int ed_row_pass(const ed_ctx* c, ed_dtype dt) {
  if (!c || !c->ops_built) return -1;
  if (!v3_usable(c, dt, (const void*)(uintptr_t)256)) return 0;  // any 16-byte aligned x
  return 1;
}

extern "C" int ed_fp64_mode(const ed_ctx* c) {
  if (!c || !c->ops_built) return -1;
  if (c->dyadic) return 1;
  if (c->classed) return c->wide ? 2 : 3;
  return 0;
}

extern "C" ed_status ed_profile_enable(ed_ctx* c, int enable) {
  if (!c) { set_error("ctx is NULL"); return ED_EINVAL; }
  c->prof = enable != 0;
  return ED_OK;
}

extern "C" ed_status ed_profile_read(ed_ctx* c, double* ms, int64_t* count, int reset) {
  if (!c) { set_error("ctx is NULL"); return ED_EINVAL; }
  for (size_t i = 0; i + 5 <= c->prof_ev.size(); i += 5) {
    cudaEvent_t* e = &c->prof_ev[i];
    ED_CUDA_TRY(cudaEventSynchronize(e[4]));
    for (int k = 0; k < 4; ++k) {
      float t = 0.f;
      ED_CUDA_TRY(cudaEventElapsedTime(&t, e[k], e[k + 1]));
      c->prof_ms[k] += t;
    }
    ++c->prof_count;
    for (int k = 0; k < 5; ++k) cudaEventDestroy(e[k]);
  }
  c->prof_ev.clear();
  if (ms)
    for (int k = 0; k < 4; ++k) ms[k] = c->prof_ms[k];
  if (count) *count = c->prof_count;
  if (reset) {
    for (double& v : c->prof_ms) v = 0.0;
    c->prof_count = 0;
  }
  return ED_OK;
}
