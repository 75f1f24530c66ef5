// Dense-block bipartite H|psi>: the operator of paper Eq. (2),
//   H = sum_q H_L,q (x) 1 + 1 (x) H_R,q + sum_m L_m (x) R_m,
// with dense side operators on symmetry blocks (the paper's DMRG setting,
// block dimensions chi_q).  A state is the concatenation of row-major blocks
// Psi_q (chi_q x chi_q); by the Vec identity each term is a product of dense
// matrices:
//   Y_q  = H_L,q Psi_q + Psi_q H_R,q^T
//   Y_q' += L_m,q Psi_q R_m,q^T,  q' = q + delta_m.
// Every product runs in k_gemm_batch: FP64, one 64 x 64 output tile per CTA,
// 64 x 16 operand slabs staged in shared memory, 4 x 4 outputs per thread,
// all problems of one stage (all blocks q) in one launch.
#include <cstring>
#include <new>
#include <vector>

#include "krylov.h"

namespace edk {
namespace {

constexpr int kDT = 64;  // output tile
constexpr int kDK = 16;  // contraction depth per step

// C (M x N, leading dimension ldc) = or += A B with A(i,k) = A[i*sai + k*sak]
// and B(k,j) = B[k*sbk + j*sbj].  An operand is an absolute device address
// (operators, scratch) or an offset into the x or y of the call, so the
// problem lists are built once and stay on the device.
enum { kAbs = 0, kX = 1, kY = 2 };
struct GemmProblem {
  const double* A;
  const double* B;
  double* C;
  long long aoff, boff, coff;
  int abase, bbase, cbase;
  long long sai, sak, sbk, sbj, ldc;
  int M, N, K;
  int acc;         // 1: C += A B, 0: C = A B
  int tiles_n;     // output tiles along N
  long long tile0; // first tile of this problem in the launch
};

__device__ __forceinline__ const double* resolve(const double* p, long long off, int base, const double* x,
                                                 const double* y) {
  return base == kX ? x + off : base == kY ? y + off : p;
}

__global__ void __launch_bounds__(256) k_gemm_batch(const GemmProblem* __restrict__ probs, int nprob,
                                                    const double* __restrict__ x, double* y) {
  __shared__ double As[kDK][kDT + 1];
  __shared__ double Bs[kDK][kDT + 1];
  // problem of this tile (tile0 ascending)
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (probs[mid].tile0 <= (long long)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const GemmProblem P = probs[lo];
  const double* Ap = resolve(P.A, P.aoff, P.abase, x, y);
  const double* Bp = resolve(P.B, P.boff, P.bbase, x, y);
  double* Cp = const_cast<double*>(resolve(P.C, P.coff, P.cbase, x, y));
  const long long t = (long long)blockIdx.x - P.tile0;
  const long long i0 = (t / P.tiles_n) * kDT, j0 = (t % P.tiles_n) * kDT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
  for (int k0 = 0; k0 < P.K; k0 += kDK) {
    // A slab (64 rows x 16 k) and B slab (16 k x 64 columns); the faster
    // index of each follows its contiguous direction
    for (int e = threadIdx.x; e < kDT * kDK; e += blockDim.x) {
      {
        const bool kfast = P.sak == 1;
        const int r = kfast ? e / kDK : e % kDT;
        const int k = kfast ? e % kDK : e / kDT;
        const long long gi = i0 + r, gk = k0 + k;
        As[k][r] = (gi < P.M && gk < P.K) ? Ap[gi * P.sai + gk * P.sak] : 0.0;
      }
      {
        const bool jfast = P.sbj == 1;
        const int c = jfast ? e % kDT : e / kDK;
        const int k = jfast ? e / kDT : e % kDK;
        const long long gj = j0 + c, gk = k0 + k;
        Bs[k][c] = (gj < P.N && gk < P.K) ? Bp[gk * P.sbk + gj * P.sbj] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kDK; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[k][ty + 16 * u];
        b[u] = Bs[k][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const long long i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
      if (i < P.M && j < P.N) {
        double* c = Cp + i * P.ldc + j;
        *c = P.acc ? *c + acc[u][v] : acc[u][v];
      }
    }
}

}  // namespace
}  // namespace edk

using namespace edk;

struct ed_dense {
  int device = 0;
  int nq = 0;
  std::vector<int64_t> chi, off;
  int64_t D = 0;
  struct Term {
    int delta;
    std::vector<const double*> L, R;  // device, per source block q (nullptr: none)
    std::vector<int64_t> toff;        // scratch offset of L Psi_q per q
  };
  std::vector<const double*> HL, HR;  // device, per block
  std::vector<Term> terms;
  double* scratch = nullptr;
  std::vector<void*> allocs;
  // problem lists of the stages (device) and their tile counts
  GemmProblem* d_probs = nullptr;
  struct Stage {
    int first, count;
    long long tiles;
  };
  std::vector<Stage> stages;
  ~ed_dense() {
    for (void* p : allocs) cudaFree(p);
  }
};

namespace {

ed_status dense_alloc(ed_dense* d, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes < 16 ? 16 : bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc(%zu) for the dense-block operator failed: %s", bytes, cudaGetErrorString(e));
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? ED_ENOMEM : ED_ECUDA;
  }
  d->allocs.push_back(*p);
  return ED_OK;
}

ed_status upload(ed_dense* d, const double* h, size_t n, const double** out) {
  double* p = nullptr;
  ED_TRY(dense_alloc(d, (void**)&p, n * sizeof(double)));
  ED_CUDA_TRY(cudaMemcpy(p, h, n * sizeof(double), cudaMemcpyHostToDevice));
  *out = p;
  return ED_OK;
}

struct Opnd {
  const double* p;
  long long off;
  int base;
};
Opnd abs_(const double* p) { return {p, 0, kAbs}; }
Opnd xo(long long off) { return {nullptr, off, kX}; }
Opnd yo(long long off) { return {nullptr, off, kY}; }

GemmProblem problem(Opnd A, long long sai, long long sak, Opnd B, long long sbk, long long sbj, Opnd C, long long ldc,
                    int M, int N, int K, int acc) {
  GemmProblem p;
  p.A = A.p;
  p.B = B.p;
  p.C = const_cast<double*>(C.p);
  p.aoff = A.off;
  p.boff = B.off;
  p.coff = C.off;
  p.abase = A.base;
  p.bbase = B.base;
  p.cbase = C.base;
  p.sai = sai;
  p.sak = sak;
  p.sbk = sbk;
  p.sbj = sbj;
  p.ldc = ldc;
  p.M = M;
  p.N = N;
  p.K = K;
  p.acc = acc;
  p.tiles_n = (N + kDT - 1) / kDT;
  p.tile0 = 0;
  return p;
}

}  // namespace

extern "C" ed_status ed_dense_create(int nq, const int64_t* chi, const double* const* HL, const double* const* HR,
                                     int n_terms, const int* delta, const double* const* Lm,
                                     const double* const* Rm, ed_dense** out) {
  if (!out) { set_error("out is NULL"); return ED_EINVAL; }
  *out = nullptr;
  if (nq < 1 || !chi || !HL || !HR || n_terms < 0 || (n_terms > 0 && (!delta || !Lm || !Rm))) {
    set_error("bad dense-block arguments");
    return ED_EINVAL;
  }
  for (int q = 0; q < nq; ++q)
    if (chi[q] < 1 || chi[q] > (1 << 20) || !HL[q] || !HR[q]) {
      set_error("block %d: dimension %lld outside 1..2^20 or a side operator is NULL", q, (long long)chi[q]);
      return ED_EINVAL;
    }
  for (int m = 0; m < n_terms; ++m) {
    if (delta[m] == 0) { set_error("cross term %d does not move the charge", m); return ED_EINVAL; }
    for (int q = 0; q < nq; ++q) {
      const bool in = q + delta[m] >= 0 && q + delta[m] < nq;
      if (!in && (Lm[(size_t)m * nq + q] || Rm[(size_t)m * nq + q])) {
        set_error("cross term %d has a block from %d to outside 0..%d", m, q, nq - 1);
        return ED_EINVAL;
      }
      if (in && (!Lm[(size_t)m * nq + q]) != (!Rm[(size_t)m * nq + q])) {
        set_error("cross term %d: block %d has only one of its two factors", m, q);
        return ED_EINVAL;
      }
    }
  }
  ed_dense* d = new (std::nothrow) ed_dense();
  if (!d) { set_error("host allocation failed"); return ED_ENOMEM; }
  struct Guard {
    ed_dense* d;
    ~Guard() { delete d; }
  } g{d};
  if (cudaGetDevice(&d->device) != cudaSuccess) { cudaGetLastError(); d->device = 0; }
  d->nq = nq;
  d->chi.assign(chi, chi + nq);
  d->off.assign(nq + 1, 0);
  for (int q = 0; q < nq; ++q) d->off[q + 1] = d->off[q] + chi[q] * chi[q];
  d->D = d->off[nq];
  d->HL.resize(nq);
  d->HR.resize(nq);
  for (int q = 0; q < nq; ++q) {
    ED_TRY(upload(d, HL[q], (size_t)(chi[q] * chi[q]), &d->HL[q]));
    ED_TRY(upload(d, HR[q], (size_t)(chi[q] * chi[q]), &d->HR[q]));
  }
  int64_t scratch = 0;
  for (int m = 0; m < n_terms; ++m) {
    ed_dense::Term t;
    t.delta = delta[m];
    t.L.assign(nq, nullptr);
    t.R.assign(nq, nullptr);
    t.toff.assign(nq, -1);
    int64_t s = 0;
    for (int q = 0; q < nq; ++q) {
      const double* l = Lm[(size_t)m * nq + q];
      if (!l) continue;
      const int64_t ct = chi[q + delta[m]];
      ED_TRY(upload(d, l, (size_t)(ct * chi[q]), &t.L[q]));
      ED_TRY(upload(d, Rm[(size_t)m * nq + q], (size_t)(ct * chi[q]), &t.R[q]));
      t.toff[q] = s;
      s += ct * chi[q];
    }
    scratch = std::max(scratch, s);
    d->terms.push_back(std::move(t));
  }
  if (scratch > 0) ED_TRY(dense_alloc(d, (void**)&d->scratch, (size_t)scratch * sizeof(double)));
  // problem lists: (1) Y_q = H_L Psi_q, (2) Y_q += Psi_q H_R^T, then per
  // term (3) T_q = L Psi_q, (4) Y_{q+delta} += T_q R^T; each stage is one
  // launch, whose problems write disjoint outputs
  std::vector<GemmProblem> all;
  auto close_stage = [&](size_t first) -> ed_status {
    long long tiles = 0;
    for (size_t i = first; i < all.size(); ++i) {
      all[i].tile0 = tiles;
      tiles += (long long)((all[i].M + kDT - 1) / kDT) * all[i].tiles_n;
    }
    if (tiles > 0x7fffffffLL) {
      set_error("dense-block stage of %lld tiles exceeds one launch", tiles);
      return ED_EUNSUPPORTED;
    }
    if (all.size() > first) d->stages.push_back({(int)first, (int)(all.size() - first), tiles});
    return ED_OK;
  };
  size_t f = all.size();
  for (int q = 0; q < nq; ++q) {
    const long long c = chi[q];
    all.push_back(problem(abs_(d->HL[q]), c, 1, xo(d->off[q]), c, 1, yo(d->off[q]), c, (int)c, (int)c, (int)c, 0));
  }
  ED_TRY(close_stage(f));
  f = all.size();
  for (int q = 0; q < nq; ++q) {
    const long long c = chi[q];
    all.push_back(problem(xo(d->off[q]), c, 1, abs_(d->HR[q]), 1, c, yo(d->off[q]), c, (int)c, (int)c, (int)c, 1));
  }
  ED_TRY(close_stage(f));
  for (const auto& t : d->terms) {
    f = all.size();
    for (int q = 0; q < nq; ++q) {
      if (!t.L[q]) continue;
      const long long c = chi[q], ct = chi[q + t.delta];
      all.push_back(problem(abs_(t.L[q]), c, 1, xo(d->off[q]), c, 1, abs_(d->scratch + t.toff[q]), c, (int)ct, (int)c,
                            (int)c, 0));
    }
    ED_TRY(close_stage(f));
    f = all.size();
    for (int q = 0; q < nq; ++q) {
      if (!t.L[q]) continue;
      const long long c = chi[q], ct = chi[q + t.delta];
      all.push_back(problem(abs_(d->scratch + t.toff[q]), c, 1, abs_(t.R[q]), 1, c, yo(d->off[q + t.delta]), ct,
                            (int)ct, (int)ct, (int)c, 1));
    }
    ED_TRY(close_stage(f));
  }
  ED_TRY(dense_alloc(d, (void**)&d->d_probs, all.size() * sizeof(GemmProblem)));
  ED_CUDA_TRY(cudaMemcpy(d->d_probs, all.data(), all.size() * sizeof(GemmProblem), cudaMemcpyHostToDevice));
  g.d = nullptr;
  *out = d;
  return ED_OK;
}

extern "C" int64_t ed_dense_dim(const ed_dense* d) { return d ? d->D : -1; }

extern "C" ed_status ed_dense_apply(ed_dense* d, const double* x, double* y, void* stream) {
  if (!d) { set_error("dense operator is NULL"); return ED_EINVAL; }
  if (!x || !y) { set_error("x or y is NULL"); return ED_EINVAL; }
  if (x < y + d->D && y < x + d->D) { set_error("x and y overlap"); return ED_EINVAL; }
  ED_DEVICE_SCOPE(d->device);
  cudaStream_t st = (cudaStream_t)stream;
  for (const auto& s : d->stages) {
    k_gemm_batch<<<(unsigned)s.tiles, 256, 0, st>>>(d->d_probs + s.first, s.count, x, y);
    ED_CUDA_TRY(cudaGetLastError());
  }
  return ED_OK;
}

extern "C" void ed_dense_destroy(ed_dense* d) { delete d; }
