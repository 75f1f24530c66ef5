// Dense-block bipartite H|psi>: the operator of paper Eq. (2),
//   H = sum_q H_L,q (x) 1 + 1 (x) H_R,q + sum_m L_m (x) R_m,
// with dense side operators on symmetry blocks (the paper's DMRG setting,
// block dimensions chi_q).  A state is the concatenation of row-major blocks
// Psi_q (chi_q x chi_q); by the Vec identity each term is a product of dense
// matrices:
//   Y_q  = H_L,q Psi_q + Psi_q H_R,q^T
//   Y_q' += L_m,q Psi_q R_m,q^T,  q' = q + delta_m.
// Every product runs on the tensor cores in FP64-accurate digit-split form
// (ozaki.cu): the side operators are split once at creation; each apply
// splits the blocks of x (as rows for Psi H_R^T, as columns for H_L Psi and
// L Psi) and the intermediate L Psi, and every stage is one launch over all
// blocks.
#include <cstring>
#include <new>
#include <vector>

#include "krylov.h"
#include "ozaki.h"

using namespace edk;

struct ed_dense {
  int device = 0;
  int nq = 0;
  std::vector<int64_t> chi, off;
  int64_t D = 0;
  struct Term {
    int delta;
    std::vector<OzOperand> L, R;  // per source block q (R == 0: none)
    std::vector<OzOperand> T;     // digit planes of L Psi_q
    std::vector<int64_t> toff;    // scratch offset of L Psi_q per q
  };
  std::vector<OzOperand> HL, HR;  // per block
  std::vector<OzOperand> XA, XB;  // per block: Psi_q by rows, by columns
  std::vector<Term> terms;
  double* scratch = nullptr;
  OzContext oz;
  // device lists of the slicing and product stages
  struct Stage {
    int kind;  // 0: slice by rows, 1: slice by columns, 2: products
    const void* list;
    int count;
    long long units;
  };
  std::vector<Stage> stages;
};

namespace {

ed_status dense_alloc(ed_dense* d, void** p, size_t bytes) { return oz_alloc(&d->oz, p, bytes); }

OzProblem oz_problem(const OzOperand& A, const OzOperand& B, double* C, long long coff, int cbase, long long ldc,
                     int acc) {
  OzProblem p;
  p.mapA = A.map;
  p.mapB = B.map;
  p.ea = A.exps;
  p.eb = B.exps;
  p.C = C;
  p.coff = coff;
  p.cbase = cbase;
  p.ldc = ldc;
  p.M = A.R;
  p.N = B.R;
  p.K = A.K;
  p.acc = acc;
  p.tiles_n = (B.R + kOzBN - 1) / kOzBN;
  p.tri = 0;
  p.tile0 = 0;
  return p;
}

OzSliceJob slice_job(const double* src, long long soff, int sbase, long long ld, int rows, int cols,
                     const OzOperand& dst) {
  OzSliceJob j;
  j.src = src;
  j.soff = soff;
  j.sbase = sbase;
  j.ld = ld;
  j.rows = rows;
  j.cols = cols;
  j.dst = dst.slices;
  j.exps = dst.exps;
  j.Kpad = dst.Kpad;
  j.first = 0;
  return j;
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
  d->oz.device = d->device;
  d->nq = nq;
  d->chi.assign(chi, chi + nq);
  d->off.assign(nq + 1, 0);
  for (int q = 0; q < nq; ++q) d->off[q + 1] = d->off[q] + chi[q] * chi[q];
  d->D = d->off[nq];
  // side operators split once: H_L as the left factor (rows = output rows),
  // H_R as B^T of Psi H_R^T (rows = output columns)
  d->HL.resize(nq);
  d->HR.resize(nq);
  d->XA.resize(nq);
  d->XB.resize(nq);
  for (int q = 0; q < nq; ++q) {
    const int c = (int)chi[q];
    ED_TRY(oz_operand_host(&d->oz, HL[q], c, c, true, &d->HL[q]));
    ED_TRY(oz_operand_host(&d->oz, HR[q], c, c, false, &d->HR[q]));
    ED_TRY(oz_operand_device(&d->oz, c, c, true, &d->XA[q]));   // Psi_q: rows
    ED_TRY(oz_operand_device(&d->oz, c, c, false, &d->XB[q]));  // Psi_q^T: columns of Psi_q
  }
  int64_t scratch = 0;
  for (int m = 0; m < n_terms; ++m) {
    ed_dense::Term t;
    t.delta = delta[m];
    t.L.assign(nq, OzOperand{});
    t.R.assign(nq, OzOperand{});
    t.T.assign(nq, OzOperand{});
    t.toff.assign(nq, -1);
    int64_t s = 0;
    for (int q = 0; q < nq; ++q) {
      const double* l = Lm[(size_t)m * nq + q];
      if (!l) continue;
      const int c = (int)chi[q], ct = (int)chi[q + delta[m]];
      ED_TRY(oz_operand_host(&d->oz, l, ct, c, true, &t.L[q]));
      ED_TRY(oz_operand_host(&d->oz, Rm[(size_t)m * nq + q], ct, c, false, &t.R[q]));
      ED_TRY(oz_operand_device(&d->oz, ct, c, true, &t.T[q]));
      t.toff[q] = s;
      s += (int64_t)ct * c;
    }
    scratch = std::max(scratch, s);
    d->terms.push_back(std::move(t));
  }
  if (scratch > 0) ED_TRY(dense_alloc(d, (void**)&d->scratch, (size_t)scratch * sizeof(double)));
  ED_TRY(oz_finish(&d->oz));
  // stage lists (device, built once): each launch covers every block
  auto put = [&](int kind, const void* host, size_t bytes, int count, long long units) -> ed_status {
    void* dp = nullptr;
    ED_TRY(dense_alloc(d, &dp, bytes));
    ED_CUDA_TRY(cudaMemcpy(dp, host, bytes, cudaMemcpyHostToDevice));
    d->stages.push_back({kind, dp, count, units});
    return ED_OK;
  };
  auto slices = [&](std::vector<OzSliceJob>& v, bool by_cols) -> ed_status {
    long long u = 0;
    for (auto& j : v) {
      j.first = u;
      u += by_cols ? (j.cols + 31) / 32 : j.rows;
    }
    if (v.empty()) return ED_OK;
    return put(by_cols ? 1 : 0, v.data(), v.size() * sizeof(OzSliceJob), (int)v.size(), u);
  };
  auto products = [&](std::vector<OzProblem>& v) -> ed_status {
    long long tiles = 0;
    for (auto& p : v) {
      p.tile0 = tiles;
      tiles += oz_tiles(p.M, p.N);
    }
    if (tiles > 0x7fffffffLL) {
      set_error("dense-block stage of %lld tiles exceeds one launch", tiles);
      return ED_EUNSUPPORTED;
    }
    if (v.empty()) return ED_OK;
    return put(2, v.data(), v.size() * sizeof(OzProblem), (int)v.size(), tiles);
  };
  {
    std::vector<OzSliceJob> ja, jb;
    for (int q = 0; q < nq; ++q) {
      const int c = (int)chi[q];
      ja.push_back(slice_job(nullptr, d->off[q], 1, c, c, c, d->XA[q]));
      jb.push_back(slice_job(nullptr, d->off[q], 1, c, c, c, d->XB[q]));
    }
    ED_TRY(slices(ja, false));
    ED_TRY(slices(jb, true));
  }
  {
    std::vector<OzProblem> s1, s2;
    for (int q = 0; q < nq; ++q) {
      const long long c = chi[q];
      s1.push_back(oz_problem(d->HL[q], d->XB[q], nullptr, d->off[q], 1, c, 0));  // Y = H_L Psi
      s2.push_back(oz_problem(d->XA[q], d->HR[q], nullptr, d->off[q], 1, c, 1));  // Y += Psi H_R^T
    }
    ED_TRY(products(s1));
    ED_TRY(products(s2));
  }
  for (const auto& t : d->terms) {
    std::vector<OzProblem> s3, s4;
    std::vector<OzSliceJob> jt;
    for (int q = 0; q < nq; ++q) {
      if (!t.L[q].slices) continue;
      const long long c = chi[q], ct = chi[q + t.delta];
      double* T = d->scratch + t.toff[q];
      s3.push_back(oz_problem(t.L[q], d->XB[q], T, 0, 0, c, 0));                   // T = L Psi
      jt.push_back(slice_job(T, 0, 0, c, (int)ct, (int)c, t.T[q]));
      s4.push_back(oz_problem(t.T[q], t.R[q], nullptr, d->off[q + t.delta], 1, ct, 1));  // Y' += T R^T
    }
    ED_TRY(products(s3));
    ED_TRY(slices(jt, false));
    ED_TRY(products(s4));
  }
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
    if (s.kind == 2)
      ED_TRY(oz_gemm(&d->oz, (const OzProblem*)s.list, s.count, s.units, y, st));
    else
      ED_TRY(oz_slice(&d->oz, (const OzSliceJob*)s.list, s.count, s.units, s.kind == 1, x, st));
  }
  return ED_OK;
}

extern "C" void ed_dense_destroy(ed_dense* d) { delete d; }
