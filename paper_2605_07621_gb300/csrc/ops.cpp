// Side operators of the block Hamiltonian (paper Eq. (2)):
//   * H_A,s and H_B,s off-diagonal parts as CSR over each side's states
//     (spin: S^+S^- + h.c. of bonds inside the side; Hubbard with the spin
//     cut: hopping of the up electrons on side A, of the down electrons on
//     side B, with the Jordan-Wigner sign of the fixed operator order);
//   * the side diagonals V_A(a), V_B(b) and packed bit words from which the
//     kernels evaluate the diagonal cross term V_AB(a,b) by popcounts (the
//     "diagonal form" the paper notes for symmetric cases);
//   * the cross-cut maps: for every A site p touched by a cross bond, the
//     rank of a XOR (1<<p) in its new charge sector (likewise for B), i.e.
//     the partial permutations L_m, R_m of Eq. (2) in index form.
#include <cstring>

#include "ed_internal.h"

using namespace edk;

namespace {

struct HostSideOps {
  std::vector<int> rowptr, col;
  std::vector<double> val64, diag;
  std::vector<float> val32;
  std::vector<unsigned long long> pack;
  std::vector<int> maps;  // [n_cross_bits][total]
};

inline int parity_between(uint32_t x, int p, int q) {
  int lo = p < q ? p : q, hi = p < q ? q : p;
  if (hi - lo <= 1) return 0;
  uint32_t m = (uint32_t)(((1ULL << hi) - 1) & ~((1ULL << (lo + 1)) - 1));
  return __builtin_popcount(x & m) & 1;
}

ed_status build_side_ops(const ed_ctx* c, const Side& sd, const std::vector<ed_ctx::SideBond>& bonds, bool sideA,
                         HostSideOps& h) {
  const bool hub = c->kind == ED_HUBBARD;
  int64_t tot = sd.total();
  h.rowptr.assign(tot + 1, 0);
  h.diag.assign(tot, 0.0);
  h.pack.assign(tot, 0ULL);
  h.col.clear();
  h.val64.clear();
  std::vector<std::pair<int, double>> row;
  for (int k = 0; k <= sd.n; ++k) {
    if (!sd.used[k]) continue;
    for (int64_t g = sd.start[k]; g < sd.start[k + 1]; ++g) {
      uint32_t x = sd.states[g];
      row.clear();
      double d = 0.0;
      for (const auto& b : bonds) {
        int bp = (x >> b.p) & 1, bq = (x >> b.q) & 1;
        if (!hub) d += b.jz * (bp == bq ? 0.25 : -0.25);
        if (bp == bq || b.off == 0.0) continue;
        uint32_t y = x ^ ((1u << b.p) | (1u << b.q));
        double v = b.off;
        if (hub && parity_between(x, b.p, b.q)) v = -v;
        row.push_back({(int)combinadic_rank(y), v});
      }
      if (hub) {
        for (int p = 0; p < sd.n; ++p)
          if ((x >> p) & 1) d += c->eps[sd.sites[p]];
      }
      std::sort(row.begin(), row.end(), [](const std::pair<int, double>& a, const std::pair<int, double>& b) {
        return a.first < b.first;
      });
      for (auto& e : row) {
        h.col.push_back(e.first);
        h.val64.push_back(e.second);
      }
      if (h.col.size() > (size_t)0x7fffffff) {
        set_error("side CSR exceeds 2^31 entries");
        return ED_EUNSUPPORTED;
      }
      h.rowptr[g + 1] = (int)h.col.size();
      h.diag[g] = d;
      unsigned long long pk = 0;
      if (hub) {
        pk = x;
      } else {
        for (size_t kk = 0; kk < c->cross.size(); ++kk) {
          int bit = sideA ? c->cross[kk].p : c->cross[kk].q;
          pk |= (unsigned long long)((x >> bit) & 1u) << kk;
        }
      }
      h.pack[g] = pk;
    }
  }
  h.val32.resize(h.val64.size());
  for (size_t e = 0; e < h.val64.size(); ++e) h.val32[e] = (float)h.val64[e];
  const std::vector<int>& bits = sideA ? c->crossA_bits : c->crossB_bits;
  h.maps.assign(bits.size() * (size_t)tot, -1);
  for (size_t i = 0; i < bits.size(); ++i) {
    for (int64_t g = 0; g < tot; ++g) {
      uint32_t y = sd.states[g] ^ (1u << bits[i]);
      int ky = __builtin_popcount(y);
      if (ky <= sd.n && sd.used[ky]) h.maps[i * (size_t)tot + g] = (int)combinadic_rank(y);
    }
  }
  return ED_OK;
}

}  // namespace

extern "C" ed_status ed_build_local_ops(ed_ctx* c, int flags) {
  if (!c) { set_error("ctx is NULL"); return ED_EINVAL; }
  if (flags < 0 || flags > 2) { set_error("bad flags %d", flags); return ED_EINVAL; }
  if (c->ops_built) return ED_OK;
  ED_CUDA_TRY(cudaSetDevice(c->device));
  HostSideOps ha, hb;
  ED_TRY(build_side_ops(c, c->A, c->bondsA, true, ha));
  ED_TRY(build_side_ops(c, c->B, c->bondsB, false, hb));
  c->nnzA = (int64_t)ha.col.size();
  c->nnzB = (int64_t)hb.col.size();
  DevTables& t = c->tab;
  int *Arp, *Acol, *Brp, *Bcol, *mA, *mB;
  double *Av64, *Bv64, *Ad, *Bd;
  float *Av32, *Bv32;
  unsigned long long *Apk, *Bpk;
  uint32_t *Ast, *Bst;
  ED_TRY(upload(c, &Arp, ha.rowptr));
  ED_TRY(upload(c, &Acol, ha.col));
  ED_TRY(upload(c, &Av64, ha.val64));
  ED_TRY(upload(c, &Av32, ha.val32));
  ED_TRY(upload(c, &Ad, ha.diag));
  ED_TRY(upload(c, &Apk, ha.pack));
  ED_TRY(upload(c, &mA, ha.maps));
  ED_TRY(upload(c, &Brp, hb.rowptr));
  ED_TRY(upload(c, &Bcol, hb.col));
  ED_TRY(upload(c, &Bv64, hb.val64));
  ED_TRY(upload(c, &Bv32, hb.val32));
  ED_TRY(upload(c, &Bd, hb.diag));
  ED_TRY(upload(c, &Bpk, hb.pack));
  ED_TRY(upload(c, &mB, hb.maps));
  ED_TRY(upload(c, &Ast, c->A.states));
  ED_TRY(upload(c, &Bst, c->B.states));
  std::vector<float> ad32(ha.diag.begin(), ha.diag.end()), bd32(hb.diag.begin(), hb.diag.end());
  std::vector<unsigned long long> akey(c->A.total()), bkey(c->B.total());
  for (int64_t g = 0; g < c->A.total(); ++g) akey[g] = state_key(c, c->A.states[g], 0u);
  for (int64_t g = 0; g < c->B.total(); ++g) bkey[g] = state_key(c, 0u, c->B.states[g]);
  float *Ad32, *Bd32;
  unsigned long long *Ak, *Bk;
  ED_TRY(upload(c, &Ad32, ad32));
  ED_TRY(upload(c, &Bd32, bd32));
  ED_TRY(upload(c, &Ak, akey));
  ED_TRY(upload(c, &Bk, bkey));
  t.A_diag32 = Ad32; t.B_diag32 = Bd32; t.A_key = Ak; t.B_key = Bk;
  c->diag.c0_32 = (float)c->diag.c0;
  for (int q = 0; q < kMaxClasses; ++q) c->diag.w32[q] = (float)c->diag.w[q];
  t.A_rowptr = Arp; t.A_col = Acol; t.A_val64 = Av64; t.A_val32 = Av32; t.A_diag = Ad; t.A_pack = Apk; t.mapA = mA;
  t.B_rowptr = Brp; t.B_col = Bcol; t.B_val64 = Bv64; t.B_val32 = Bv32; t.B_diag = Bd; t.B_pack = Bpk; t.mapB = mB;
  t.A_states = Ast; t.B_states = Bst;
  t.A_total = c->A.total();
  t.B_total = c->B.total();

  c->h_blocks.clear();
  std::vector<long long> rs;
  for (const Block& b : c->blocks) {
    DevBlock db;
    db.s = b.s;
    db.kB = b.kB;
    db.nbr_lo = (b.s - 1 >= 0) ? c->block_of_s[b.s - 1] : -1;
    db.nbr_hi = (b.s + 1 < (int)c->block_of_s.size()) ? c->block_of_s[b.s + 1] : -1;
    db.dA = b.dA; db.dB = b.dB; db.off = b.off; db.gA0 = b.gA0; db.gB0 = b.gB0; db.row0 = b.row0;
    c->h_blocks.push_back(db);
    rs.push_back(b.row0);
  }
  rs.push_back(c->n_rows);
  ED_TRY(upload(c, &c->d_blocks, c->h_blocks));
  ED_TRY(upload(c, &c->d_row_start, rs));
  c->h_cross.clear();
  for (const auto& cb : c->cross) c->h_cross.push_back(DevCross{cb.ia, cb.ib, cb.coef});
  ED_TRY(upload(c, &c->d_cross, c->h_cross));
  c->ops_flags = flags;
  c->ops_built = true;
  return ED_OK;
}
