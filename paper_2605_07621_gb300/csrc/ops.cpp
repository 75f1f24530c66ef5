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
#include <cmath>
#include <cstring>

#include "ed_internal.h"

using namespace edk;

namespace {

inline int parity_between(uint32_t x, int p, int q) {
  int lo = p < q ? p : q, hi = p < q ? q : p;
  if (hi - lo <= 1) return 0;
  uint32_t m = (uint32_t)(((1ULL << hi) - 1) & ~((1ULL << (lo + 1)) - 1));
  return __builtin_popcount(x & m) & 1;
}

}  // namespace

namespace edk {
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
}  // namespace edk

namespace {

// exact test: v * 2^k is an integer of magnitude <= 2^24
bool dyadic_at(double v, int k) {
  double t = std::ldexp(v, k);
  return std::fabs(t) <= 16777216.0 && t == std::trunc(t);
}

struct Side3 {
  std::vector<uint2> meta;
  std::vector<uint16_t> col;
  std::vector<uint32_t> pack;
  std::vector<int> dI;
  std::vector<uint2> meta4;
  std::vector<uint16_t> col4;
};

// padded copy: class segments start at multiples of 4 entries and are filled
// up with `zero_idx` (an always-zero slot after the row in shared memory)
bool build_padded(const Side& sd, Side3& o) {
  const int64_t tot = (int64_t)o.meta.size();
  o.meta4.resize(tot);
  o.col4.clear();
  for (int k = 0; k <= sd.n; ++k) {
    if (!sd.used[k]) continue;
    const uint16_t zero_idx = (uint16_t)sd.dim(k);
    for (int64_t g = sd.start[k]; g < sd.start[k + 1]; ++g) {
      const uint2 m = o.meta[g];
      if (o.col4.size() / 4 > 0xFFFFFFFFull) return false;
      const uint32_t start4 = (uint32_t)(o.col4.size() / 4);
      uint32_t e = m.x, packed = 0;
      for (int c = 0; c < kMaxCls; ++c) {
        const uint32_t n = (m.y >> (8 * c)) & 255u;
        const uint32_t n4 = (n + 3) / 4;
        for (uint32_t i = 0; i < 4 * n4; ++i) o.col4.push_back(i < n ? o.col[e + i] : zero_idx);
        e += n;
        packed |= n4 << (8 * c);
      }
      o.meta4[g] = make_uint2(start4, packed);
    }
  }
  return true;
}

// class-sorted copy of one side's CSR
bool build_side3(const HostSideOps& h, const std::vector<double>& cls_val, Side3& o) {
  const int64_t tot = (int64_t)h.rowptr.size() - 1;
  o.meta.resize(tot);
  o.col.clear();
  o.col.reserve(h.col.size());
  for (int64_t g = 0; g < tot; ++g) {
    uint32_t cnt[kMaxCls] = {0, 0, 0, 0};
    const uint32_t start = (uint32_t)o.col.size();
    for (int c = 0; c < (int)cls_val.size(); ++c) {
      for (int e = h.rowptr[g]; e < h.rowptr[g + 1]; ++e) {
        if (h.val64[e] != cls_val[c]) continue;
        if (h.col[e] > 0xFFFF) return false;
        o.col.push_back((uint16_t)h.col[e]);
        ++cnt[c];
      }
      if (cnt[c] > 255) return false;
    }
    o.meta[g] = make_uint2(start, cnt[0] | (cnt[1] << 8) | (cnt[2] << 16) | (cnt[3] << 24));
  }
  o.pack.resize(tot);
  for (int64_t g = 0; g < tot; ++g) o.pack[g] = (uint32_t)h.pack[g];
  return true;
}

}  // namespace

// Tables of the class-sorted path; leaves c->v3_ok false when the model
// needs more than kMaxCls off-diagonal values, more than 32 cross bonds or
// sides with more than 65535 states per charge.
static ed_status build_v3(ed_ctx* c, const HostSideOps& ha, const HostSideOps& hb) {
  c->v3_ok = false;
  c->dyadic = false;
  c->diag_split = false;
  if (c->cross.size() > 32) return ED_OK;
  if (c->kind == ED_HUBBARD && c->n_sites > 32) return ED_OK;
  for (const Block& b : c->blocks)
    if (b.dA > 65535 || b.dB > 65535) return ED_OK;
  std::vector<double> cls;
  auto add_cls = [&](double v) {
    if (std::find(cls.begin(), cls.end(), v) == cls.end()) cls.push_back(v);
  };
  for (double v : ha.val64) add_cls(v);
  for (double v : hb.val64) add_cls(v);
  for (const auto& cb : c->cross) add_cls(cb.coef);
  if (cls.size() > (size_t)kMaxCls) return ED_OK;
  Side3 a3, b3;
  if (!build_side3(ha, cls, a3) || !build_side3(hb, cls, b3)) return ED_OK;
  for (const Block& b : c->blocks)
    if (b.dB >= 65535) return ED_OK;  // the zero slot index d_B must fit 16 bits
  if (!build_padded(c->B, b3)) return ED_OK;
  Dev3& t = c->t3;
  t = Dev3{};
  for (size_t i = 0; i < cls.size(); ++i) {
    t.w64[i] = cls[i];
    t.w32[i] = (float)cls[i];
  }
  c->cross_cls.assign(c->cross.size(), 0);
  for (size_t k = 0; k < c->cross.size(); ++k) {
    int ci = (int)(std::find(cls.begin(), cls.end(), c->cross[k].coef) - cls.begin());
    c->cross_cls[k] = ci;
    t.cross_cls_mask[ci] |= 1u << k;
    t.ib_mask[c->cross[k].ib] |= 1u << k;
    t.ia_mask[c->cross[k].ia] |= 1u << k;
    t.bond_ia[k] = (unsigned char)c->cross[k].ia;
    t.bond_ib[k] = (unsigned char)c->cross[k].ib;
    t.bond_w64[k] = c->cross[k].coef;
    t.bond_w32[k] = (float)c->cross[k].coef;
  }
  t.n_ib = (int)c->crossB_bits.size();
  t.n_ia = (int)c->crossA_bits.size();
  // bond lists of the row pass: per B cross site and value class at most two
  // bonds, at most two classes over all cross bonds
  {
    std::vector<int> cc;
    for (int ci : c->cross_cls)
      if (std::find(cc.begin(), cc.end(), ci) == cc.end()) cc.push_back(ci);
    t.xl_ok = cc.size() <= 2 ? 1 : 0;
    t.xl_c[0] = cc.empty() ? 0 : cc[0];
    t.xl_c[1] = cc.size() > 1 ? cc[1] : t.xl_c[0];
    t.xl_c1_mask = cc.size() > 1 ? t.cross_cls_mask[cc[1]] : 0u;
    for (int ib = 0; t.xl_ok && ib < t.n_ib; ++ib)
      if (__builtin_popcount(t.ib_mask[ib] & ~t.xl_c1_mask) > 2 || __builtin_popcount(t.ib_mask[ib] & t.xl_c1_mask) > 2)
        t.xl_ok = 0;
  }
  const DevDiagParams& dp = c->diag;
  t.vab_and = dp.vab_and;
  t.ncls_d = dp.ncls;
  for (int q = 0; q < dp.ncls; ++q) {
    if (dp.mask[q] >> 32) return ED_OK;
    t.dmask[q] = (unsigned)dp.mask[q];
    t.dw64[q] = dp.w[q];
    t.dw32[q] = (float)dp.w[q];
  }
  t.dc0_64 = dp.c0;
  t.dc0_32 = (float)dp.c0;
  // dyadic scale for the exact fixed-point FP64 path
  std::vector<double> vals(cls.begin(), cls.end());
  vals.push_back(dp.c0);
  for (int q = 0; q < dp.ncls; ++q) vals.push_back(dp.w[q]);
  int qs = -1;
  for (int k = 0; k <= 30 && qs < 0; ++k) {
    bool ok = true;
    for (double v : vals) ok = ok && dyadic_at(v, k);
    for (size_t g = 0; ok && g < ha.diag.size(); ++g) ok = dyadic_at(ha.diag[g], k);
    for (size_t g = 0; ok && g < hb.diag.size(); ++g) ok = dyadic_at(hb.diag[g], k);
    if (ok) qs = k;
  }
  // otherwise, when only the diagonal is not dyadic (disordered on-site
  // energies, say), the integer passes take the off-diagonal terms and the
  // diagonal is added in FP64 after them (one FMA per element)
  c->diag_split = false;
  for (int k = 0; qs < 0 && k <= 30; ++k) {
    bool ok = true;
    for (double v : cls) ok = ok && dyadic_at(v, k);
    if (ok) {
      qs = k;
      c->diag_split = true;
    }
  }
  if (qs >= 0) {
    t.q_shift = qs;
    for (size_t i = 0; i < cls.size(); ++i) t.wI[i] = (long long)std::ldexp(cls[i], qs);
    for (size_t k = 0; k < c->cross.size(); ++k) t.bond_wI[k] = (long long)std::ldexp(c->cross[k].coef, qs);
    const bool sd = c->diag_split;  // diagonal tables of the integer passes stay zero
    for (int q = 0; q < dp.ncls; ++q) t.dwI[q] = sd ? 0 : (long long)std::ldexp(dp.w[q], qs);
    t.dc0_I = sd ? 0 : (long long)std::ldexp(dp.c0, qs);
    a3.dI.assign(ha.diag.size(), 0);
    b3.dI.assign(hb.diag.size(), 0);
    for (size_t g = 0; !sd && g < ha.diag.size(); ++g) a3.dI[g] = (int)std::ldexp(ha.diag[g], qs);
    for (size_t g = 0; !sd && g < hb.diag.size(); ++g) b3.dI[g] = (int)std::ldexp(hb.diag[g], qs);
    // bound on sum_j |M_ij| (units 2^-q_shift) -> headroom of the int64 sums
    auto side_max = [&](const Side3& s3, const std::vector<int>& dI) {
      double m = 0.0;
      for (size_t g = 0; g < s3.meta.size(); ++g) {
        double r = std::fabs((double)dI[g]);
        for (int cc = 0; cc < kMaxCls; ++cc) r += ((s3.meta[g].y >> (8 * cc)) & 255u) * std::fabs((double)t.wI[cc]);
        m = std::max(m, r);
      }
      return m;
    };
    double rmax = side_max(a3, a3.dI) + side_max(b3, b3.dI) + std::fabs((double)t.dc0_I);
    for (int q = 0; q < dp.ncls; ++q) rmax += std::fabs((double)t.dwI[q]) * __builtin_popcountll(dp.mask[q]);
    // (the diagonal terms of a split diagonal are zero here: dI, dwI, dc0_I)
    for (size_t k = 0; k < c->cross.size(); ++k) rmax += std::fabs((double)t.wI[c->cross_cls[k]]);
    int bits = (int)std::ceil(std::log2(rmax + 1.0));
    t.P = std::min(60, 62 - bits);
    c->dyadic = t.P >= 40;
  }
  if (!c->dyadic) c->diag_split = false;
  // couplings that are not dyadic: fixed-point input summed exactly per value
  // class (at most the largest per-class count of one row's terms in one
  // pass, plus the cross bonds).  Every FP64 coupling and diagonal value is
  // an integer multiple of 2^-qw, qw from the smallest unit among them; when
  // those integers fit 61 bits they are the 64-bit weights of exact 128-bit
  // sums (wide path), otherwise each class sum is weighted in FP64
  c->classed = false;
  c->wide = false;
  std::vector<long long> AdW, BdW;
  if (!c->dyadic) {
    long long mx = 1;
    for (const Side3* s3 : {&a3, &b3})
      for (const uint2& m : s3->meta)
        for (int cc = 0; cc < kMaxCls; ++cc) mx = std::max<long long>(mx, (m.y >> (8 * cc)) & 255u);
    mx += (long long)c->cross.size();
    const int bits = (int)std::ceil(std::log2((double)mx + 1.0));
    t.q_shift = 0;
    t.P = std::min(60, 62 - bits);
    c->classed = t.P >= 40;
    // the values the wide path multiplies: off-diagonal classes, cross-bond
    // coefficients, and the terms of the diagonal (bond jz / 4, on-site
    // energies, the cross-cut diagonal's weights); the side diagonals and
    // c0 are then exact integer sums of these terms (not the rounded FP64
    // sums, whose cancellation residues would need far smaller units)
    const bool hub = c->kind == ED_HUBBARD;
    std::vector<double> base(cls.begin(), cls.end());
    for (const auto& cr : c->cross) {
      base.push_back(cr.coef);
      base.push_back(0.25 * cr.jz);
    }
    for (int q = 0; q < dp.ncls; ++q) base.push_back(dp.w[q]);
    for (const auto* bl : {&c->bondsA, &c->bondsB})
      for (const auto& b : *bl) base.push_back(0.25 * b.jz);
    if (hub)
      for (double e : c->eps) base.push_back(e);
    int emin = 1 << 30, emx = -(1 << 30);
    for (double v : base)
      if (v != 0.0 && std::isfinite(v)) {
        const int e = std::ilogb(v);
        emin = std::min(emin, e - 52);
        emx = std::max(emx, e);
      }
    if (c->classed && emin < (1 << 30) && emx - emin <= 55) {
      const int qw = -emin;
      auto W = [&](double v) { return (long long)std::ldexp(v, qw); };  // exact: v is k 2^-qw, |k| < 2^56
      long long wW[kMaxCls] = {0, 0, 0, 0}, dwW[kMaxClasses] = {};
      for (size_t i = 0; i < cls.size(); ++i) wW[i] = W(cls[i]);
      for (int q = 0; q < dp.ncls; ++q) dwW[q] = W(dp.w[q]);
      long long c0W = 0;
      if (!hub)
        for (const auto& cr : c->cross) c0W += W(0.25 * cr.jz);
      auto side_diag = [&](const Side& sd, const std::vector<ed_ctx::SideBond>& bonds, std::vector<long long>& out) {
        out.assign(sd.total(), 0);
        for (int64_t g = 0; g < sd.total(); ++g) {
          const uint32_t x = sd.states[g];
          long long d = 0;
          if (!hub) {
            for (const auto& b : bonds) d += (((x >> b.p) & 1) == ((x >> b.q) & 1) ? 1 : -1) * W(0.25 * b.jz);
          } else {
            for (int p = 0; p < sd.n; ++p)
              if ((x >> p) & 1) d += W(c->eps[sd.sites[p]]);
          }
          out[g] = d;
        }
      };
      side_diag(c->A, c->bondsA, AdW);
      side_diag(c->B, c->bondsB, BdW);
      // the integer diagonal fits 62 bits, the 128-bit sums fit with P bits of x
      double dmax = std::fabs((double)c0W);
      for (int q = 0; q < dp.ncls; ++q) dmax += std::fabs((double)dwW[q]) * __builtin_popcountll(dp.mask[q]);
      auto side_max = [&](const Side3& s3, const std::vector<long long>& dW, double* dm) {
        double m = 0.0, d = 0.0;
        for (size_t g = 0; g < s3.meta.size(); ++g) {
          double r = std::fabs((double)dW[g]);
          d = std::max(d, r);
          for (int cc = 0; cc < kMaxCls; ++cc) r += ((s3.meta[g].y >> (8 * cc)) & 255u) * std::fabs((double)wW[cc]);
          m = std::max(m, r);
        }
        *dm += d;
        return m;
      };
      double rmax = side_max(a3, AdW, &dmax) + side_max(b3, BdW, &dmax) + std::fabs((double)c0W);
      for (int q = 0; q < dp.ncls; ++q) rmax += std::fabs((double)dwW[q]) * __builtin_popcountll(dp.mask[q]);
      for (size_t k = 0; k < c->cross.size(); ++k) rmax += std::fabs((double)wW[c->cross_cls[k]]);
      const int Pw = std::min(t.P, 126 - (int)std::ceil(std::log2(rmax + 1.0)));
      if (dmax < 4.6e18 && Pw >= 40) {
        c->wide = true;
        t.P = Pw;
        t.q_shift = qw;
        for (int i = 0; i < kMaxCls; ++i) t.wI[i] = wW[i];
        for (size_t k = 0; k < c->cross.size(); ++k) t.bond_wI[k] = W(c->cross[k].coef);
        for (int q = 0; q < dp.ncls; ++q) t.dwI[q] = dwW[q];
        t.dc0_I = c0W;
      }
    }
  }
  // upload
  uint2 *Am, *Bm;
  uint16_t *Ac, *Bc, *mA, *mB;
  uint32_t *Ap, *Bp;
  int *AdI = nullptr, *BdI = nullptr;
  ED_TRY(upload(c, &Am, a3.meta));
  ED_TRY(upload(c, &Bm, b3.meta));
  ED_TRY(upload(c, &Ac, a3.col));
  ED_TRY(upload(c, &Bc, b3.col));
  ED_TRY(upload(c, &Ap, a3.pack));
  ED_TRY(upload(c, &Bp, b3.pack));
  long long *AdWd = nullptr, *BdWd = nullptr;
  if (c->dyadic) {
    ED_TRY(upload(c, &AdI, a3.dI));
    ED_TRY(upload(c, &BdI, b3.dI));
  }
  if (c->wide) {
    ED_TRY(upload(c, &AdWd, AdW));
    ED_TRY(upload(c, &BdWd, BdW));
  }
  std::vector<uint16_t> ma(ha.maps.size()), mb(hb.maps.size());
  for (size_t i = 0; i < ma.size(); ++i) ma[i] = ha.maps[i] < 0 ? 0xFFFF : (uint16_t)ha.maps[i];
  for (size_t i = 0; i < mb.size(); ++i) mb[i] = hb.maps[i] < 0 ? 0xFFFF : (uint16_t)hb.maps[i];
  ED_TRY(upload(c, &mA, ma));
  ED_TRY(upload(c, &mB, mb));
  uint2 *Bm4, *Bc4;
  {
    std::vector<uint2> c4(b3.col4.size() / 4);
    std::memcpy(c4.data(), b3.col4.data(), b3.col4.size() * sizeof(uint16_t));
    ED_TRY(upload(c, &Bm4, b3.meta4));
    ED_TRY(upload(c, &Bc4, c4));
  }
  t.B_meta4 = Bm4;
  t.B_col4 = Bc4;
  t.A_meta = Am; t.B_meta = Bm; t.A_col = Ac; t.B_col = Bc; t.A_pack = Ap; t.B_pack = Bp;
  t.A_dI = AdI; t.B_dI = BdI; t.A_dW = AdWd; t.B_dW = BdWd; t.mapA = mA; t.mapB = mB;
  t.A_d32 = c->tab.A_diag32; t.B_d32 = c->tab.B_diag32; t.A_d64 = c->tab.A_diag; t.B_d64 = c->tab.B_diag;
  t.A_total = c->A.total();
  t.B_total = c->B.total();
  ED_TRY(dev_alloc(c, (void**)&c->d_exp, 64));
  c->v3_ok = true;
  return ED_OK;
}

extern "C" ed_status ed_build_local_ops(ed_ctx* c, int flags) {
  if (!c) { set_error("ctx is NULL"); return ED_EINVAL; }
  if (flags < 0 || flags > 3 || flags == 3) {
    set_error("bad flags %d", flags);
    return ED_EINVAL;
  }
  if (c->ops_built) return ED_OK;
  ED_DEVICE_SCOPE(c->device);
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
    db.has_hA = ha.rowptr[c->A.start[b.s] + b.dA] != ha.rowptr[c->A.start[b.s]] ? 1 : 0;
    db.pad_ = 0;
    c->h_blocks.push_back(db);
    rs.push_back(b.row0);
  }
  rs.push_back(c->n_rows);
  ED_TRY(upload(c, &c->d_blocks, c->h_blocks));
  ED_TRY(upload(c, &c->d_row_start, rs));
  {
    std::vector<long long> g2;
    long long acc = 0;
    for (const Block& b : c->blocks) {
      g2.push_back(acc);
      acc += (b.dA + 1) / 2;
    }
    g2.push_back(acc);
    c->n_grp2 = acc;
    ED_TRY(upload(c, &c->d_grp2_start, g2));
    std::vector<long long> g4;
    acc = 0;
    for (const Block& b : c->blocks) {
      g4.push_back(acc);
      acc += (b.dA + 3) / 4;
    }
    g4.push_back(acc);
    c->n_grp4 = acc;
    ED_TRY(upload(c, &c->d_grp4_start, g4));
  }
  c->h_cross.clear();
  for (const auto& cb : c->cross) c->h_cross.push_back(DevCross{cb.ia, cb.ib, cb.coef});
  ED_TRY(upload(c, &c->d_cross, c->h_cross));
  // H_A work items: block by block, column panel by column panel, 8 rows each
  {
    std::vector<int4> items;
    const int panel_cols = 256, panel_rows = 8;
    for (size_t bi = 0; bi < c->blocks.size(); ++bi) {
      const Block& b = c->blocks[bi];
      const int64_t r0 = c->A.start[b.s];
      if (ha.rowptr[r0 + b.dA] == ha.rowptr[r0]) continue;  // no H_A entries in this sector
      for (int64_t col = 0; col < b.dB; col += panel_cols)
        for (int64_t a = 0; a < b.dA; a += panel_rows)
          items.push_back(make_int4((int)bi, (int)col, (int)a, (int)std::min<int64_t>(panel_rows, b.dA - a)));
    }
    c->n_panel_items = (long long)items.size();
    ED_TRY(upload(c, &c->d_panel_items, items));
  }
  {
    std::vector<int> z(4, 0);
    ED_TRY(upload(c, &c->d_err, z));
  }
  ED_TRY(build_v3(c, ha, hb));
  c->ops_flags = flags;
  c->ops_built = true;
  return ED_OK;
}
