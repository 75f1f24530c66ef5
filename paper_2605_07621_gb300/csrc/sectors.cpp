// Sector/block structure of the entanglement-cut representation (paper
// Eqs. (2)-(3)): the charges s on side A and N - s on side B of each block,
// the side states of every charge in ascending bit-string order with their
// combinadic ranks, block dimensions d_A(s) x d_B(s) and vector offsets.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "ed_internal.h"

namespace edk {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int64_t binom(int n, int k) {
  if (k < 0 || k > n || n < 0) return 0;
  if (k > n - k) k = n - k;
  int64_t r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

int64_t combinadic_rank(uint64_t x) {
  int64_t r = 0;
  int j = 0;
  while (x) {
    int p = __builtin_ctzll(x);
    r += binom(p, j + 1);
    ++j;
    x &= x - 1;
  }
  return r;
}

ed_status dev_alloc(ed_ctx* c, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? ED_ENOMEM : ED_ECUDA;
  }
  c->dev_allocs.push_back(*p);
  c->dev_bytes += (int64_t)bytes;
  return ED_OK;
}

uint64_t state_key(const ed_ctx* c, uint32_t a, uint32_t b) {
  if (c->kind == ED_HUBBARD) return (uint64_t)a | ((uint64_t)b << c->n_sites);
  uint64_t k = 0;
  for (int p = 0; p < c->A.n; ++p)
    if ((a >> p) & 1u) k |= 1ULL << c->A.sites[p];
  for (int q = 0; q < c->B.n; ++q)
    if ((b >> q) & 1u) k |= 1ULL << c->B.sites[q];
  return k;
}

// all n-bit strings of popcount k in ascending order (Gosper's next-combination step)
static void list_strings(int n, int k, std::vector<uint32_t>& out) {
  if (k == 0) {
    out.push_back(0u);
    return;
  }
  uint64_t v = (1ULL << k) - 1, lim = 1ULL << n;
  while (v < lim) {
    out.push_back((uint32_t)v);
    uint64_t t = v | (v - 1);
    v = (t + 1) | (((~t & (t + 1)) - 1) >> (__builtin_ctzll(v) + 1));
  }
}

static void build_side(Side& sd, int n, const std::vector<int>& sites, const std::vector<char>& used) {
  sd.n = n;
  sd.sites = sites;
  sd.used = used;
  sd.start.assign(n + 2, 0);
  sd.states.clear();
  for (int k = 0; k <= n; ++k) {
    sd.start[k] = (int64_t)sd.states.size();
    if (used[k]) list_strings(n, k, sd.states);
  }
  sd.start[n + 1] = (int64_t)sd.states.size();
}

// Side-local bit order of a spin model's two sides.  On side B the sites
// on a cross-cut bond take the high bits: the columns with one
// configuration of those sites are then a contiguous run, and flipping one
// of them maps the run onto a run of the neighbouring block shifted as a
// whole, so the cross-term gathers of consecutive columns read consecutive
// elements.  On side A they take the low bits: consecutive rows then differ
// at the cut sites and a row group often shares cross-term source rows.
void order_spin_sides(const ed_model_desc* m, std::vector<int>& sitesA, std::vector<int>& sitesB) {
  const int n = m->n_sites;
  std::vector<char> atCut(n, 0), inA(n, 0);
  for (int i = 0; i < n; ++i) inA[i] = (char)((m->cut_mask >> i) & 1ULL);
  for (int b = 0; b < m->n_bonds; ++b) {
    const int i = m->bi[b], j = m->bj[b];
    if (inA[i] != inA[j]) atCut[i] = atCut[j] = 1;
  }
  sitesA.clear();
  sitesB.clear();
  for (int pass = 0; pass < 2; ++pass)
    for (int i = 0; i < n; ++i) {
      if (inA[i] && atCut[i] == 1 - pass) sitesA.push_back(i);
      if (!inA[i] && atCut[i] == pass) sitesB.push_back(i);
    }
}

}  // namespace edk

using namespace edk;

ed_ctx::~ed_ctx() {
  for (void* p : dev_allocs) cudaFree(p);
  if (h_pinned) cudaFreeHost(h_pinned);
  if (lz_stream) cudaStreamDestroy(lz_stream);
}

extern "C" const char* ed_last_error(void) { return edk::g_err; }

static ed_status validate(const ed_model_desc* m) {
  if (!m) { set_error("model is NULL"); return ED_EINVAL; }
  if (m->kind != ED_SPIN && m->kind != ED_HUBBARD) { set_error("unknown model kind %d", m->kind); return ED_EINVAL; }
  int maxn = m->kind == ED_SPIN ? 64 : 32;
  if (m->n_sites < 1 || m->n_sites > maxn) { set_error("n_sites=%d outside 1..%d", m->n_sites, maxn); return ED_EINVAL; }
  if (m->n_bonds < 0 || (m->n_bonds > 0 && (!m->bi || !m->bj))) { set_error("bad bond arrays"); return ED_EINVAL; }
  for (int b = 0; b < m->n_bonds; ++b) {
    int i = m->bi[b], j = m->bj[b];
    if (i < 0 || j < 0 || i >= m->n_sites || j >= m->n_sites || i == j) {
      set_error("bond %d = (%d,%d) invalid for %d sites", b, i, j, m->n_sites);
      return ED_EINVAL;
    }
  }
  if (m->n_up < 0 || m->n_up > m->n_sites) { set_error("n_up=%d outside 0..%d", m->n_up, m->n_sites); return ED_EINVAL; }
  if (m->kind == ED_HUBBARD) {
    if (m->n_dw < 0 || m->n_dw > m->n_sites) { set_error("n_dw=%d outside 0..%d", m->n_dw, m->n_sites); return ED_EINVAL; }
    if (!m->spin_cut) { set_error("Hubbard models need the spin-up|spin-down cut (spin_cut=1)"); return ED_EUNSUPPORTED; }
    if (m->n_sites > kMaxSideBits) { set_error("Hubbard side of %d bits exceeds %d", m->n_sites, kMaxSideBits); return ED_EUNSUPPORTED; }
  } else {
    if (m->n_sites < 64 && (m->cut_mask >> m->n_sites) != 0) { set_error("cut_mask has bits beyond n_sites"); return ED_EINVAL; }
  }
  return ED_OK;
}

extern "C" ed_status ed_build_sectors(const ed_model_desc* m, ed_ctx** out) {
  if (!out) { set_error("out is NULL"); return ED_EINVAL; }
  *out = nullptr;
  ED_TRY(validate(m));
  ed_ctx* c = new (std::nothrow) ed_ctx();
  if (!c) { set_error("host allocation failed"); return ED_ENOMEM; }
  c->kind = m->kind;
  c->n_sites = m->n_sites;
  c->n_up = m->n_up;
  c->n_dw = m->n_dw;
  c->cut_mask = m->cut_mask;
  c->spin_cut = m->spin_cut;
  int nb = m->n_bonds, n = m->n_sites;
  c->bi.assign(m->bi, m->bi + nb);
  c->bj.assign(m->bj, m->bj + nb);
  auto copy_or_zero = [](const double* p, int cnt) {
    std::vector<double> v(cnt, 0.0);
    if (p) std::memcpy(v.data(), p, sizeof(double) * cnt);
    return v;
  };
  c->jxy = copy_or_zero(m->jxy, nb);
  c->jz = copy_or_zero(m->jz, nb);
  c->t = copy_or_zero(m->t, nb);
  c->U = copy_or_zero(m->U, n);
  c->eps = copy_or_zero(m->eps, n);

  std::vector<int> sitesA, sitesB, local(n, -1);
  std::vector<char> sideOf(n, 0);  // 0 = A, 1 = B
  if (c->kind == ED_SPIN) {
    order_spin_sides(m, sitesA, sitesB);
    for (size_t p = 0; p < sitesA.size(); ++p) { local[sitesA[p]] = (int)p; sideOf[sitesA[p]] = 0; }
    for (size_t q = 0; q < sitesB.size(); ++q) { local[sitesB[q]] = (int)q; sideOf[sitesB[q]] = 1; }
  } else {
    for (int i = 0; i < n; ++i) { sitesA.push_back(i); sitesB.push_back(i); local[i] = i; }
  }
  int nA = (int)sitesA.size(), nB = (int)sitesB.size();
  if (nA > kMaxSideBits || nB > kMaxSideBits) {
    set_error("cut sides of %d|%d sites exceed %d", nA, nB, kMaxSideBits);
    delete c;
    return ED_EUNSUPPORTED;
  }
  // charges of the blocks: q_l + q_r = q
  std::vector<std::pair<int, int>> charges;
  if (c->kind == ED_SPIN) {
    int lo = std::max(0, m->n_up - nB), hi = std::min(nA, m->n_up);
    for (int s = lo; s <= hi; ++s) charges.push_back({s, m->n_up - s});
  } else {
    charges.push_back({m->n_up, m->n_dw});
  }
  std::vector<char> usedA(nA + 1, 0), usedB(nB + 1, 0);
  int64_t stA = 0, stB = 0;
  for (auto& q : charges) {
    usedA[q.first] = 1;
    usedB[q.second] = 1;
  }
  for (int k = 0; k <= nA; ++k) if (usedA[k]) stA += binom(nA, k);
  for (int k = 0; k <= nB; ++k) if (usedB[k]) stB += binom(nB, k);
  if (stA > (1LL << 28) || stB > (1LL << 28)) {
    set_error("side state count %lld|%lld exceeds 2^28", (long long)stA, (long long)stB);
    delete c;
    return ED_EUNSUPPORTED;
  }
  build_side(c->A, nA, sitesA, usedA);
  build_side(c->B, nB, sitesB, usedB);

  int64_t off = 0, row = 0;
  c->block_of_s.assign(nA + 1, -1);
  for (auto& q : charges) {
    Block bl;
    bl.s = q.first;
    bl.kB = q.second;
    bl.dA = c->A.dim(q.first);
    bl.dB = c->B.dim(q.second);
    bl.off = off;
    bl.gA0 = c->A.start[q.first];
    bl.gB0 = c->B.start[q.second];
    bl.row0 = row;
    c->block_of_s[q.first] = (int)c->blocks.size();
    c->blocks.push_back(bl);
    off += bl.dA * bl.dB;
    row += bl.dA;
  }
  c->D = off;
  c->n_rows = row;

  // bonds by side (side-local bits)
  c->bondsA.clear();
  c->bondsB.clear();
  c->cross.clear();
  if (c->kind == ED_SPIN) {
    for (int b = 0; b < nb; ++b) {
      int i = m->bi[b], j = m->bj[b];
      double off_el = 0.5 * c->jxy[b];
      if (sideOf[i] == sideOf[j]) {
        ed_ctx::SideBond sb{local[i], local[j], off_el, c->jz[b]};
        (sideOf[i] == 0 ? c->bondsA : c->bondsB).push_back(sb);
      } else {
        int ia = sideOf[i] == 0 ? i : j, jb = sideOf[i] == 0 ? j : i;
        CrossBond cb{local[ia], local[jb], -1, -1, off_el, c->jz[b]};
        c->cross.push_back(cb);
      }
    }
  } else {
    for (int b = 0; b < nb; ++b) {
      ed_ctx::SideBond sb{m->bi[b], m->bj[b], -c->t[b], 0.0};
      c->bondsA.push_back(sb);
      c->bondsB.push_back(sb);
    }
  }
  if ((int)c->cross.size() > kMaxCross) {
    set_error("%d cross-cut bonds exceed %d", (int)c->cross.size(), kMaxCross);
    delete c;
    return ED_EUNSUPPORTED;
  }
  for (auto& cb : c->cross) {
    auto fa = std::find(c->crossA_bits.begin(), c->crossA_bits.end(), cb.p);
    if (fa == c->crossA_bits.end()) { cb.ia = (int)c->crossA_bits.size(); c->crossA_bits.push_back(cb.p); }
    else cb.ia = (int)(fa - c->crossA_bits.begin());
    auto fb = std::find(c->crossB_bits.begin(), c->crossB_bits.end(), cb.q);
    if (fb == c->crossB_bits.end()) { cb.ib = (int)c->crossB_bits.size(); c->crossB_bits.push_back(cb.q); }
    else cb.ib = (int)(fb - c->crossB_bits.begin());
  }
  // bond k is bit k of the packed cross words; order the bonds by their B
  // site (then A site) so that the bonds of one B site are a contiguous bit
  // range and a kernel loads each B-side map entry once per column
  std::stable_sort(c->cross.begin(), c->cross.end(), [](const CrossBond& x, const CrossBond& y) {
    return x.ib != y.ib ? x.ib < y.ib : x.ia < y.ia;
  });
  // diagonal cross term V_AB(a,b) as weighted popcounts of packed bit words
  DevDiagParams dp{};
  if (c->kind == ED_SPIN) {
    // sum_k jz_k/4 (1 - 2[a_p != b_q]) = c0 - sum_classes (jz_c/2) popc((pa^pb) & mask_c)
    dp.vab_and = 0;
    for (size_t k = 0; k < c->cross.size(); ++k) {
      double jz = c->cross[k].jz;
      dp.c0 += 0.25 * jz;
      if (jz == 0.0) continue;
      int cl = -1;
      for (int q = 0; q < dp.ncls; ++q) if (dp.w[q] == -0.5 * jz) cl = q;
      if (cl < 0) {
        if (dp.ncls == kMaxClasses) { set_error("more than %d distinct cross jz values", kMaxClasses); delete c; return ED_EUNSUPPORTED; }
        cl = dp.ncls++;
        dp.w[cl] = -0.5 * jz;
      }
      dp.mask[cl] |= 1ULL << k;
    }
  } else {
    // sum_i U_i [up_i and dw_i] = sum_classes U_c popc(a & b & mask_c)
    dp.vab_and = 1;
    for (int i = 0; i < n; ++i) {
      double u = c->U[i];
      if (u == 0.0) continue;
      int cl = -1;
      for (int q = 0; q < dp.ncls; ++q) if (dp.w[q] == u) cl = q;
      if (cl < 0) {
        if (dp.ncls == kMaxClasses) { set_error("more than %d distinct U values", kMaxClasses); delete c; return ED_EUNSUPPORTED; }
        cl = dp.ncls++;
        dp.w[cl] = u;
      }
      dp.mask[cl] |= 1ULL << i;
    }
  }
  c->diag = dp;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); dev = 0; }
  c->device = dev;
  *out = c;
  return ED_OK;
}

extern "C" int64_t ed_dim(const ed_ctx* c) { return c ? c->D : -1; }
extern "C" int ed_num_blocks(const ed_ctx* c) { return c ? (int)c->blocks.size() : -1; }

extern "C" ed_status ed_blocks(const ed_ctx* c, int* s, int64_t* dA, int64_t* dB, int64_t* off) {
  if (!c) { set_error("ctx is NULL"); return ED_EINVAL; }
  for (size_t i = 0; i < c->blocks.size(); ++i) {
    if (s) s[i] = c->blocks[i].s;
    if (dA) dA[i] = c->blocks[i].dA;
    if (dB) dB[i] = c->blocks[i].dB;
    if (off) off[i] = c->blocks[i].off;
  }
  return ED_OK;
}

extern "C" ed_status ed_state_keys(const ed_ctx* c, int64_t start, int64_t count, uint64_t* keys) {
  if (!c || !keys || start < 0 || count < 0 || start + count > c->D) {
    set_error("ed_state_keys: bad arguments");
    return ED_EINVAL;
  }
  size_t bi = 0;
  for (int64_t g = start; g < start + count; ++g) {
    while (bi + 1 < c->blocks.size() && c->blocks[bi + 1].off <= g) ++bi;
    while (bi > 0 && c->blocks[bi].off > g) --bi;
    const Block& bl = c->blocks[bi];
    int64_t loc = g - bl.off;
    int64_t r = loc / bl.dB, col = loc % bl.dB;
    keys[g - start] = state_key(c, c->A.states[bl.gA0 + r], c->B.states[bl.gB0 + col]);
  }
  return ED_OK;
}

extern "C" ed_status ed_side_sites(const ed_ctx* c, int side, int* sites, int* n_bits) {
  if (!c || !sites || !n_bits || (side != 0 && side != 1)) {
    set_error("ed_side_sites: bad arguments");
    return ED_EINVAL;
  }
  const Side& sd = side == 0 ? c->A : c->B;
  for (int p = 0; p < sd.n; ++p) sites[p] = sd.sites[p];
  *n_bits = sd.n;
  return ED_OK;
}

extern "C" int64_t ed_device_bytes(const ed_ctx* c) { return c ? c->dev_bytes : -1; }

extern "C" void ed_destroy(ed_ctx* c) { delete c; }
