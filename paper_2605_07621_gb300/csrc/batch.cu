// Batched Lanczos engine (see batch.h).  Kernels take the active set from
// device memory (count, instance list, row and chunk prefix sums), so one
// captured graph of the Lanczos step stays valid while instances join and
// leave between replays.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>

#include <array>
#include <map>
#include <mutex>

#include "batch.h"
#include "batch_dev.cuh"
#include "krylov.h"
#include "ozaki.h"
#include "reduce.cuh"
#include "splitmix.cuh"

namespace edk {

constexpr int kBW = 8;          // warps per CTA in the apply kernel
constexpr int kBStage = 1024;   // row elements staged in shared memory per warp

// y = H x for the active instances in CSR mode; one warp per row a (lanes
// over b).  user_mode: x, y are a caller's concatenated vectors (offset
// uoff); otherwise v -> w inside each instance's arena triple.
__global__ void __launch_bounds__(256) k_bapply(const BInst* __restrict__ insts, const int* __restrict__ idx,
                                                const long long* __restrict__ rowpref, const int* __restrict__ cnt,
                                                const float* __restrict__ ux, float* __restrict__ uy, float* arena,
                                                int user_mode) {
  __shared__ float stage[kBW][kBStage];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = cnt[0];
  if (n <= 0) return;
  const long long total = rowpref[n];
  for (long long row = (long long)blockIdx.x * kBW + warp; row < total; row += (long long)gridDim.x * kBW) {
    const int ai = find_pref(rowpref, n, row);
    const BInst& I = insts[idx[ai]];
    const long long a = row - rowpref[ai];
    // the instance's fields in registers (y stores could alias them otherwise)
    const int dB = I.dB;
    const float* __restrict__ x = user_mode ? ux + I.uoff : arena + I.voff + I.D;
    float* __restrict__ y = user_mode ? uy + I.uoff : arena + I.voff + 2 * I.D;
    const int* __restrict__ Brp = I.B_rp;
    const int* __restrict__ Bcol = I.B_col;
    const float* __restrict__ Bval = I.B_val;
    const float* __restrict__ Bd = I.B_diag;
    const uint32_t* __restrict__ Bs = I.B_str;
    const int* __restrict__ Acol = I.A_col;
    const float* __restrict__ Aval = I.A_val;
    const int ncls = I.ncls, vand = I.vab_and;
    float w[kMaxClasses];
    unsigned mk[kMaxClasses];
#pragma unroll
    for (int q = 0; q < kMaxClasses; ++q) {
      w[q] = I.w[q];
      mk[q] = I.mask[q];
    }
    const float* xrow = x + a * dB;
    const bool staged = dB <= kBStage;
    if (staged) {
      for (int b = lane; b < dB; b += 32) stage[warp][b] = xrow[b];
      __syncwarp();
    }
    const float* xs = staged ? stage[warp] : xrow;
    const float da = I.A_diag[a] + I.c0;
    const uint32_t sa = I.A_str[a];
    const int ea0 = I.A_rp[a], ea1 = I.A_rp[a + 1];
    for (int b = lane; b < dB; b += 32) {
      const uint32_t sb = Bs[b];
      const uint32_t z = vand ? (sa & sb) : (sa ^ sb);
      float v = da + Bd[b];
      for (int q = 0; q < ncls; ++q) v += w[q] * (float)__popc(z & mk[q]);
      float acc = v * xs[b];
      const int eb0 = Brp[b], eb1 = Brp[b + 1];
      for (int e = eb0; e < eb1; ++e) acc += Bval[e] * xs[Bcol[e]];
      for (int e = ea0; e < ea1; ++e) acc += Aval[e] * x[(long long)Acol[e] * dB + b];
      y[a * dB + b] = acc;
    }
    __syncwarp();
  }
}

// chunk c of the active set -> (instance, element range)
struct ChunkRef {
  int slot;
  long long i0, i1;
};
__device__ __forceinline__ ChunkRef chunk_of(const BInst* insts, const int* idx, const long long* chunkpref, int n,
                                             long long c) {
  const int ai = find_pref(chunkpref, n, c);
  ChunkRef r;
  r.slot = idx[ai];
  const long long D = insts[r.slot].D;
  r.i0 = (c - chunkpref[ai]) * kBatchChunk;
  r.i1 = min(D, r.i0 + kBatchChunk);
  return r;
}

// w -= beta vprev; part[c] = <v, w>
__global__ void k_blz_a(const BInst* __restrict__ insts, const int* __restrict__ idx,
                        const long long* __restrict__ chunkpref, const int* __restrict__ nact, float* arena,
                        const double* __restrict__ beta, double* part) {
  const int n = *nact;
  if (n <= 0) return;
  const long long total = chunkpref[n];
  for (long long c = blockIdx.x; c < total; c += gridDim.x) {
    const ChunkRef r = chunk_of(insts, idx, chunkpref, n, c);
    const BInst& I = insts[r.slot];
    float* vp = arena + I.voff;
    float* v = vp + I.D;
    float* w = v + I.D;
    const float bt = (float)beta[r.slot];
    FAcc acc;
    for (long long i = r.i0 + threadIdx.x; i < r.i1; i += blockDim.x) {
      const float wi = w[i] - bt * vp[i];
      w[i] = wi;
      acc.add_prod(v[i], wi);
    }
    const double s = block_sum(acc.value());
    if (threadIdx.x == 0) part[c] = s;
  }
}

// w -= alpha v; part[c] = ||w||^2
__global__ void k_blz_b(const BInst* __restrict__ insts, const int* __restrict__ idx,
                        const long long* __restrict__ chunkpref, const int* __restrict__ nact, float* arena,
                        const double* __restrict__ alpha, double* part) {
  const int n = *nact;
  if (n <= 0) return;
  const long long total = chunkpref[n];
  for (long long c = blockIdx.x; c < total; c += gridDim.x) {
    const ChunkRef r = chunk_of(insts, idx, chunkpref, n, c);
    const BInst& I = insts[r.slot];
    float* v = arena + I.voff + I.D;
    float* w = v + I.D;
    const float al = (float)alpha[r.slot];
    FAcc acc;
    for (long long i = r.i0 + threadIdx.x; i < r.i1; i += blockDim.x) {
      const float wi = w[i] - al * v[i];
      w[i] = wi;
      acc.add_prod(wi, wi);
    }
    const double s = block_sum(acc.value());
    if (threadIdx.x == 0) part[c] = s;
  }
}

// vprev <- v; v <- w / beta
__global__ void k_blz_c(const BInst* __restrict__ insts, const int* __restrict__ idx,
                        const long long* __restrict__ chunkpref, const int* __restrict__ nact, float* arena,
                        const double* __restrict__ beta) {
  const int n = *nact;
  if (n <= 0) return;
  const long long total = chunkpref[n];
  for (long long c = blockIdx.x; c < total; c += gridDim.x) {
    const ChunkRef r = chunk_of(insts, idx, chunkpref, n, c);
    const BInst& I = insts[r.slot];
    float* vp = arena + I.voff;
    float* v = vp + I.D;
    const float* w = v + I.D;
    const double b = beta[r.slot];
    const float inv = (float)(b > 0.0 ? 1.0 / b : 0.0);
    for (long long i = r.i0 + threadIdx.x; i < r.i1; i += blockDim.x) {
      vp[i] = v[i];
      v[i] = w[i] * inv;
    }
  }
}

// per active instance: sum its chunk partials (fixed order) into out[slot];
// op 0 -> alpha (kept in hist_a), op 1 -> beta = sqrt (kept in hist_b)
__global__ void k_bfin(const BInst* __restrict__ insts, const int* __restrict__ idx,
                       const long long* __restrict__ chunkpref, const int* __restrict__ nact,
                       const double* __restrict__ part, double* out, const int* __restrict__ it, int max_iter, int op) {
  const int n = *nact;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int ai = warp; ai < n; ai += nw) {
    double s = 0.0;
    for (long long c = chunkpref[ai] + lane; c < chunkpref[ai + 1]; c += 32) s += part[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) {
      const int slot = idx[ai];
      const double val = op ? sqrt(s > 0.0 ? s : 0.0) : s;
      out[slot] = val;
      const int j = it[slot];
      if (j < max_iter) (op ? insts[slot].hist_b : insts[slot].hist_a)[j] = val;
    }
  }
}

__global__ void k_bstep(const int* __restrict__ idx, const int* __restrict__ nact, int* it) {
  const int n = *nact;
  for (int ai = blockIdx.x * blockDim.x + threadIdx.x; ai < n; ai += gridDim.x * blockDim.x) ++it[idx[ai]];
}

// start vector of one instance (key = up | dw << n_sites) and cleared history
__global__ void k_binit(BInst I, unsigned long long seed, float* arena) {
  float* vp = arena + I.voff;
  float* v = vp + I.D;
  float* w = v + I.D;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < I.D; i += (long long)gridDim.x * blockDim.x) {
    const long long a = i / I.dB, b = i % I.dB;
    const unsigned long long key = (unsigned long long)I.A_str[a] | ((unsigned long long)I.B_str[b] << I.n_sites);
    v[i] = (float)splitmix_value(seed, key);
    vp[i] = 0.f;
    w[i] = 0.f;
  }
}

__global__ void k_bsumsq(const float* __restrict__ v, long long n, double* part) {
  FAcc acc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc.add_prod(v[i], v[i]);
  const double s = block_sum(acc.value());
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_bscale(float* v, long long n, const double* __restrict__ part, int np) {
  __shared__ double inv;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < np; ++i) s += part[i];
    inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
  }
  __syncthreads();
  const float f = (float)inv;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    v[i] *= f;
}

// ---------------------------------------------------------------- host

namespace {
struct HostTables {
  int64_t dA = 0, dB = 0;
  int n_sites = 0;
  std::vector<int> A_rp, A_col, B_rp, B_col;
  std::vector<float> A_val, B_val, A_diag, B_diag;
  std::vector<uint32_t> A_str, B_str;
  float c0 = 0.f;
  int ncls = 0, vab_and = 0;
  float w[kMaxClasses] = {};
  unsigned mask[kMaxClasses] = {};
};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }
// row stride of the BF16 pieces: 64 elements (128 bytes), so every row a
// TMA box reads starts on a 128-byte line
int pad64(int64_t d) { return (int)((d + 63) / 64 * 64); }

ed_status host_tables(const ed_model_desc& m, HostTables& h) {
  if (m.kind != ED_HUBBARD || !m.spin_cut) {
    set_error("batched instances must be Hubbard models with the spin cut");
    return ED_EUNSUPPORTED;
  }
  ed_ctx* c = nullptr;
  ED_TRY(ed_build_sectors(&m, &c));
  std::unique_ptr<ed_ctx, void (*)(ed_ctx*)> guard(c, ed_destroy);
  if (c->blocks.size() != 1) {
    set_error("batched instance must have one block");
    return ED_EUNSUPPORTED;
  }
  const Block& bl = c->blocks[0];
  if (bl.dA > (1 << 20) || bl.dB > (1 << 20)) {
    set_error("batched instance too large");
    return ED_EUNSUPPORTED;
  }
  HostSideOps ha, hb;
  ED_TRY(build_side_ops(c, c->A, c->bondsA, true, ha));
  ED_TRY(build_side_ops(c, c->B, c->bondsB, false, hb));
  h.dA = bl.dA;
  h.dB = bl.dB;
  h.n_sites = c->n_sites;
  auto side = [](const HostSideOps& s, const Side& sd, int k, std::vector<int>& rp, std::vector<int>& col,
                 std::vector<float>& val, std::vector<float>& diag, std::vector<uint32_t>& str) {
    const int64_t g0 = sd.start[k], g1 = sd.start[k + 1];
    const int base = s.rowptr[g0];
    for (int64_t g = g0; g <= g1; ++g) rp.push_back(s.rowptr[g] - base);
    for (int e = s.rowptr[g0]; e < s.rowptr[g1]; ++e) {
      col.push_back(s.col[e]);
      val.push_back((float)s.val64[e]);
    }
    for (int64_t g = g0; g < g1; ++g) {
      diag.push_back((float)s.diag[g]);
      str.push_back(sd.states[g]);
    }
  };
  side(ha, c->A, bl.s, h.A_rp, h.A_col, h.A_val, h.A_diag, h.A_str);
  side(hb, c->B, bl.kB, h.B_rp, h.B_col, h.B_val, h.B_diag, h.B_str);
  h.c0 = (float)c->diag.c0;
  h.ncls = c->diag.ncls;
  h.vab_and = c->diag.vab_and;
  for (int q = 0; q < h.ncls; ++q) {
    h.w[q] = (float)c->diag.w[q];
    h.mask[q] = (unsigned)c->diag.mask[q];
  }
  return ED_OK;
}

bool dense_capable(const HostTables& h) { return h.dA <= kBDenseMax && h.dB <= kBDenseMax; }

// bytes of the CSR tables (uploaded), then of the dense form: the pieces of
// H_A, H_B (uploaded) and of Psi, Psi^T (written by every apply)
size_t csr_bytes(const HostTables& h) {
  size_t b = 0;
  b += align256(h.A_rp.size() * 4) + align256(h.A_col.size() * 4) + align256(h.A_val.size() * 4);
  b += align256(h.A_diag.size() * 4) + align256(h.A_str.size() * 4);
  b += align256(h.B_rp.size() * 4) + align256(h.B_col.size() * 4) + align256(h.B_val.size() * 4);
  b += align256(h.B_diag.size() * 4) + align256(h.B_str.size() * 4);
  return b;
}
// words of the nonzero-K-block masks: 128-row tiles of H_A, 64- and 128-row tiles of H_B
size_t kmask_words(const HostTables& h) {
  return (size_t)((h.dA + 127) / 128 + (h.dB + 63) / 64 + (h.dB + 127) / 128);
}
size_t h_piece_bytes(const HostTables& h) {
  return align256((size_t)3 * h.dA * pad64(h.dA) * 2) + align256((size_t)3 * h.dB * pad64(h.dB) * 2) +
         align256(kmask_words(h) * 4);
}
size_t x_piece_bytes(const HostTables& h) {
  return align256((size_t)3 * h.dA * pad64(h.dB) * 2) + align256((size_t)3 * h.dB * pad64(h.dA) * 2);
}
size_t tables_bytes(const HostTables& h, bool dense) {
  size_t b = align256((size_t)3 * h.dA * h.dB * 4) + csr_bytes(h);
  if (dense && dense_capable(h)) b += h_piece_bytes(h) + x_piece_bytes(h);
  return b;
}

// chosen mode per instance shape, shared by every engine of the process
using ShapeKey = std::array<long long, 4>;
std::mutex g_mode_mu;
std::map<ShapeKey, int> g_mode_cache;

bool cached_mode(const long long* key, int* mode) {
  std::lock_guard<std::mutex> lk(g_mode_mu);
  auto it = g_mode_cache.find(ShapeKey{key[0], key[1], key[2], key[3]});
  if (it == g_mode_cache.end()) return false;
  *mode = it->second;
  return true;
}
void cache_mode(const long long* key, int mode) {
  std::lock_guard<std::mutex> lk(g_mode_mu);
  g_mode_cache[ShapeKey{key[0], key[1], key[2], key[3]}] = mode;
}
}  // namespace

BatchEngine::~BatchEngine() {
  if (exec_) cudaGraphExecDestroy(exec_);
  if (graph_) cudaGraphDestroy(graph_);
  for (void* p : dev_) cudaFree(p);
  if (st_) cudaStreamDestroy(st_);
}

ed_status BatchEngine::init(int device, size_t arena_bytes, int max_slots, int max_iter, bool dense) {
  device_ = device;
  ED_DEVICE_SCOPE(device);
  if (cudaDeviceGetAttribute(&sms_, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    sms_ = 148;
  }
  ED_CUDA_TRY(cudaStreamCreateWithFlags(&st_, cudaStreamNonBlocking));
  dense_ = dense;
  if (dense_) ED_TRY(bdense_prepare());
  max_slots_ = std::max(1, max_slots);
  max_iter_ = std::max(2, max_iter);
  list_cap_ = max_slots_ + 4096;  // the tuner's replicated lists are longer than the slot count
  arena_bytes_ = align256(std::max<size_t>(arena_bytes, 1 << 20));
  auto get = [&](void** p, size_t bytes) -> ed_status {
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("batch engine: cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
      return ED_ENOMEM;
    }
    dev_.push_back(*p);
    return ED_OK;
  };
  ED_TRY(get((void**)&arena_, arena_bytes_));
  free_.assign(1, {0, arena_bytes_});
  slots_.assign(max_slots_, BSlot{});
  ED_TRY(get((void**)&d_inst_, sizeof(BInst) * max_slots_));
  ED_CUDA_TRY(cudaMemset(d_inst_, 0, sizeof(BInst) * max_slots_));
  ED_TRY(get((void**)&d_idx_, sizeof(int) * max_slots_));
  ED_TRY(get((void**)&d_chunkpref_, sizeof(long long) * (max_slots_ + 1)));
  ED_TRY(get((void**)&d_nact_, sizeof(int) * 4));
  ED_TRY(get((void**)&d_cnt_, sizeof(int) * 4));
  ED_TRY(get((void**)&d_cidx_, sizeof(int) * list_cap_));
  ED_TRY(get((void**)&d_crowpref_, sizeof(long long) * (list_cap_ + 1)));
  ED_TRY(get((void**)&d_didx_, sizeof(int) * list_cap_));
  ED_TRY(get((void**)&d_dspref_, sizeof(long long) * (list_cap_ + 1)));
  ED_TRY(get((void**)&d_idx64_, sizeof(int) * list_cap_));
  ED_TRY(get((void**)&d_tpref64_, sizeof(long long) * (list_cap_ + 1)));
  ED_TRY(get((void**)&d_idx128_, sizeof(int) * list_cap_));
  ED_TRY(get((void**)&d_tpref128_, sizeof(long long) * (list_cap_ + 1)));
  ED_TRY(get((void**)&d_maps_, sizeof(CUtensorMap) * kBMaps * (size_t)max_slots_));
  ED_TRY(get((void**)&d_err_, sizeof(int) * 4));
  ED_CUDA_TRY(cudaMemset(d_err_, 0, sizeof(int) * 4));
  ED_TRY(get((void**)&d_it_, sizeof(int) * max_slots_));
  ED_TRY(get((void**)&d_alpha_, sizeof(double) * max_slots_));
  ED_TRY(get((void**)&d_beta_, sizeof(double) * max_slots_));
  // every element of every instance takes >= 12 arena bytes
  part_cap_ = (long long)(arena_bytes_ / (12 * (size_t)kBatchChunk)) + max_slots_ + 1024;
  ED_TRY(get((void**)&d_part_, sizeof(double) * part_cap_));
  double* hist = nullptr;
  ED_TRY(get((void**)&hist, sizeof(double) * 2 * (size_t)max_slots_ * max_iter_));
  d_hist_ = hist;
  for (int s = 0; s < max_slots_; ++s) {
    slots_[s].d.hist_a = hist + (size_t)s * max_iter_;
    slots_[s].d.hist_b = hist + ((size_t)max_slots_ + s) * max_iter_;
  }
  ED_CUDA_TRY(cudaMemsetAsync(d_nact_, 0, sizeof(int) * 4, st_));
  ED_CUDA_TRY(cudaMemsetAsync(d_it_, 0, sizeof(int) * max_slots_, st_));
  ED_TRY(rebuild_active());
  return capture();
}

bool BatchEngine::alloc(size_t len, size_t* off) {
  len = align256(len);
  for (size_t i = 0; i < free_.size(); ++i) {
    if (free_[i].second >= len) {
      *off = free_[i].first;
      free_[i].first += len;
      free_[i].second -= len;
      if (free_[i].second == 0) free_.erase(free_.begin() + i);
      return true;
    }
  }
  return false;
}

void BatchEngine::release(size_t off, size_t len) {
  len = align256(len);
  free_.push_back({off, len});
  std::sort(free_.begin(), free_.end());
  std::vector<std::pair<size_t, size_t>> merged;
  for (auto& f : free_) {
    if (!merged.empty() && merged.back().first + merged.back().second == f.first) merged.back().second += f.second;
    else merged.push_back(f);
  }
  free_.swap(merged);
}

size_t BatchEngine::arena_free() const {
  size_t s = 0;
  for (auto& f : free_) s += f.second;
  return s;
}

int BatchEngine::active_count() const {
  int n = 0;
  for (auto& s : slots_) n += s.active ? 1 : 0;
  return n;
}

ed_status BatchEngine::instance_bytes(const ed_model_desc& m, bool dense, size_t* bytes, int64_t* dim) {
  HostTables h;
  ED_TRY(host_tables(m, h));
  *bytes = tables_bytes(h, dense);
  if (dim) *dim = h.dA * h.dB;
  return ED_OK;
}

ed_status BatchEngine::add(const ed_model_desc& m, uint64_t seed, int* slot_out, bool commit) {
  // the calling thread may be new to CUDA (the serving worker): make the
  // device's context current for the tensor-map encoding (a driver call)
  ED_DEVICE_SCOPE(device_);
  HostTables h;
  ED_TRY(host_tables(m, h));
  int slot = -1;
  for (int s = 0; s < max_slots_; ++s)
    if (!slots_[s].used) {
      slot = s;
      break;
    }
  if (slot < 0) {
    set_error("batch engine: no free slot");
    return ED_ENOMEM;
  }
  const bool dn = dense_ && dense_capable(h);
  const size_t need = tables_bytes(h, dense_);
  size_t off;
  if (!alloc(need, &off)) {
    set_error("batch engine: instance needs %zu bytes, %zu free", need, arena_free());
    return ED_ENOMEM;
  }
  // lay the instance out in its arena range: three vectors, the CSR tables
  // (uploaded), the dense form's tables (built on the device) and the Psi
  // pieces (scratch)
  const size_t tab0 = align256((size_t)3 * h.dA * h.dB * 4);
  const size_t up_end = tab0 + csr_bytes(h);
  std::vector<char> host(up_end, 0);
  size_t cur = tab0;
  BSlot& S = slots_[slot];
  BInst& d = S.d;
  double* ha = d.hist_a;
  double* hb = d.hist_b;
  d = BInst{};
  d.hist_a = ha;
  d.hist_b = hb;
  auto put = [&](const void* src, size_t bytes) -> void* {
    void* dst = arena_ + off + cur;
    if (bytes && src) std::memcpy(host.data() + cur, src, bytes);
    cur += align256(bytes);
    return dst;
  };
  d.voff = (long long)(off / 4);
  d.D = h.dA * h.dB;
  d.dA = (int)h.dA;
  d.dB = (int)h.dB;
  d.n_sites = h.n_sites;
  d.A_rp = (const int*)put(h.A_rp.data(), h.A_rp.size() * 4);
  d.A_col = (const int*)put(h.A_col.data(), h.A_col.size() * 4);
  d.A_val = (const float*)put(h.A_val.data(), h.A_val.size() * 4);
  d.A_diag = (const float*)put(h.A_diag.data(), h.A_diag.size() * 4);
  d.A_str = (const uint32_t*)put(h.A_str.data(), h.A_str.size() * 4);
  d.B_rp = (const int*)put(h.B_rp.data(), h.B_rp.size() * 4);
  d.B_col = (const int*)put(h.B_col.data(), h.B_col.size() * 4);
  d.B_val = (const float*)put(h.B_val.data(), h.B_val.size() * 4);
  d.B_diag = (const float*)put(h.B_diag.data(), h.B_diag.size() * 4);
  d.B_str = (const uint32_t*)put(h.B_str.data(), h.B_str.size() * 4);
  d.c0 = h.c0;
  d.ncls = h.ncls;
  d.vab_and = h.vab_and;
  for (int q = 0; q < kMaxClasses; ++q) {
    d.w[q] = h.w[q];
    d.mask[q] = h.mask[q];
  }
  S.key[0] = h.dA;
  S.key[1] = h.dB;
  S.key[2] = h.A_rp.back();
  S.key[3] = h.B_rp.back();
  d.mode = kModeCSR;
  if (dn) {
    d.KpA = pad64(h.dA);
    d.KpB = pad64(h.dB);
    d.HA = (const uint16_t*)put(nullptr, (size_t)3 * h.dA * d.KpA * 2);
    d.HB = (const uint16_t*)put(nullptr, (size_t)3 * h.dB * d.KpB * 2);
    d.kmask = (const uint32_t*)put(nullptr, kmask_words(h) * 4);
    d.XN = (uint16_t*)put(nullptr, (size_t)3 * h.dA * d.KpB * 2);
    d.XT = (uint16_t*)put(nullptr, (size_t)3 * h.dB * d.KpA * 2);
    // A-role maps (H_A, Psi) with 128-row boxes; B-role maps (Psi^T, H_B)
    // with 64- and 128-row boxes, one pair per output tile width
    CUtensorMap mp[kBMaps];
    ED_TRY(tmap_bf16_planes(&mp[0], d.HA, d.dA, d.dA, 3, d.KpA, 128));
    ED_TRY(tmap_bf16_planes(&mp[1], d.XN, d.dB, d.dA, 3, d.KpB, 128));
    ED_TRY(tmap_bf16_planes(&mp[2], d.XT, d.dA, d.dB, 3, d.KpA, 64));
    ED_TRY(tmap_bf16_planes(&mp[3], d.HB, d.dB, d.dB, 3, d.KpB, 64));
    ED_TRY(tmap_bf16_planes(&mp[4], d.XT, d.dA, d.dB, 3, d.KpA, 128));
    ED_TRY(tmap_bf16_planes(&mp[5], d.HB, d.dB, d.dB, 3, d.KpB, 128));
    ED_CUDA_TRY(cudaMemcpyAsync(d_maps_ + (size_t)slot * kBMaps, mp, sizeof(mp), cudaMemcpyHostToDevice, st_));
  }
  ED_CUDA_TRY(cudaMemcpyAsync(arena_ + off + tab0, host.data() + tab0, up_end - tab0, cudaMemcpyHostToDevice, st_));
  if (dn) {
    ED_CUDA_TRY(cudaMemsetAsync(arena_ + off + up_end, 0, h_piece_bytes(h), st_));
    ED_TRY(bdense_tables(d, st_));
  }
  S.used = true;
  S.active = false;
  S.alloc_off = off;
  S.alloc_len = need;
  S.dense_ok = dn ? 1 : 0;
  d.mode = dn ? default_mode(S) : kModeCSR;
  // (copies from pageable host memory return once the source has been staged,
  // so the host buffers may go; the stream orders everything after them)
  ED_CUDA_TRY(cudaMemcpyAsync(d_inst_ + slot, &d, sizeof(BInst), cudaMemcpyHostToDevice, st_));
  ED_TRY(restart(slot, seed, commit));
  *slot_out = slot;
  return ED_OK;
}

ed_status BatchEngine::restart(int slot, uint64_t seed, bool commit) {
  BSlot& S = slots_[slot];
  float* arena_f = (float*)arena_;
  const long long n = S.d.D;
  const int g = (int)std::min<long long>((n + 255) / 256, 1024);
  k_binit<<<std::max(g, 1), 256, 0, st_>>>(S.d, seed, arena_f);
  k_bsumsq<<<std::max(g, 1), 256, 0, st_>>>(arena_f + S.d.voff + n, n, d_part_);
  k_bscale<<<std::max(g, 1), 256, 0, st_>>>(arena_f + S.d.voff + n, n, d_part_, std::max(g, 1));
  ED_CUDA_TRY(cudaGetLastError());
  ED_CUDA_TRY(cudaMemsetAsync(d_it_ + slot, 0, sizeof(int), st_));
  ED_CUDA_TRY(cudaMemsetAsync(d_alpha_ + slot, 0, sizeof(double), st_));
  ED_CUDA_TRY(cudaMemsetAsync(d_beta_ + slot, 0, sizeof(double), st_));
  S.active = true;
  S.converged = false;
  S.iters_seen = 0;
  S.theta = S.theta_prev = 0.0;
  return commit ? rebuild_active() : ED_OK;
}

void BatchEngine::remove(int slot, bool commit) {
  BSlot& S = slots_[slot];
  if (!S.used) return;
  const bool was_active = S.active;
  release(S.alloc_off, S.alloc_len);
  S.used = false;
  S.active = false;
  if (commit && was_active) rebuild_active();
}

ed_status BatchEngine::set_mode(int slot, int mode) {
  BSlot& S = slots_[slot];
  if (S.used) S.d.mode = S.dense_ok ? mode : kModeCSR;  // takes effect at the next rebuild_active
  return ED_OK;
}

int BatchEngine::default_mode(const BSlot& S) const {
  int md;
  if (cached_mode(S.key, &md)) return md;
  return S.d.dB <= 64 ? kModeD64 : kModeD128;
}

ed_status BatchEngine::upload_inst(int slot) {
  ED_CUDA_TRY(cudaMemcpyAsync(d_inst_ + slot, &slots_[slot].d, sizeof(BInst), cudaMemcpyHostToDevice, st_));
  ED_CUDA_TRY(cudaStreamSynchronize(st_));
  return ED_OK;
}

ed_status BatchEngine::upload_lists(const std::vector<int>& csr, const std::vector<int>& d64,
                                    const std::vector<int>& d128) {
  if ((int)csr.size() > list_cap_ || (int)(d64.size() + d128.size()) > list_cap_) {
    set_error("batch engine: work list exceeds capacity");
    return ED_ENOMEM;
  }
  std::vector<long long> crp(1, 0), sp(1, 0), tp64(1, 0), tp128(1, 0);
  std::vector<int> dall(d64);
  dall.insert(dall.end(), d128.begin(), d128.end());
  for (int s : csr) crp.push_back(crp.back() + slots_[s].d.dA);
  for (int s : dall) sp.push_back(sp.back() + (long long)((slots_[s].d.dA + 63) / 64) * ((slots_[s].d.dB + 63) / 64));
  for (int s : d64) tp64.push_back(tp64.back() + (long long)((slots_[s].d.dA + 127) / 128) * ((slots_[s].d.dB + 63) / 64));
  for (int s : d128)
    tp128.push_back(tp128.back() + (long long)((slots_[s].d.dA + 127) / 128) * ((slots_[s].d.dB + 127) / 128));
  auto up = [&](void* dst, const void* src, size_t bytes) -> ed_status {
    if (bytes) ED_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st_));
    return ED_OK;
  };
  ED_TRY(up(d_cidx_, csr.data(), csr.size() * 4));
  ED_TRY(up(d_crowpref_, crp.data(), crp.size() * 8));
  ED_TRY(up(d_didx_, dall.data(), dall.size() * 4));
  ED_TRY(up(d_dspref_, sp.data(), sp.size() * 8));
  ED_TRY(up(d_idx64_, d64.data(), d64.size() * 4));
  ED_TRY(up(d_tpref64_, tp64.data(), tp64.size() * 8));
  ED_TRY(up(d_idx128_, d128.data(), d128.size() * 4));
  ED_TRY(up(d_tpref128_, tp128.data(), tp128.size() * 8));
  const int cnt[4] = {(int)csr.size(), (int)dall.size(), (int)d64.size(), (int)d128.size()};
  ED_TRY(up(d_cnt_, cnt, sizeof(cnt)));
  ED_CUDA_TRY(cudaStreamSynchronize(st_));
  return ED_OK;
}

ed_status BatchEngine::rebuild_active() {
  std::vector<int> idx, csr, d64, d128;
  std::vector<long long> cp(1, 0);
  for (int s = 0; s < max_slots_; ++s) {
    const BSlot& S = slots_[s];
    if (!S.used || !S.active) continue;
    idx.push_back(s);
    cp.push_back(cp.back() + (S.d.D + kBatchChunk - 1) / kBatchChunk);
    (S.d.mode == kModeD64 ? d64 : S.d.mode == kModeD128 ? d128 : csr).push_back(s);
  }
  if (cp.back() > part_cap_) {
    set_error("batch engine: reduction chunks exceed capacity");
    return ED_ENOMEM;
  }
  int n = (int)idx.size();
  if (!idx.empty()) ED_CUDA_TRY(cudaMemcpyAsync(d_idx_, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice, st_));
  ED_CUDA_TRY(cudaMemcpyAsync(d_chunkpref_, cp.data(), cp.size() * 8, cudaMemcpyHostToDevice, st_));
  ED_CUDA_TRY(cudaMemcpyAsync(d_nact_, &n, 4, cudaMemcpyHostToDevice, st_));
  return upload_lists(csr, d64, d128);
}

ed_status BatchEngine::launch_apply(cudaStream_t s, const float* x, float* y) {
  const int user = x != nullptr;
  if (dense_) {
    BDenseArgs a;
    a.insts = d_inst_;
    a.cnt = d_cnt_;
    a.didx = d_didx_;
    a.dspref = d_dspref_;
    a.idx64 = d_idx64_;
    a.tpref64 = d_tpref64_;
    a.idx128 = d_idx128_;
    a.tpref128 = d_tpref128_;
    a.maps = d_maps_;
    a.ux = x;
    a.uy = y;
    a.arena = (float*)arena_;
    a.user_mode = user;
    a.sms = sms_;
    a.err = d_err_;
    ED_TRY(bdense_apply(a, s));
  }
  k_bapply<<<sms_ * 4, 256, 0, s>>>(d_inst_, d_cidx_, d_crowpref_, d_cnt_, x, y, (float*)arena_, user);
  ED_CUDA_TRY(cudaGetLastError());
  return ED_OK;
}

ed_status BatchEngine::launch_step(cudaStream_t s) {
  float* arena_f = (float*)arena_;
  const int g_red = sms_ * 4;
  ED_TRY(launch_apply(s, nullptr, nullptr));
  k_blz_a<<<g_red, 256, 0, s>>>(d_inst_, d_idx_, d_chunkpref_, d_nact_, arena_f, d_beta_, d_part_);
  k_bfin<<<(max_slots_ * 32 + 255) / 256, 256, 0, s>>>(d_inst_, d_idx_, d_chunkpref_, d_nact_, d_part_, d_alpha_, d_it_,
                                                     max_iter_, 0);
  k_blz_b<<<g_red, 256, 0, s>>>(d_inst_, d_idx_, d_chunkpref_, d_nact_, arena_f, d_alpha_, d_part_);
  k_bfin<<<(max_slots_ * 32 + 255) / 256, 256, 0, s>>>(d_inst_, d_idx_, d_chunkpref_, d_nact_, d_part_, d_beta_, d_it_,
                                                     max_iter_, 1);
  k_blz_c<<<g_red, 256, 0, s>>>(d_inst_, d_idx_, d_chunkpref_, d_nact_, arena_f, d_beta_);
  k_bstep<<<(max_slots_ + 255) / 256, 256, 0, s>>>(d_idx_, d_nact_, d_it_);
  return ED_OK;
}

ed_status BatchEngine::time_apply(int reps, float* ms) {
  cudaEvent_t e0, e1;
  ED_CUDA_TRY(cudaEventCreate(&e0));
  ED_CUDA_TRY(cudaEventCreate(&e1));
  ed_status st = launch_apply(st_, nullptr, nullptr);  // warm
  if (st == ED_OK) {
    cudaEventRecord(e0, st_);
    for (int i = 0; i < reps && st == ED_OK; ++i) st = launch_apply(st_, nullptr, nullptr);
    cudaEventRecord(e1, st_);
    cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    *ms = t / (float)std::max(1, reps);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

// Modes of a set of instances (normally the whole batch) chosen on the
// batch itself: start from the dense form everywhere it exists (64-wide
// tiles when d_B <= 64, else 128-wide), then, for classes of instances of
// similar size (D in [4^k, 4^(k+1))), largest total first, try each other
// mode for the whole class and keep it when the timed batched H psi gets
// at least 1 % faster.  Timing the real mix accounts for what a shape timed
// alone would not: cache sharing between instances and the split of the
// apply into the CSR and dense launches.  Each shape's choice is cached
// for later engines of the process (the serving loop's admissions).
ed_status BatchEngine::tune(const std::vector<int>& slots) {
  ED_DEVICE_SCOPE(device_);
  std::map<int, std::vector<int>> cls;  // size class -> dense-capable slots
  for (int s : slots) {
    BSlot& S = slots_[s];
    if (!S.used) continue;
    S.d.mode = S.dense_ok ? default_mode(S) : kModeCSR;
    if (!S.dense_ok) continue;
    int k = 0;
    for (long long D = S.d.D; D >= 4; D >>= 2) ++k;
    cls[k].push_back(s);
  }
  std::vector<std::pair<long long, int>> order;
  for (auto& kv : cls) {
    long long tot = 0;
    for (int s : kv.second) tot += slots_[s].d.D;
    order.push_back({-tot, kv.first});
  }
  std::sort(order.begin(), order.end());
  ED_TRY(rebuild_active());
  float best = 0.f;
  ED_TRY(time_apply(5, &best));
  for (auto& o : order) {
    std::vector<int>& g = cls[o.second];
    std::vector<int> keep(g.size());
    for (size_t i = 0; i < g.size(); ++i) keep[i] = slots_[g[i]].d.mode;
    for (int m : {kModeCSR, kModeD64, kModeD128}) {
      bool same = true;
      for (int s : g) same = same && slots_[s].d.mode == m;
      if (same) continue;
      std::vector<int> prev(g.size());
      for (size_t i = 0; i < g.size(); ++i) {
        prev[i] = slots_[g[i]].d.mode;
        slots_[g[i]].d.mode = m;
      }
      ED_TRY(rebuild_active());
      float t = 0.f;
      ED_TRY(time_apply(5, &t));
      if (t < 0.99f * best) {
        best = t;
      } else {
        for (size_t i = 0; i < g.size(); ++i) slots_[g[i]].d.mode = prev[i];
      }
    }
  }
  for (int s : slots)
    if (slots_[s].used && slots_[s].dense_ok) cache_mode(slots_[s].key, slots_[s].d.mode);
  int err = 0;
  ED_CUDA_TRY(cudaMemcpy(&err, d_err_, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    set_error("batch engine: a tensor-core wait ran out while tuning");
    return ED_ETIMEOUT;
  }
  return rebuild_active();
}

ed_status BatchEngine::capture() {
  ED_CUDA_TRY(cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal));
  launch_step(st_);
  cudaError_t e = cudaStreamEndCapture(st_, &graph_);
  if (e != cudaSuccess) {
    set_error("graph capture failed: %s", cudaGetErrorString(e));
    return ED_ECUDA;
  }
  ED_CUDA_TRY(cudaGraphInstantiate(&exec_, graph_, 0));
  return ED_OK;
}

ed_status BatchEngine::steps(int k) {
  for (int i = 0; i < k; ++i) ED_CUDA_TRY(cudaGraphLaunch(exec_, st_));
  return ED_OK;
}

ed_status BatchEngine::apply_user(const float* x, float* y, cudaStream_t st) {
  return launch_apply(st, x, y);
}

ed_status BatchEngine::sync() {
  ED_CUDA_TRY(cudaStreamSynchronize(st_));
  int err = 0;
  ED_CUDA_TRY(cudaMemcpy(&err, d_err_, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    set_error("batch engine: a tensor-core wait ran out; results are incomplete");
    return ED_ETIMEOUT;
  }
  return ED_OK;
}

// Convergence of every active instance, evaluated only at iteration counts
// that are multiples of `every` since the instance (re)started, so the
// stopping step and the returned energy do not depend on which other
// instances share the batch or when this one joined.
ed_status BatchEngine::poll(double tol, int every, std::vector<int>* done) {
  every = std::max(1, every);
  std::vector<int> it(max_slots_);
  hist_host_.resize(2 * (size_t)max_slots_ * max_iter_);
  ED_CUDA_TRY(cudaMemcpyAsync(it.data(), d_it_, sizeof(int) * max_slots_, cudaMemcpyDeviceToHost, st_));
  ED_CUDA_TRY(cudaMemcpyAsync(hist_host_.data(), d_hist_, sizeof(double) * hist_host_.size(), cudaMemcpyDeviceToHost,
                              st_));
  int err = 0;
  ED_CUDA_TRY(cudaMemcpyAsync(&err, d_err_, sizeof(int), cudaMemcpyDeviceToHost, st_));
  ED_CUDA_TRY(cudaStreamSynchronize(st_));
  if (err) {
    set_error("batch engine: a tensor-core wait ran out; the Lanczos state is invalid");
    return ED_ETIMEOUT;
  }
  bool changed = false;
  for (int s = 0; s < max_slots_; ++s) {
    BSlot& S = slots_[s];
    if (!S.used || !S.active) continue;
    const int m = std::min(it[s], max_iter_);
    const double* a = hist_host_.data() + (size_t)s * max_iter_;
    const double* b = hist_host_.data() + ((size_t)max_slots_ + s) * max_iter_;
    bool stop = false;
    while (!stop && S.iters_seen + every <= m) {
      const int mm = S.iters_seen + every;
      // Krylov space exhausted (FP32 vectors): beta_j tiny against the scale
      double scale = 0.0;
      int me = mm;
      bool exhausted = false;
      for (int j = 0; j < mm; ++j) {
        scale = std::max(scale, std::fabs(a[j]) + b[j]);
        if (b[j] <= 1e-5 * scale) {
          me = j + 1;
          exhausted = true;
          break;
        }
      }
      const double th = tridiag_lowest(a, b, me);
      const bool stable = S.iters_seen > 0 && std::fabs(th - S.theta) <= tol * std::fabs(th);
      S.theta_prev = S.theta;
      S.theta = th;
      S.iters_seen = exhausted ? me : mm;
      if (exhausted || stable || mm + every > max_iter_) {
        S.converged = exhausted || stable;
        stop = true;
      }
    }
    if (stop) {
      S.active = false;
      changed = true;
      if (done) done->push_back(s);
    }
  }
  if (changed) ED_TRY(rebuild_active());
  return ED_OK;
}

}  // namespace edk
