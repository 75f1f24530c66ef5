// Batched Lanczos engine (see batch.h).  Kernels take the active set from
// device memory (count, instance list, row and chunk prefix sums), so one
// captured graph of the Lanczos step stays valid while instances join and
// leave between replays.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>

#include "batch.h"
#include "krylov.h"
#include "reduce.cuh"
#include "splitmix.cuh"

namespace edk {

constexpr int kBW = 8;          // warps per CTA in the apply kernel
constexpr int kBStage = 1024;   // row elements staged in shared memory per warp

__device__ __forceinline__ int find_pref(const long long* pref, int n, long long v) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (pref[mid] <= v) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// y = H x for every active instance; one warp per row a (lanes over b).
// user_mode: x, y are a caller's concatenated vectors (offset uoff);
// otherwise v -> w inside each instance's arena triple.
__global__ void __launch_bounds__(256) k_bapply(const BInst* __restrict__ insts, const int* __restrict__ idx,
                                                const long long* __restrict__ rowpref, const int* __restrict__ nact,
                                                const float* __restrict__ ux, float* __restrict__ uy, float* arena,
                                                int user_mode) {
  __shared__ float stage[kBW][kBStage];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = *nact;
  if (n <= 0) return;
  const long long total = rowpref[n];
  for (long long row = (long long)blockIdx.x * kBW + warp; row < total; row += (long long)gridDim.x * kBW) {
    const int ai = find_pref(rowpref, n, row);
    const BInst& I = insts[idx[ai]];
    const long long a = row - rowpref[ai];
    const int dA = I.dA, dB = I.dB;
    const float* x = user_mode ? ux + I.uoff : arena + I.voff + I.D;
    float* y = user_mode ? uy + I.uoff : arena + I.voff + 2 * I.D;
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
    const float* Drow = I.use_dense ? I.A_dense + a * dA : nullptr;
    for (int b = lane; b < dB; b += 32) {
      const uint32_t sb = I.B_str[b];
      const uint32_t z = I.vab_and ? (sa & sb) : (sa ^ sb);
      float v = da + I.B_diag[b];
      for (int q = 0; q < I.ncls; ++q) v += I.w[q] * (float)__popc(z & I.mask[q]);
      float acc = v * xs[b];
      const int eb0 = I.B_rp[b], eb1 = I.B_rp[b + 1];
      for (int e = eb0; e < eb1; ++e) acc += I.B_val[e] * xs[I.B_col[e]];
      if (Drow) {
        for (int a2 = 0; a2 < dA; ++a2) acc += Drow[a2] * x[(long long)a2 * dB + b];
      } else {
        for (int e = ea0; e < ea1; ++e) acc += I.A_val[e] * x[(long long)I.A_col[e] * dB + b];
      }
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
  std::vector<float> A_val, B_val, A_diag, B_diag, A_dense;
  std::vector<uint32_t> A_str, B_str;
  float c0 = 0.f;
  int ncls = 0, vab_and = 0;
  float w[kMaxClasses] = {};
  unsigned mask[kMaxClasses] = {};
};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

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
  if (h.dA <= kBatchMaxDense) {
    h.A_dense.assign(h.dA * h.dA, 0.f);
    for (int64_t a = 0; a < h.dA; ++a)
      for (int e = h.A_rp[a]; e < h.A_rp[a + 1]; ++e) h.A_dense[a * h.dA + h.A_col[e]] += h.A_val[e];
  }
  h.c0 = (float)c->diag.c0;
  h.ncls = c->diag.ncls;
  h.vab_and = c->diag.vab_and;
  for (int q = 0; q < h.ncls; ++q) {
    h.w[q] = (float)c->diag.w[q];
    h.mask[q] = (unsigned)c->diag.mask[q];
  }
  return ED_OK;
}

size_t tables_bytes(const HostTables& h, int max_iter) {
  size_t b = 0;
  b += align256((size_t)3 * h.dA * h.dB * 4);
  b += align256(h.A_rp.size() * 4) + align256(h.A_col.size() * 4) + align256(h.A_val.size() * 4);
  b += align256(h.A_diag.size() * 4) + align256(h.A_str.size() * 4);
  b += align256(h.B_rp.size() * 4) + align256(h.B_col.size() * 4) + align256(h.B_val.size() * 4);
  b += align256(h.B_diag.size() * 4) + align256(h.B_str.size() * 4);
  b += align256(h.A_dense.size() * 4);
  (void)max_iter;
  return b;
}
}  // namespace

BatchEngine::~BatchEngine() {
  if (exec_) cudaGraphExecDestroy(exec_);
  if (graph_) cudaGraphDestroy(graph_);
  for (void* p : dev_) cudaFree(p);
  if (st_) cudaStreamDestroy(st_);
}

ed_status BatchEngine::init(int device, size_t arena_bytes, int max_slots, int max_iter) {
  device_ = device;
  ED_DEVICE_SCOPE(device);
  if (cudaDeviceGetAttribute(&sms_, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    sms_ = 148;
  }
  ED_CUDA_TRY(cudaStreamCreateWithFlags(&st_, cudaStreamNonBlocking));
  max_slots_ = std::max(1, max_slots);
  max_iter_ = std::max(2, max_iter);
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
  ED_TRY(get((void**)&d_idx_, sizeof(int) * max_slots_));
  ED_TRY(get((void**)&d_rowpref_, sizeof(long long) * (max_slots_ + 1)));
  ED_TRY(get((void**)&d_chunkpref_, sizeof(long long) * (max_slots_ + 1)));
  ED_TRY(get((void**)&d_nact_, sizeof(int) * 4));
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

ed_status BatchEngine::instance_bytes(const ed_model_desc& m, int max_iter, size_t* bytes, int64_t* dim) {
  HostTables h;
  ED_TRY(host_tables(m, h));
  *bytes = tables_bytes(h, max_iter);
  if (dim) *dim = h.dA * h.dB;
  return ED_OK;
}

ed_status BatchEngine::add(const ed_model_desc& m, uint64_t seed, int* slot_out) {
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
  const size_t need = tables_bytes(h, max_iter_);
  size_t off;
  if (!alloc(need, &off)) {
    set_error("batch engine: instance needs %zu bytes, %zu free", need, arena_free());
    return ED_ENOMEM;
  }
  // lay the instance out in its arena range
  std::vector<char> host(need, 0);
  size_t cur = align256((size_t)3 * h.dA * h.dB * 4);
  BSlot& S = slots_[slot];
  BInst& d = S.d;
  double* ha = d.hist_a;
  double* hb = d.hist_b;
  d = BInst{};
  d.hist_a = ha;
  d.hist_b = hb;
  auto put = [&](const void* src, size_t bytes) -> void* {
    void* dst = arena_ + off + cur;
    if (bytes) std::memcpy(host.data() + cur, src, bytes);
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
  d.A_dense = h.A_dense.empty() ? nullptr : (const float*)put(h.A_dense.data(), h.A_dense.size() * 4);
  d.use_dense = (d.A_dense && h.dA <= dense_threshold_) ? 1 : 0;
  d.c0 = h.c0;
  d.ncls = h.ncls;
  d.vab_and = h.vab_and;
  for (int q = 0; q < kMaxClasses; ++q) {
    d.w[q] = h.w[q];
    d.mask[q] = h.mask[q];
  }
  const size_t tab0 = align256((size_t)3 * h.dA * h.dB * 4);
  ED_CUDA_TRY(cudaMemcpyAsync(arena_ + off + tab0, host.data() + tab0, need - tab0, cudaMemcpyHostToDevice, st_));
  S.used = true;
  S.active = false;
  S.alloc_off = off;
  S.alloc_len = need;
  S.has_dense = d.A_dense != nullptr;
  ED_CUDA_TRY(cudaMemcpyAsync(d_inst_ + slot, &d, sizeof(BInst), cudaMemcpyHostToDevice, st_));
  ED_CUDA_TRY(cudaStreamSynchronize(st_));
  ED_TRY(restart(slot, seed));
  *slot_out = slot;
  return ED_OK;
}

ed_status BatchEngine::restart(int slot, uint64_t seed) {
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
  ED_CUDA_TRY(cudaStreamSynchronize(st_));
  S.active = true;
  S.converged = false;
  S.iters_seen = 0;
  S.theta = S.theta_prev = 0.0;
  return rebuild_active();
}

void BatchEngine::remove(int slot) {
  BSlot& S = slots_[slot];
  if (!S.used) return;
  release(S.alloc_off, S.alloc_len);
  S.used = false;
  S.active = false;
  rebuild_active();
}

ed_status BatchEngine::set_dense_threshold(int t) {
  dense_threshold_ = t;
  for (int s = 0; s < max_slots_; ++s) {
    BSlot& S = slots_[s];
    if (!S.used) continue;
    S.d.use_dense = (S.has_dense && S.d.dA <= t) ? 1 : 0;
    ED_CUDA_TRY(cudaMemcpyAsync(d_inst_ + s, &S.d, sizeof(BInst), cudaMemcpyHostToDevice, st_));
  }
  ED_CUDA_TRY(cudaStreamSynchronize(st_));
  return ED_OK;
}

ed_status BatchEngine::rebuild_active() {
  std::vector<int> idx;
  std::vector<long long> rp(1, 0), cp(1, 0);
  for (int s = 0; s < max_slots_; ++s) {
    const BSlot& S = slots_[s];
    if (!S.used || !S.active) continue;
    idx.push_back(s);
    rp.push_back(rp.back() + S.d.dA);
    cp.push_back(cp.back() + (S.d.D + kBatchChunk - 1) / kBatchChunk);
  }
  if (cp.back() > part_cap_) {
    set_error("batch engine: reduction chunks exceed capacity");
    return ED_ENOMEM;
  }
  int n = (int)idx.size();
  if (!idx.empty()) ED_CUDA_TRY(cudaMemcpyAsync(d_idx_, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice, st_));
  ED_CUDA_TRY(cudaMemcpyAsync(d_rowpref_, rp.data(), rp.size() * 8, cudaMemcpyHostToDevice, st_));
  ED_CUDA_TRY(cudaMemcpyAsync(d_chunkpref_, cp.data(), cp.size() * 8, cudaMemcpyHostToDevice, st_));
  ED_CUDA_TRY(cudaMemcpyAsync(d_nact_, &n, 4, cudaMemcpyHostToDevice, st_));
  ED_CUDA_TRY(cudaStreamSynchronize(st_));
  return ED_OK;
}

ed_status BatchEngine::launch_step(cudaStream_t s) {
  float* arena_f = (float*)arena_;
  const int g_apply = sms_ * 4;
  const int g_red = sms_ * 4;
  k_bapply<<<g_apply, 256, 0, s>>>(d_inst_, d_idx_, d_rowpref_, d_nact_, nullptr, nullptr, arena_f, 0);
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
  k_bapply<<<sms_ * 4, 256, 0, st>>>(d_inst_, d_idx_, d_rowpref_, d_nact_, x, y, (float*)arena_, 1);
  ED_CUDA_TRY(cudaGetLastError());
  return ED_OK;
}

ed_status BatchEngine::sync() {
  ED_CUDA_TRY(cudaStreamSynchronize(st_));
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
  ED_CUDA_TRY(cudaStreamSynchronize(st_));
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
