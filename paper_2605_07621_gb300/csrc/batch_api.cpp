// Batched form: many independent Hubbard instances (spin-up|spin-down cut)
// in one persistent launch per kernel with a captured Lanczos-step graph;
// the per-instance choice between a CSR and a dense H_A is autotuned by
// timing the batched apply.
#include <chrono>
#include <cstring>
#include <new>

#include "batch.h"
#include "krylov.h"

using namespace edk;

struct ed_batch {
  BatchEngine eng;
  std::vector<int> slot;
  std::vector<int64_t> off;
  int n = 0;
  int threshold = 0;
  float tune_ms[5] = {0, 0, 0, 0, 0};
};

static const int kThresholds[5] = {0, 8, 16, 32, 64};
static const int kBatchHist = 1024;

extern "C" ed_status ed_batch_create(const ed_model_desc* models, int n, int flags, ed_batch** out) {
  if (!out || !models || n < 1) { set_error("ed_batch_create: bad arguments"); return ED_EINVAL; }
  if (flags < 0 || flags > 2) { set_error("bad flags %d", flags); return ED_EINVAL; }
  *out = nullptr;
  size_t total = 0;
  std::vector<int64_t> dims(n);
  for (int i = 0; i < n; ++i) {
    size_t b;
    ED_TRY(BatchEngine::instance_bytes(models[i], kBatchHist, &b, &dims[i]));
    total += b + 512;
  }
  ed_batch* B = new (std::nothrow) ed_batch();
  if (!B) { set_error("host allocation failed"); return ED_ENOMEM; }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); dev = 0; }
  ed_status st = B->eng.init(dev, total + (1 << 20), n, kBatchHist);
  if (st != ED_OK) { delete B; return st; }
  B->n = n;
  B->slot.resize(n);
  B->off.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    st = B->eng.add(models[i], 20260507ULL, &B->slot[i]);
    if (st != ED_OK) { delete B; return st; }
    B->off[i + 1] = B->off[i] + dims[i];
    BSlot& S = B->eng.slots()[B->slot[i]];
    S.d.uoff = B->off[i];
  }
  // descriptors with user offsets and the dense threshold
  int thr = (flags & 3) == ED_OPS_FORCE_CSR ? 0 : (flags & 3) == ED_OPS_FORCE_DENSE ? kBatchMaxDense : 16;
  st = B->eng.set_dense_threshold(thr);
  if (st != ED_OK) { delete B; return st; }
  if (flags == ED_OPS_DEFAULT) {
    // autotune: time the batched apply for each dense threshold
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int best_t = 0;
    for (int k = 0; k < 5; ++k) {
      B->eng.set_dense_threshold(kThresholds[k]);
      B->eng.steps(1);  // warm
      cudaEventRecord(e0, B->eng.stream());
      B->eng.steps(3);
      cudaEventRecord(e1, B->eng.stream());
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      B->tune_ms[k] = ms / 3.f;
      if (ms < best) { best = ms; best_t = kThresholds[k]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    thr = best_t;
    st = B->eng.set_dense_threshold(thr);
    if (st != ED_OK) { delete B; return st; }
  }
  B->threshold = thr;
  *out = B;
  return ED_OK;
}

extern "C" int64_t ed_batch_dim(const ed_batch* b) { return b ? b->off[b->n] : -1; }

extern "C" ed_status ed_batch_offsets(const ed_batch* b, int64_t* off) {
  if (!b || !off) { set_error("NULL argument"); return ED_EINVAL; }
  std::memcpy(off, b->off.data(), sizeof(int64_t) * (b->n + 1));
  return ED_OK;
}

extern "C" ed_status ed_batch_info(const ed_batch* b, int* dense_threshold, float* tune_ms) {
  if (!b) { set_error("NULL batch"); return ED_EINVAL; }
  if (dense_threshold) *dense_threshold = b->threshold;
  if (tune_ms) std::memcpy(tune_ms, b->tune_ms, sizeof(b->tune_ms));
  return ED_OK;
}

static ed_status activate_all(ed_batch* b) {
  for (int i = 0; i < b->n; ++i) b->eng.slots()[b->slot[i]].active = true;
  ED_TRY(b->eng.set_dense_threshold(b->threshold));
  return b->eng.rebuild_active();
}

extern "C" ed_status ed_batch_apply(ed_batch* b, const void* x, void* y, ed_dtype dt, void* stream) {
  if (!b || !x || !y) { set_error("NULL argument"); return ED_EINVAL; }
  if (dt != ED_F32) { set_error("the batched apply stores vectors in FP32"); return ED_EUNSUPPORTED; }
  ED_TRY(activate_all(b));
  ed_status st = b->eng.apply_user((const float*)x, (float*)y, (cudaStream_t)stream);
  return st;
}

extern "C" ed_status ed_batch_lanczos(ed_batch* b, const ed_lanczos_opts* opts, double* e0, int* iters,
                                      ed_report* rep) {
  auto t0 = std::chrono::steady_clock::now();
  if (!b || !e0) { set_error("NULL argument"); return ED_EINVAL; }
  ed_lanczos_opts o;
  ed_lanczos_default_opts(&o);
  o.tol = 1e-7;
  if (opts) o = *opts;
  if (o.mode != ED_LZ_F32) { set_error("the batched Lanczos runs FP32 storage with FP64 reductions (ED_LZ_F32)"); return ED_EUNSUPPORTED; }
  const int max_iter = std::min(o.max_iter, b->eng.max_iter());
  const int K = std::max(1, o.check_every);
  for (int i = 0; i < b->n; ++i) ED_TRY(b->eng.restart(b->slot[i], o.seed));
  ED_TRY(b->eng.set_dense_threshold(b->threshold));
  int steps = 0;
  while (b->eng.active_count() > 0 && steps < max_iter) {
    const int k = std::min(K, max_iter - steps);
    ED_TRY(b->eng.steps(k));
    steps += k;
    ED_TRY(b->eng.poll(o.tol, K, nullptr));
  }
  int nconv = 0, maxit = 0;
  for (int i = 0; i < b->n; ++i) {
    const int s = b->slot[i];
    e0[i] = b->eng.energy(s);
    if (iters) iters[i] = b->eng.iterations(s);
    nconv += b->eng.converged(s) ? 1 : 0;
    maxit = std::max(maxit, b->eng.iterations(s));
  }
  if (rep) {
    double* al = rep->alpha;
    double* be = rep->beta;
    int cap = rep->ab_capacity;
    std::memset(rep, 0, sizeof(*rep));
    rep->alpha = al;
    rep->beta = be;
    rep->ab_capacity = cap;
    rep->iterations = steps;
    rep->iterations_low = maxit;
    rep->converged = nconv == b->n;
    rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (nconv != b->n) { set_error("%d of %d instances did not converge", b->n - nconv, b->n); return ED_ENOCONV; }
  return ED_OK;
}

extern "C" void ed_batch_destroy(ed_batch* b) { delete b; }
