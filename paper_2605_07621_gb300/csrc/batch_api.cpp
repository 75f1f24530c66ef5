// Batched form: many independent Hubbard instances (spin-up|spin-down cut)
// in one persistent launch per kernel with a captured Lanczos-step graph;
// the per-instance choice between the CSR apply and the dense tensor-core
// apply (and its output tile width) is autotuned per instance shape.
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
  float tune_ms[4] = {0, 0, 0, 0};
};

static const int kBatchHist = 1024;

// whole-batch apply (ms) with every instance in `mode` (dense modes only
// where the instance has the dense form)
static ed_status time_uniform(ed_batch* B, int mode, float* ms) {
  for (int i = 0; i < B->n; ++i) ED_TRY(B->eng.set_mode(B->slot[i], mode));
  ED_TRY(B->eng.rebuild_active());
  return B->eng.time_apply(3, ms);
}

extern "C" ed_status ed_batch_create(const ed_model_desc* models, int n, int flags, ed_batch** out) {
  if (!out || !models || n < 1) { set_error("ed_batch_create: bad arguments"); return ED_EINVAL; }
  if (flags < 0 || flags > 2) { set_error("bad flags %d", flags); return ED_EINVAL; }
  *out = nullptr;
  const bool dense = flags != ED_OPS_FORCE_CSR;
  size_t total = 0;
  std::vector<int64_t> dims(n);
  for (int i = 0; i < n; ++i) {
    size_t b;
    ED_TRY(BatchEngine::instance_bytes(models[i], dense, &b, &dims[i]));
    total += b + 512;
  }
  ed_batch* B = new (std::nothrow) ed_batch();
  if (!B) { set_error("host allocation failed"); return ED_ENOMEM; }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); dev = 0; }
  ed_status st = B->eng.init(dev, total + (1 << 20), n, kBatchHist, dense);
  if (st != ED_OK) { delete B; return st; }
  B->n = n;
  B->slot.resize(n);
  B->off.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    st = B->eng.add(models[i], 20260507ULL, &B->slot[i], false);
    if (st != ED_OK) { delete B; return st; }
    B->off[i + 1] = B->off[i] + dims[i];
    BSlot& S = B->eng.slots()[B->slot[i]];
    S.d.uoff = B->off[i];
    st = B->eng.upload_inst(B->slot[i]);
    if (st != ED_OK) { delete B; return st; }
  }
  st = B->eng.rebuild_active();
  if (st != ED_OK) { delete B; return st; }
  if (flags == ED_OPS_DEFAULT) {
    // the batch with every instance in each mode, then the tuned choice
    for (int k = 0; k < 3 && st == ED_OK; ++k) st = time_uniform(B, k, &B->tune_ms[k]);
    if (st == ED_OK) st = B->eng.tune(B->slot);
    if (st == ED_OK) st = B->eng.time_apply(3, &B->tune_ms[3]);
  } else {
    if (flags == ED_OPS_FORCE_DENSE)
      for (int i = 0; i < n && st == ED_OK; ++i) {
        const BSlot& S = B->eng.slots()[B->slot[i]];
        st = B->eng.set_mode(B->slot[i], S.d.dB <= 64 ? kModeD64 : kModeD128);
      }
    if (st == ED_OK) st = B->eng.rebuild_active();
    if (st == ED_OK) st = B->eng.time_apply(3, &B->tune_ms[3]);
  }
  if (st == ED_OK) st = B->eng.sync();
  if (st != ED_OK) { delete B; return st; }
  *out = B;
  return ED_OK;
}

extern "C" int64_t ed_batch_dim(const ed_batch* b) { return b ? b->off[b->n] : -1; }

extern "C" ed_status ed_batch_offsets(const ed_batch* b, int64_t* off) {
  if (!b || !off) { set_error("NULL argument"); return ED_EINVAL; }
  std::memcpy(off, b->off.data(), sizeof(int64_t) * (b->n + 1));
  return ED_OK;
}

extern "C" ed_status ed_batch_info(const ed_batch* b, int* modes, float* tune_ms) {
  if (!b) { set_error("NULL batch"); return ED_EINVAL; }
  if (modes)
    for (int i = 0; i < b->n; ++i) modes[i] = b->eng.mode(b->slot[i]);
  if (tune_ms) std::memcpy(tune_ms, b->tune_ms, sizeof(b->tune_ms));
  return ED_OK;
}

static ed_status activate_all(ed_batch* b) {
  for (int i = 0; i < b->n; ++i) b->eng.slots()[b->slot[i]].active = true;
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
  for (int i = 0; i < b->n; ++i) ED_TRY(b->eng.restart(b->slot[i], o.seed, false));
  ED_TRY(b->eng.rebuild_active());
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
