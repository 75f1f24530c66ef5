// Batched Lanczos engine: many independent single-block instances (Hubbard
// models with the spin-up|spin-down cut) stepped together, one persistent
// launch per kernel over all active instances, the whole Lanczos step
// captured once in a CUDA graph.  Used by the batch API and by the serving
// loop (which adds and removes instances between steps).
#pragma once

#include <cstdint>
#include <vector>

#include "ed_internal.h"

namespace edk {

constexpr int kBatchChunk = 4096;  // elements per reduction chunk
constexpr int kBatchMaxDense = 64; // largest d_A with a dense H_A table

struct BInst {
  long long voff;      // start of the instance's three FP32 Lanczos vectors in the arena
  long long uoff;      // offset in a caller's concatenated vector (ed_batch_apply)
  long long D;
  int dA, dB;
  int n_sites;
  int use_dense;       // H_A applied as a dense d_A x d_A matrix
  const int* A_rp;
  const int* A_col;
  const float* A_val;
  const float* A_diag;
  const uint32_t* A_str;
  const int* B_rp;
  const int* B_col;
  const float* B_val;
  const float* B_diag;
  const uint32_t* B_str;
  const float* A_dense;
  double* hist_a;      // alpha_j, j < max_iter
  double* hist_b;      // beta_{j+1}
  float c0;
  int ncls;
  int vab_and;
  int pad_;
  float w[kMaxClasses];
  unsigned mask[kMaxClasses];
};

// host side of one instance
struct BSlot {
  bool used = false;
  bool active = false;
  BInst d{};
  size_t alloc_off = 0, alloc_len = 0;
  int has_dense = 0;
  int iters_seen = 0;
  double theta_prev = 0.0;
  double theta = 0.0;
  bool converged = false;
  uint64_t tag = 0;
};

class BatchEngine {
 public:
  ~BatchEngine();
  ed_status init(int device, size_t arena_bytes, int max_slots, int max_iter);
  // bytes an instance needs in the arena (tables + 3 vectors + history)
  static ed_status instance_bytes(const ed_model_desc& m, int max_iter, size_t* bytes, int64_t* dim);
  ed_status add(const ed_model_desc& m, uint64_t seed, int* slot);
  void remove(int slot);
  // fresh start vector (keyed SplitMix64 values, normalised) for an instance
  ed_status restart(int slot, uint64_t seed);
  ed_status set_dense_threshold(int t);
  ed_status apply_user(const float* x, float* y, cudaStream_t st);
  ed_status steps(int k);
  // convergence test of every active instance; converged ones are deactivated
  ed_status poll(double tol, int every, std::vector<int>* done);
  int max_iter() const { return max_iter_; }
  int active_count() const;
  int iterations(int slot) const { return slots_[slot].iters_seen; }
  double energy(int slot) const { return slots_[slot].theta; }
  bool converged(int slot) const { return slots_[slot].converged; }
  size_t arena_free() const;
  size_t arena_size() const { return arena_bytes_; }
  int dense_threshold() const { return dense_threshold_; }
  cudaStream_t stream() const { return st_; }
  std::vector<BSlot>& slots() { return slots_; }
  ed_status sync();
  // upload the active set (after changing BSlot::active flags)
  ed_status rebuild_active();

 private:
  ed_status capture();
  ed_status launch_step(cudaStream_t s);
  bool alloc(size_t len, size_t* off);
  void release(size_t off, size_t len);

  int device_ = 0;
  int sms_ = 148;
  cudaStream_t st_ = nullptr;
  char* arena_ = nullptr;
  size_t arena_bytes_ = 0;
  std::vector<std::pair<size_t, size_t>> free_;  // (offset, length), sorted
  std::vector<BSlot> slots_;
  int max_slots_ = 0, max_iter_ = 0;
  int dense_threshold_ = 16;
  // device state
  BInst* d_inst_ = nullptr;
  int* d_idx_ = nullptr;
  long long* d_rowpref_ = nullptr;
  long long* d_chunkpref_ = nullptr;
  int* d_nact_ = nullptr;
  int* d_it_ = nullptr;
  double* d_alpha_ = nullptr;
  double* d_beta_ = nullptr;
  double* d_part_ = nullptr;
  double* d_hist_ = nullptr;         // [2][max_slots][max_iter]: alpha then beta
  std::vector<double> hist_host_;
  long long part_cap_ = 0;
  cudaGraph_t graph_ = nullptr;
  cudaGraphExec_t exec_ = nullptr;
  std::vector<void*> dev_;
};

}  // namespace edk
