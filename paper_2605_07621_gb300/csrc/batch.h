// Batched Lanczos engine: many independent single-block instances (Hubbard
// models with the spin-up|spin-down cut) stepped together, one persistent
// launch per kernel over all active instances, the whole Lanczos step
// captured once in a CUDA graph.  Used by the batch API and by the serving
// loop (which adds and removes instances between steps).  Each instance's
// H psi runs either from its CSR side operators (k_bapply) or as two dense
// products on the tensor cores (bdense.cu); the choice, and the output tile
// width of the dense form, is made per instance shape by timing both.
#pragma once

#include <cuda.h>

#include <cstdint>
#include <vector>

#include "ed_internal.h"

namespace edk {

constexpr int kBatchChunk = 4096;  // elements per reduction chunk
constexpr int kBDenseMax = 1024;   // largest d_A, d_B with a dense (tensor-core) form
constexpr int kBMaps = 6;          // tensor maps per instance (see bdense.cu)
enum BMode { kModeCSR = 0, kModeD64 = 1, kModeD128 = 2 };

struct BInst {
  long long voff;      // start of the instance's three FP32 Lanczos vectors in the arena
  long long uoff;      // offset in a caller's concatenated vector (ed_batch_apply)
  long long D;
  int dA, dB;
  int n_sites;
  int mode;            // BMode
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
  // dense form (null when the instance has none): H_A, H_B as three BF16
  // pieces each ([3][d][Kp]), and the pieces of Psi (rows a, [3][d_A][KpB])
  // and of Psi^T (rows b, [3][d_B][KpA]) written before each product
  const uint16_t* HA;
  const uint16_t* HB;
  uint16_t* XN;
  uint16_t* XT;
  int KpA, KpB;        // row strides of the pieces (d rounded up to 64)
  // nonzero 64-wide K blocks (bit kb) of each 128-row tile of H_A, then of
  // each 64-row and each 128-row tile of H_B: the dense products skip zero blocks
  const uint32_t* kmask;
  double* hist_a;      // alpha_j, j < max_iter
  double* hist_b;      // beta_{j+1}
  float c0;
  int ncls;
  int vab_and;
  int pad_;
  float w[kMaxClasses];
  unsigned mask[kMaxClasses];
};

// arguments of the dense (tensor-core) H psi over the dense work lists
struct BDenseArgs {
  const BInst* insts;
  const int* cnt;            // {CSR, dense, 64-wide, 128-wide} list lengths
  const int* didx;           // dense slots, with their 64 x 64 slicing tiles
  const long long* dspref;
  const int* idx64;          // slots with 128 x 64 output tiles
  const long long* tpref64;
  const int* idx128;         // slots with 128 x 128 output tiles
  const long long* tpref128;
  const CUtensorMap* maps;   // kBMaps per slot
  const float* ux;           // user vectors (user_mode) or the Lanczos arena
  float* uy;
  float* arena;
  int user_mode;
  int sms;
  int* err;
};
ed_status bdense_prepare();  // kernel attributes; once, before any graph capture
ed_status bdense_apply(const BDenseArgs& a, cudaStream_t st);
// the dense form's tables of one instance (pieces of H_A, H_B, nonzero-block
// masks; their arena ranges zeroed first) built on the device from its CSR
ed_status bdense_tables(const BInst& I, cudaStream_t st);

// host side of one instance
struct BSlot {
  bool used = false;
  bool active = false;
  BInst d{};
  size_t alloc_off = 0, alloc_len = 0;
  int dense_ok = 0;    // has the dense form's tables
  long long key[4] = {0, 0, 0, 0};  // shape: d_A, d_B, nnz of H_A, nnz of H_B
  int iters_seen = 0;
  double theta_prev = 0.0;
  double theta = 0.0;
  bool converged = false;
  uint64_t tag = 0;
};

class BatchEngine {
 public:
  ~BatchEngine();
  // dense: instances small enough get the tables of the tensor-core form
  ed_status init(int device, size_t arena_bytes, int max_slots, int max_iter, bool dense);
  // bytes an instance needs in the arena (tables + 3 vectors)
  static ed_status instance_bytes(const ed_model_desc& m, bool dense, size_t* bytes, int64_t* dim);
  // new instance (active); its mode is the cached choice for its shape, else
  // the dense form where it has one.  commit = false leaves the device work
  // lists to one rebuild_active after several adds
  ed_status add(const ed_model_desc& m, uint64_t seed, int* slot, bool commit = true);
  // free an instance's arena range; an active instance leaves the device work
  // lists at once (commit) or at the next rebuild_active
  void remove(int slot, bool commit = true);
  // fresh start vector (keyed SplitMix64 values, normalised) for an instance;
  // commit as for add
  ed_status restart(int slot, uint64_t seed, bool commit = true);
  // per-instance mode (kModeD64 / kModeD128 fall back to CSR without the
  // dense form); takes effect at the next rebuild_active
  ed_status set_mode(int slot, int mode);
  // the instance descriptor (user offset) to the device
  ed_status upload_inst(int slot);
  // choose the modes of the listed (active) slots by timing the batched
  // apply over them, cache the choice per shape
  ed_status tune(const std::vector<int>& slots);
  // the cached choice for the instance's shape, else the dense form with
  // 64-wide tiles when d_B <= 64, 128-wide otherwise
  int default_mode(const BSlot& S) const;
  // device time (ms) of one H psi over all active instances (Lanczos vectors)
  ed_status time_apply(int reps, float* ms);
  int mode(int slot) const { return slots_[slot].d.mode; }
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
  bool dense() const { return dense_; }
  cudaStream_t stream() const { return st_; }
  std::vector<BSlot>& slots() { return slots_; }
  ed_status sync();
  // upload the active set (after changing BSlot::active flags)
  ed_status rebuild_active();

 private:
  ed_status capture();
  ed_status launch_step(cudaStream_t s);
  // H psi over the uploaded lists (user vectors when x, y are set)
  ed_status launch_apply(cudaStream_t s, const float* x, float* y);
  // upload work lists: CSR slots and dense slots by tile width
  ed_status upload_lists(const std::vector<int>& csr, const std::vector<int>& d64, const std::vector<int>& d128);
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
  bool dense_ = false;
  int list_cap_ = 0;
  // device state
  BInst* d_inst_ = nullptr;
  int* d_idx_ = nullptr;             // active slots (reductions)
  long long* d_chunkpref_ = nullptr;
  int* d_nact_ = nullptr;
  // apply work lists; d_cnt_ = {CSR, dense (all widths), 64-wide, 128-wide}
  int* d_cnt_ = nullptr;
  int* d_cidx_ = nullptr;
  long long* d_crowpref_ = nullptr;
  int* d_didx_ = nullptr;
  long long* d_dspref_ = nullptr;    // 64 x 64 slicing tiles
  int* d_idx64_ = nullptr;
  long long* d_tpref64_ = nullptr;
  int* d_idx128_ = nullptr;
  long long* d_tpref128_ = nullptr;
  CUtensorMap* d_maps_ = nullptr;    // kBMaps per slot
  int* d_err_ = nullptr;             // bounded tensor-core waits that ran out
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
