// Internal structures of the bipartite engine (host + device views).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ed.h"

namespace edk {

constexpr int kMaxCross = 64;     // cross-cut bonds packed into one 64-bit word
constexpr int kMaxClasses = 8;    // distinct diagonal cross weights
constexpr int kMaxSideBits = 30;  // sites on one side of the cut

void set_error(const char* fmt, ...);

#define ED_CUDA_TRY(call)                                                                     \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      ::edk::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return ED_ECUDA;                                                                        \
    }                                                                                         \
  } while (0)

#define ED_TRY(call)                 \
  do {                               \
    ed_status s_ = (call);           \
    if (s_ != ED_OK) return s_;      \
  } while (0)

int64_t binom(int n, int k);
// colex (combinadic) rank of an n-bit string among strings of equal popcount:
// rank(x) = sum_j C(p_j, j+1) over the set-bit positions p_0 < p_1 < ...
int64_t combinadic_rank(uint64_t x);

// One side of the cut: its sites and its states grouped by popcount.
struct Side {
  int n = 0;                                  // bits
  std::vector<int> sites;                     // bit p -> lattice site
  std::vector<int64_t> start;                 // start[k]: global index of first popcount-k state
  std::vector<uint32_t> states;               // strings of the used popcounts, grouped by popcount, ascending
  std::vector<char> used;                     // used[k]: popcount k appears in some block
  int64_t total() const { return (int64_t)states.size(); }
  int64_t dim(int k) const { return (k < 0 || k > n) ? 0 : start[k + 1] - start[k]; }
};

// Block of Eq. (3): charge s on side A.
struct Block {
  int s;        // A-side charge (popcount)
  int kB;       // B-side popcount
  int64_t dA, dB;
  int64_t off;  // element offset in the vector
  int64_t gA0;  // global side-A index of row 0
  int64_t gB0;  // global side-B index of column 0
  int64_t row0; // index of row 0 among all rows of all blocks
};

// Cross-cut bond between A bit p and B bit q.
struct CrossBond {
  int p, q;      // side-local bits
  int ia, ib;    // index into the distinct cross-site lists (map tables)
  double coef;   // jxy/2
  double jz;
};

// Plain-old-data view passed to kernels by value.
struct DevBlock {
  int s, kB;
  int nbr_lo, nbr_hi;   // block index of charge s-1 / s+1 (-1 if absent)
  long long dA, dB, off, gA0, gB0, row0;
};

struct DevCross {
  int ia, ib;
  double coef;
};

struct DevTables {
  // side A
  const int* A_rowptr;
  const int* A_col;
  const double* A_val64;
  const float* A_val32;
  const double* A_diag;
  const unsigned long long* A_pack;
  const int* mapA;          // [n_cross_A][A.total]
  // side B
  const int* B_rowptr;
  const int* B_col;
  const double* B_val64;
  const float* B_val32;
  const double* B_diag;
  const unsigned long long* B_pack;
  const int* mapB;          // [n_cross_B][B.total]
  const uint32_t* A_states; // side-local bit strings by global index
  const uint32_t* B_states;
  const float* A_diag32;
  const float* B_diag32;
  const unsigned long long* A_key;  // bit-string key part of each side state
  const unsigned long long* B_key;  //   (key = A_key | B_key)
  long long A_total, B_total;
};

struct DevDiagParams {
  int ncls;
  int vab_and;              // 0: spin (xor of packed bits), 1: Hubbard (and)
  double c0;
  double w[kMaxClasses];
  float c0_32;
  float w32[kMaxClasses];
  unsigned long long mask[kMaxClasses];
};

}  // namespace edk

struct ed_ctx {
  // model copy
  int kind = ED_SPIN;
  int n_sites = 0;
  std::vector<int> bi, bj;
  std::vector<double> jxy, jz, t, U, eps;
  int n_up = 0, n_dw = 0;
  uint64_t cut_mask = 0;
  int spin_cut = 0;
  // structure
  edk::Side A, B;
  std::vector<edk::Block> blocks;
  int64_t D = 0;
  int64_t n_rows = 0;
  std::vector<int> block_of_s;  // s -> block index or -1
  // side bonds (side-local bits), couplings
  struct SideBond { int p, q; double off, jz; };
  std::vector<SideBond> bondsA, bondsB;
  std::vector<edk::CrossBond> cross;
  std::vector<int> crossA_bits, crossB_bits;  // distinct bits
  edk::DevDiagParams diag{};
  // device state
  int device = 0;
  bool ops_built = false;
  int ops_flags = 0;
  std::vector<void*> dev_allocs;
  int64_t dev_bytes = 0;
  edk::DevTables tab{};
  edk::DevBlock* d_blocks = nullptr;
  edk::DevCross* d_cross = nullptr;
  std::vector<edk::DevBlock> h_blocks;
  std::vector<edk::DevCross> h_cross;
  long long* d_row_start = nullptr;  // per block first row (for row -> block lookup)
  // per-side CSR stats
  int64_t nnzA = 0, nnzB = 0;
  // Lanczos / GF work buffers (lazily allocated)
  void* work = nullptr;
  size_t work_bytes = 0;
  double* d_partials = nullptr;
  double* h_pinned = nullptr;
  ~ed_ctx();
};

namespace edk {
ed_status dev_alloc(ed_ctx* c, void** p, size_t bytes);
template <typename T>
ed_status upload(ed_ctx* c, T** dptr, const std::vector<T>& h) {
  size_t bytes = std::max<size_t>(h.size() * sizeof(T), 16);
  ED_TRY(dev_alloc(c, (void**)dptr, bytes));
  if (!h.empty()) ED_CUDA_TRY(cudaMemcpy(*dptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return ED_OK;
}
uint64_t state_key(const ed_ctx* c, uint32_t a, uint32_t b);
}  // namespace edk
