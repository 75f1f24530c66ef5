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

// Makes `dev` the current device for the scope of one entry point and puts
// the caller's current device back on exit, so no call changes the calling
// thread's current device.
class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev_) != cudaSuccess) {
      cudaGetLastError();
      prev_ = -1;
    }
    if (prev_ != dev) {
      err_ = cudaSetDevice(dev);
      if (err_ != cudaSuccess) cudaGetLastError();
      else switched_ = true;
    }
  }
  ~DeviceGuard() {
    if (switched_ && prev_ >= 0) cudaSetDevice(prev_);
  }
  ed_status status() const {
    if (err_ == cudaSuccess) return ED_OK;
    set_error("cudaSetDevice failed: %s", cudaGetErrorString(err_));
    return ED_ECUDA;
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;

 private:
  int prev_ = -1;
  bool switched_ = false;
  cudaError_t err_ = cudaSuccess;
};

#define ED_DEVICE_SCOPE(dev)                 \
  ::edk::DeviceGuard ed_dev_guard_(dev);     \
  do {                                       \
    ed_status s_ = ed_dev_guard_.status();   \
    if (s_ != ED_OK) return s_;              \
  } while (0)

int64_t binom(int n, int k);
// side-local bit orders of a spin model (side A: sites on a cross-cut bond
// low; side B: those sites high)
void order_spin_sides(const ed_model_desc* m, std::vector<int>& sitesA, std::vector<int>& sitesB);
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
  int has_hA;           // the block's rows have H_A entries (second pass needed)
  int pad_;
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

// Tables of the class-sorted apply path.  Off-diagonal matrix elements take
// at most kMaxCls distinct values ("classes"); each CSR row lists its
// columns grouped by class (16-bit indices), so no value is stored per
// entry.  When every coupling is a dyadic rational (value * 2^q_shift is a
// small integer) the FP64 apply runs in exact 64-bit fixed point.
constexpr int kMaxCls = 4;

struct Dev3 {
  const uint2* A_meta;      // x: first entry, y: per-class counts (8 bits each)
  const uint16_t* A_col;
  const uint2* B_meta;
  const uint16_t* B_col;
  const uint32_t* A_pack;   // packed cross-bond bits (spin) or up string (Hubbard)
  const uint32_t* B_pack;
  const float* A_d32;
  const float* B_d32;
  const double* A_d64;
  const double* B_d64;
  const int* A_dI;          // side diagonal in units of 2^-q_shift
  const int* B_dI;
  const long long* A_dW;    // the same as 64-bit integers (wide-weight path)
  const long long* B_dW;
  const uint16_t* mapA;     // [n_cross_A_bits][A_total]
  const uint16_t* mapB;     // [n_cross_B_bits][B_total]
  long long A_total, B_total;
  float w32[kMaxCls];
  double w64[kMaxCls];
  long long wI[kMaxCls];
  // diagonal cross term: c0 + sum_c dw_c popc(f(pa,pb) & dmask_c)
  int vab_and;
  int ncls_d;
  unsigned dmask[kMaxClasses];
  float dw32[kMaxClasses];
  double dw64[kMaxClasses];
  long long dwI[kMaxClasses];
  float dc0_32;
  double dc0_64;
  long long dc0_I;
  unsigned cross_cls_mask[kMaxCls];  // cross bonds (bit k) with off-diagonal class c
  int q_shift;              // values * 2^q_shift are integers (fixed-point path)
  int P;                    // fraction bits of the fixed-point vector
  // padded side-B lists of the row pass: every class segment starts at a
  // multiple of 4 entries and is padded to one with the zero-slot index d_B
  const uint2* B_meta4;     // x: first entry / 4, y: per-class group-of-4 counts
  const uint2* B_col4;      // 4 x uint16 per element
  // cross bonds grouped by B site: bonds with B site ib are bits ib_mask[ib]
  int n_ib;
  int n_ia;
  int xl_ok;                // row-pass bond lists apply: the cross bonds take at most two
                            // value classes, each B cross site at most two bonds of each
  int xl_c[2];              // the two classes (equal when there is one)
  unsigned xl_c1_mask;      // cross bonds (bit k) of class xl_c[1] (the rest are xl_c[0])
  unsigned ib_mask[32];
  unsigned ia_mask[32];     // bonds (bits) whose A site is ia
  unsigned char bond_ib[32];
  unsigned char bond_ia[32];
  float bond_w32[32];
  double bond_w64[32];
  long long bond_wI[32];
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
  int4* d_panel_items = nullptr;     // (block, first column, first row, rows) of the H_A pass
  long long* d_grp2_start = nullptr; // per block: first two-row group (plus total)
  long long n_grp2 = 0;
  long long* d_grp4_start = nullptr; // per block: first four-row group (plus total)
  long long n_grp4 = 0;
  long long n_panel_items = 0;
  int* d_err = nullptr;              // set by kernels whose bounded waits ran out
  // class-sorted path
  bool v3_ok = false;                // tables below are valid
  bool dyadic = false;               // FP64 apply may use exact fixed point
  bool wide = false;                 // couplings not dyadic: integer weights, exact 128-bit sums
  bool classed = false;              // couplings not dyadic: the FP64 apply sums the fixed-point
                                     // input exactly per value class and weights each sum in FP64
  bool diag_split = false;           // ... for the off-diagonal terms only; the
                                     // diagonal is added in FP64 afterwards
  edk::Dev3 t3{};
  long long* d_fixed = nullptr;      // fixed-point copy of x (lazily allocated, D entries)
  int* d_exp = nullptr;              // exponent scratch of the fixed-point path
  std::vector<int> cross_cls;        // class of each cross bond
  // per-stage CUDA-event timing of apply_H (ed_profile_*)
  bool prof = false;
  std::vector<cudaEvent_t> prof_ev;  // 5 events per recorded apply
  double prof_ms[4] = {0, 0, 0, 0};
  int64_t prof_count = 0;
  // per-side CSR stats
  int64_t nnzA = 0, nnzB = 0;
  // Lanczos / GF work buffers (lazily allocated)
  void* work = nullptr;
  size_t work_bytes = 0;
  double* d_partials = nullptr;
  double* h_pinned = nullptr;
  cudaStream_t lz_stream = nullptr;  // private stream for captured Lanczos steps
  ~ed_ctx();
};

namespace edk {
// host copy of one side's operators (CSR over the side's global state index)
struct HostSideOps {
  std::vector<int> rowptr, col;
  std::vector<double> val64, diag;
  std::vector<float> val32;
  std::vector<unsigned long long> pack;
  std::vector<int> maps;  // [n_cross_bits][total]
};
ed_status build_side_ops(const ed_ctx* c, const Side& sd, const std::vector<ed_ctx::SideBond>& bonds, bool sideA,
                         HostSideOps& h);
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
