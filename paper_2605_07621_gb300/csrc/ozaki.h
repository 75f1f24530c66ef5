// FP64-accurate matrix products on the BF16 tensor cores (Ozaki-style
// splitting).  Each row of an operand is scaled by a power of two 2^E (E per
// row) and written as 8 signed base-64 digits, each exact in BF16; a digit
// product is exact in FP32 and a K-sum of up to kOzKChunk products of one
// digit order stays an exact integer in the FP32 accumulator, so
//   C = sum_{p+q <= 7} 2^(E_A + E_B - 10 - 6 (p+q)) sum_k a_p b_q
// is formed with one FP64 rounding per digit order (the dropped orders
// p + q >= 8 are below 2^-48 of the leading one).
//   Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix
//   multiplication by using fast routines of matrix multiplication and its
//   applications", Numer. Algorithms 59 (2012).
#pragma once

#include <cuda.h>

#include <cstdint>
#include <vector>

#include "ed_internal.h"

namespace edk {

constexpr int kOzDigits = 8;    // digits per value
constexpr int kOzBits = 6;      // bits per digit (|digit| <= 32)
constexpr int kOzFrac = 47;     // value = U * 2^(E - 47), |U| <= 2^47
constexpr int kOzBM = 128;      // output tile rows (UMMA M)
constexpr int kOzBN = 64;       // output tile columns (UMMA N)
constexpr int kOzBK = 64;       // K per pipeline step (one 128-byte swizzle row of BF16)
constexpr int kOzKChunk = 2048; // 8 digit pairs x 2048 x 32^2 < 2^24: FP32 sums stay exact

// Digit planes of one matrix with R rows and K columns, K contiguous.
struct OzOperand {
  uint16_t* slices = nullptr;  // device [8][R][Kpad] BF16 bit patterns
  int* exps = nullptr;         // device [R]: E of each row (|v| < 2^E)
  int R = 0, K = 0, Kpad = 0;
  int map = -1;                // index into the owner's tensor-map table
};

// One product of a launch: C (M x N, row stride ldc) = or += A B, with A the
// M x K operand `a` and B^T the N x K operand `b` (both as digit planes).
struct OzProblem {
  int mapA, mapB;
  const int* ea;       // exponents of A's rows
  const int* eb;       // exponents of B^T's rows (C's columns)
  double* C;           // absolute address, or an offset into y (cbase = 1)
  long long coff;
  int cbase;
  long long ldc;
  int M, N, K, acc;
  int tiles_n;
  int tri;             // 1: only the tiles on or below the diagonal (C symmetric, its lower triangle)
  long long tile0;
};

// Tensor maps and device buffers of one set of operands.
struct OzContext {
  int device = 0;
  std::vector<CUtensorMap> maps;
  CUtensorMap* d_maps = nullptr;
  std::vector<void*> allocs;
  int* d_err = nullptr;
  ~OzContext();
};

ed_status oz_alloc(OzContext* o, void** p, size_t bytes);
// 3-D BF16 tensor map over `planes` planes of an R x K matrix (row stride
// Kpad elements, a multiple of 8; planes one after another), box
// (64, box_rows, 1), 128-byte swizzle, elements outside the matrix read as 0
ed_status tmap_bf16_planes(CUtensorMap* m, const void* base, int K, int R, int planes, long long Kpad, int box_rows);
// 2-D tensor map over a rows x cols matrix of 8-byte elements (row stride ld
// elements, ld * 8 a multiple of 16), box (box_cols, box_rows), no swizzle,
// elements outside the matrix read as 0
ed_status tmap_8b_2d(CUtensorMap* m, const void* base, long long cols, long long rows, long long ld, int box_cols,
                     int box_rows);
// reads and clears the flag that the tensor-core kernels set when one of
// their bounded waits ran out (synchronises the stream); ED_ECUDA if set
ed_status oz_status(OzContext* o, cudaStream_t st);
// operand from a host FP64 row-major matrix (digits formed on the host)
ed_status oz_operand_host(OzContext* o, const double* h, int R, int K, bool a_role, OzOperand* out);
// operand buffers filled on the device by oz_slice_* (no data yet)
ed_status oz_operand_device(OzContext* o, int R, int K, bool a_role, OzOperand* out);
ed_status oz_finish(OzContext* o);  // upload the tensor maps
// operand buffers for up to R x K (no map); a map over its first R rows and K
// columns (digit planes of an R x K operand with row stride Kpad)
ed_status oz_operand_buffer(OzContext* o, long long max_elems, long long max_rows, OzOperand* out);
ed_status oz_map(OzContext* o, OzOperand* op, int R, int K, bool a_role, int* map);

// digit planes of matrices on the device (FP64, row-major, leading dimension
// ld), one job per matrix; rows: the matrix rows become the operand's rows;
// cols: its columns do (the operand is the transpose, exponent per column)
struct OzSliceJob {
  const double* src;   // absolute, or offset into x (sbase = 1)
  long long soff;
  int sbase;
  long long ld;
  int rows, cols;      // of the source matrix
  uint16_t* dst;
  int* exps;
  int Kpad;            // of the destination operand
  long long first;     // first work unit of this job in the launch
};
ed_status oz_slice(OzContext* o, const OzSliceJob* d_jobs, int njobs, long long units, bool transpose,
                   const double* x, cudaStream_t st);
ed_status oz_gemm(OzContext* o, const OzProblem* d_probs, int nprob, long long tiles, double* y, cudaStream_t st);
long long oz_tiles(int M, int N, int tri = 0);
// host-side digit planes (for tests and static operands): U and digits of v
void oz_digits_host(double v, int E, int* d);
int oz_row_exponent(double maxabs);

}  // namespace edk
