// Eigenvalues of dense symmetric FP64 matrices: Householder tridiagonal
// reduction on the GPU, then implicit-shift QL on the tridiagonal matrix.
#pragma once

#include <vector>

#include "ed_internal.h"
#include "ozaki.h"

namespace edk {
// Blocked reduction: panels of kTriNb reflectors, each followed by the
// trailing update A -= V W^T + W V^T as one FP64-accurate tensor-core product
constexpr int kTriNb = 64;
struct TriPanel {
  int k0, jb, t0;  // first column, reflectors, first row of the trailing matrix
};
std::vector<TriPanel> tridiag_panels(int m);
// the panel buffers (device [m][2 kTriNb] FP64 each, and WVf), the float-float copy
// of the matrix (device [m][ldF] float2, ldF = tridiag_ldF(m); every value
// finite, since the reduction also reads entries outside the trailing
// triangle, multiplied by zero), a 2-D tensor map over it (m x m 8-byte
// elements, row stride ldF, box 34 x 32), the flag that bounded waits set,
// and, per panel, two slicing jobs and one product (built by
// tridiag_blocked_setup, on device)
inline long long tridiag_ldF(int m) { return m + (m & 1); }
struct TriBlocked {
  OzContext* oz;
  double* NVW;
  double* WV;
  float2* WVf;  // the panel's W and sigma V as float-float pairs (device [m][2 kTriNb])
  float2* F;
  long long ldF;
  CUtensorMap tmF;
  int* err;
  const OzSliceJob* d_jobs;
  const OzProblem* d_probs;
};
// appends the jobs and products of an m x m reduction of A (tensor maps in oz;
// opA / opB: digit-plane buffers for m x 2 kTriNb operands)
ed_status tridiag_blocked_setup(OzContext* oz, double* A, int m, const OzOperand& opA, const OzOperand& opB,
                                const double* NVW, const double* WV, std::vector<OzSliceJob>& jobs,
                                std::vector<OzProblem>& probs);
inline long long tridiag_blocked_work_doubles(int m) {
  return 6LL * m + 2LL * ((m + 63) / 64) * m + 128LL * (2 * kTriNb + 1) + 2 * kTriNb + 4096 + 1024 + 8;
}
// Reduce the symmetric m x m row-major A (device; only its lower triangle,
// diagonal included, is read and overwritten) to tridiagonal form; the
// diagonal (m) and off-diagonal (m - 1) entries are copied to the host
// arrays (pinned), asynchronously on `st` (wait on the stream before use).
// work: device scratch of tridiag_blocked_work_doubles(m) doubles.
ed_status tridiag_reduce_blocked(double* A, int m, double* work, double* d_host, double* e_host, cudaStream_t st,
                                 int sms, const TriBlocked& tb);
// all eigenvalues of the tridiagonal (d, e) into d (unordered); false if the
// iteration did not converge
bool tridiag_eigenvalues(std::vector<double>& d, std::vector<double>& e);
}  // namespace edk
