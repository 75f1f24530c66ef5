// Eigenvalues of dense symmetric FP64 matrices: Householder tridiagonal
// reduction on the GPU, then implicit-shift QL on the tridiagonal matrix.
#pragma once

#include <vector>

#include "ed_internal.h"

namespace edk {
// Reduce the symmetric m x m row-major A (device; only its lower triangle,
// diagonal included, is read and overwritten) to tridiagonal form; the
// diagonal (m) and off-diagonal (m - 1) entries are
// copied to the host arrays, asynchronously on `st` (synchronise before use).
// work: device scratch of tridiag_work_doubles(m) doubles.
inline long long tridiag_work_doubles(int m) { return 8LL * m + 2LL * ((m + 31) / 32) * m; }
ed_status tridiag_reduce(double* A, int m, double* work, double* d_host, double* e_host, cudaStream_t st, int sms);
// all eigenvalues of the tridiagonal (d, e) into d (unordered); false if the
// iteration did not converge
bool tridiag_eigenvalues(std::vector<double>& d, std::vector<double>& e);
}  // namespace edk
