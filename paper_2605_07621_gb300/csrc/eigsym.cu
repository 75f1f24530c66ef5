// Eigenvalues of a dense symmetric FP64 matrix (the Gram matrices of the
// entanglement spectrum), in two stages:
//  1. Householder reduction to tridiagonal form on the GPU (Golub and Van
//     Loan, Matrix Computations, Sec. 8.3.1): step k takes the Householder
//     reflector H_k = I - beta v v^T of column k below the diagonal and
//     applies H_k A H_k = A - v w^T - w v^T to the trailing matrix, with
//     p = beta A v and w = p - (beta p.v / 2) v.  Only the lower triangle is
//     stored and touched.  The rank-2 update of step k and the product A v of
//     step k + 1 share one pass over 32 x 32 tiles of that triangle (the next
//     reflector comes from the next column updated on the fly); a tile writes
//     its row sums and, below the diagonal, its column sums to slots of its
//     own that a second kernel adds up, so each step reads and writes the
//     stored triangle once.
//  2. The eigenvalues of the tridiagonal matrix by implicit QL steps with
//     shifts and deflation, on the host, one thread per matrix.
#include <algorithm>
#include <cmath>
#include <vector>

#include "eigsym.h"

namespace edk {
namespace {

constexpr int kEigThreads = 1024;

__device__ inline double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = l < (int)(blockDim.x >> 5) ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (l == 0) red[32] = v;
  }
  __syncthreads();
  return red[32];
}

// Reflector of column c of the matrix after the pending update of step k - 1
// (v, w of that step; have_prev = 0 for the first column): rows c+1 .. m-1.
// Writes v_c (rows c+1..), beta_c, the diagonal d_c and off-diagonal e_c.
__global__ void __launch_bounds__(kEigThreads) k_reflector(const double* __restrict__ A, int m, int c,
                                                           const double* __restrict__ vprev,
                                                           const double* __restrict__ wprev, int have_prev,
                                                           double* __restrict__ v, double* beta, double* d,
                                                           double* e) {
  __shared__ double red[33];
  const long long ld = m;
  // updated column c: A[i][c] - vprev[i] wprev[c] - wprev[i] vprev[c]
  const double vc = have_prev ? vprev[c] : 0.0, wc = have_prev ? wprev[c] : 0.0;
  double s2 = 0.0;
  for (int i = c + 1 + threadIdx.x; i < m; i += blockDim.x) {
    double x = A[(long long)i * ld + c];
    if (have_prev) x -= vprev[i] * wc + wprev[i] * vc;
    v[i] = x;
    if (i > c + 1) s2 += x * x;
  }
  const double tail = block_sum(s2, red);  // sum of squares below the first entry
  if (threadIdx.x == 0) {
    double dc = A[(long long)c * ld + c];
    if (have_prev) dc -= 2.0 * vc * wc;
    d[c] = dc;
    const double x0 = v[c + 1];
    const double nrm = sqrt(x0 * x0 + tail);
    if (tail == 0.0) {  // nothing to annihilate
      e[c] = x0;
      beta[c] = 0.0;
    } else {
      const double alpha = x0 >= 0.0 ? -nrm : nrm;
      v[c + 1] = x0 - alpha;
      beta[c] = 1.0 / (nrm * (nrm + fabs(x0)));  // 2 / (v.v) with v.v = 2 nrm (nrm + |x0|)
      e[c] = alpha;
    }
  }
}

// One pass over the lower triangle of the trailing matrix (rows and columns
// >= r0) in 32 x 32 tiles: apply the pending update of step r0 - 1 (if
// have_upd) and, if have_next, write the tile's partial sums of p = A vn
// (rows and columns >= r0 + 1): each stored a_ij (j < i) counts for row i and
// for row j, a diagonal entry once.  Tile (I, J), J <= I (numbered row by
// row, relative to r0) writes its row sums to slot J and its column sums to
// slot T + I of `part` (slot s, row i at part[s * m + i]; T = tile rows of
// the whole matrix), so no two tiles write one place; k_psum adds the slots.
// One warp per tile, lane = column: the column sums stay in registers; the
// products of each row go through a 32 x 33 shared-memory tile so that lane
// r adds row r (one FP64 add per element, the FP64 pipe being this GPU's
// bottleneck here, instead of a shuffle reduction per row).
constexpr int kT = 32;
constexpr int kEigWarps = 4;
__global__ void __launch_bounds__(32 * kEigWarps) k_update_matvec(double* __restrict__ A, int m, int r0,
                                                                  const double* __restrict__ vu,
                                                                  const double* __restrict__ wu, int have_upd,
                                                                  const double* __restrict__ vn, int have_next,
                                                                  double* __restrict__ part, int T, long long ntiles) {
  __shared__ double prod[kEigWarps][kT][kT + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long ld = m;
  const long long warps = (long long)gridDim.x * kEigWarps;
  for (long long t = (long long)blockIdx.x * kEigWarps + wid; t < ntiles; t += warps) {
    // tile (I, J) of the triangle: t = I (I + 1) / 2 + J
    long long I = (long long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (I * (I + 1) / 2 > t) --I;
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    const long long J = t - I * (I + 1) / 2;
    const int i0 = r0 + (int)I * kT, j = r0 + (int)J * kT + lane;
    const bool jin = j < m;
    const double vj = jin && have_upd ? __ldg(vu + j) : 0.0, wj = jin && have_upd ? __ldg(wu + j) : 0.0;
    const double nj = jin && have_next && j > r0 ? __ldg(vn + j) : 0.0;
    double csum = 0.0;
    const int rows = min(kT, m - i0);
#pragma unroll 4
    for (int li = 0; li < rows; ++li) {
      const int i = i0 + li;
      double rp = 0.0;
      if (jin && j <= i) {
        double* ap = A + (long long)i * ld + j;
        double a = *ap;
        if (have_upd) {
          a -= __ldg(vu + i) * wj + __ldg(wu + i) * vj;
          *ap = a;
        }
        if (have_next) {
          rp = a * nj;                                     // row i, column j
          if (j < i && i > r0) csum += a * __ldg(vn + i);  // row j, column i (mirror)
        }
      }
      if (have_next) prod[wid][li][lane] = rp;
    }
    if (have_next) {
      __syncwarp();
      if (lane < rows) {
        double rs = 0.0;
#pragma unroll 8
        for (int q = 0; q < kT; ++q) rs += prod[wid][lane][q];
        part[(long long)J * ld + i0 + lane] = rs;
      }
      if (jin) part[(long long)(T + I) * ld + j] = csum;
      __syncwarp();
    }
  }
}

// p[i] for rows i > r0: the row slots 0 .. I(i) and the column slots
// T + I(i) .. T + Tn - 1 that the tile pass wrote (I(i) = tile row of i,
// Tn = tile rows of the trailing matrix); one warp per row, lanes over slots
__global__ void __launch_bounds__(256) k_psum(const double* __restrict__ part, int m, int r0, int T, int Tn,
                                              double* __restrict__ p) {
  const int lane = threadIdx.x & 31;
  const long long ld = m;
  const int warps = gridDim.x * (blockDim.x >> 5);
  for (int i = r0 + 1 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < m; i += warps) {
    const int Ii = (i - r0) / kT;
    double s = 0.0;
    for (int J = lane; J <= Ii; J += 32) s += part[(long long)J * ld + i];
    for (int I2 = Ii + lane; I2 < Tn; I2 += 32) s += part[(long long)(T + I2) * ld + i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) p[i] = s;
  }
}

// w = beta p - (beta^2 p.v / 2) v over rows c+1..m-1 (p = A v without beta)
__global__ void __launch_bounds__(kEigThreads) k_wvec(int m, int c, const double* __restrict__ v,
                                                      const double* __restrict__ p, const double* beta,
                                                      double* __restrict__ w) {
  __shared__ double red[33];
  const double b = beta[c];
  double s = 0.0;
  for (int i = c + 1 + threadIdx.x; i < m; i += blockDim.x) s += p[i] * v[i];
  const double pv = block_sum(s, red);
  const double K = 0.5 * b * b * pv;
  for (int i = c + 1 + threadIdx.x; i < m; i += blockDim.x) w[i] = b * p[i] - K * v[i];
}

// the last 2 x 2 (or 1 x 1) block after every reflector was applied
__global__ void k_tail(const double* __restrict__ A, int m, double* d, double* e) {
  if (threadIdx.x != 0) return;
  const long long ld = m;
  d[m - 1] = A[(long long)(m - 1) * ld + (m - 1)];
  if (m >= 2) {
    d[m - 2] = A[(long long)(m - 2) * ld + (m - 2)];
    e[m - 2] = A[(long long)(m - 1) * ld + (m - 2)];
  }
}

}  // namespace

ed_status tridiag_reduce(double* A, int m, double* work, double* d_host, double* e_host, cudaStream_t st,
                         int sms) {
  if (m <= 0) return ED_OK;
  double* v[2] = {work, work + m};
  double* w[2] = {work + 2 * m, work + 3 * m};
  double* p = work + 4 * m;
  double* beta = work + 5 * m;
  double* d = work + 6 * m;
  double* e = work + 7 * m;
  const int T = (m + kT - 1) / kT;
  double* part = work + 8 * m;  // 2 T slots of m
  auto tri = [](int n) { const long long t = (n + kT - 1) / kT; return t * (t + 1) / 2; };
  auto grid = [&](long long nt) { return (unsigned)std::max<long long>(1, std::min<long long>(nt, (long long)sms * 8)); };
  auto pass = [&](int r0, const double* vu, const double* wu, int upd, const double* vn, int nxt) {
    const int n = m - r0;
    const long long nt = tri(n);
    k_update_matvec<<<grid((nt + kEigWarps - 1) / kEigWarps), 32 * kEigWarps, 0, st>>>(A, m, r0, vu, wu, upd, vn,
                                                                                       nxt, part, T, nt);
    if (nxt) {
      const int Tn = (n + kT - 1) / kT;
      k_psum<<<(unsigned)std::max(1, std::min((n + 7) / 8, sms * 8)), 256, 0, st>>>(part, m, r0, T, Tn, p);
    }
  };
  if (m >= 3) {
    // step 0: reflector of column 0, p = A v over the trailing matrix, w
    k_reflector<<<1, kEigThreads, 0, st>>>(A, m, 0, nullptr, nullptr, 0, v[0], beta, d, e);
    pass(0, nullptr, nullptr, 0, v[0], 1);
    k_wvec<<<1, kEigThreads, 0, st>>>(m, 0, v[0], p, beta, w[0]);
    for (int k = 0; k <= m - 3; ++k) {
      const int cur = k & 1, nxt = cur ^ 1;
      const bool more = k + 1 <= m - 3;
      if (more)
        k_reflector<<<1, kEigThreads, 0, st>>>(A, m, k + 1, v[cur], w[cur], 1, v[nxt], beta, d, e);
      // update with (v_k, w_k) on rows/columns >= k+1, product with v_{k+1}
      pass(k + 1, v[cur], w[cur], 1, v[nxt], more ? 1 : 0);
      if (more) k_wvec<<<1, kEigThreads, 0, st>>>(m, k + 1, v[nxt], p, beta, w[nxt]);
    }
  }
  k_tail<<<1, 32, 0, st>>>(A, m, d, e);
  ED_CUDA_TRY(cudaGetLastError());
  ED_CUDA_TRY(cudaMemcpyAsync(d_host, d, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (m >= 2) ED_CUDA_TRY(cudaMemcpyAsync(e_host, e, (size_t)(m - 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
  return ED_OK;
}

// All eigenvalues of the symmetric tridiagonal matrix (d, e) by implicit QL
// steps (Bowdler, Martin, Reinsch and Wilkinson, "The QR and QL algorithms
// for symmetric matrices", Numer. Math. 11, 1968): for the unreduced block
// starting at row l, a shift from its leading 2 x 2, then plane rotations
// chased from the bottom of the block up, in the recurrences that carry the
// running quantities (g, p) instead of forming each rotated 2 x 2 -- the
// numerically favoured form.  e[i] couples i and i+1; d is overwritten with
// the eigenvalues (unordered), each within a few eps of the matrix norm.
// false if a block needs more than 60 steps.
bool tridiag_eigenvalues(std::vector<double>& d, std::vector<double>& e) {
  const int n = (int)d.size();
  if (n <= 1) return true;
  e.resize(n);
  e[n - 1] = 0.0;
  const double eps = std::ldexp(1.0, -53);
  // an off-diagonal counts as zero below eps times its neighbours or below
  // eps times the norm of the whole matrix (eigenvalues far below the norm,
  // here the many vanishing ones of a Gram matrix, are resolved absolutely)
  double tnorm = 0.0;
  for (int i = 0; i < n; ++i)
    tnorm = std::max(tnorm, std::fabs(d[i]) + (i > 0 ? std::fabs(e[i - 1]) : 0.0) + std::fabs(e[i]));
  const double tiny = eps * tnorm;
  for (int l = 0; l < n; ++l) {
    for (int iter = 0;; ++iter) {
      int m = l;  // end of the unreduced block that starts at l
      while (m < n - 1 && std::fabs(e[m]) > eps * (std::fabs(d[m]) + std::fabs(d[m + 1])) && std::fabs(e[m]) > tiny)
        ++m;
      if (m == l) break;
      if (iter == 60) return false;
      // shift: the eigenvalue of the leading 2 x 2 nearer d[l]
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = std::hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + std::copysign(r, g));
      double s = 1.0, c = 1.0, p = 0.0;
      bool split = false;
      for (int i = m - 1; i >= l; --i) {
        const double f = s * e[i], b = c * e[i];
        r = std::hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {  // the rotation vanished: the block splits at i + 1
          d[i + 1] -= p;
          e[m] = 0.0;
          split = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * b;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - b;
      }
      if (split) continue;
      d[l] -= p;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  return true;
}

}  // namespace edk
