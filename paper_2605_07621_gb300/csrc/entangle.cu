// Entanglement spectrum across the cut: the spectrum xi = -log(lambda) of
// the entanglement Hamiltonian H_E = -log(rho_A), rho_A = Tr_B |psi><psi|,
// resolved by the conserved charge of side A (the paper's discussion of
// its figure "Distributed entanglement spectrum", with the sector weights W_q).
//
// In the block layout rho_A is block diagonal, rho_A(s) = Psi_s Psi_s^T, and
// its nonzero eigenvalues are those of the Gram matrix of Psi_s in the
// smaller of its two dimensions (the squared singular values of Psi_s).
// k_gram forms that Gram matrix in FP64 (one 64 x 64 output tile per CTA,
// upper-triangle tiles only: the matrix is symmetric); the eigenvalues of
// each Gram matrix come from cuSOLVER's dense symmetric divide-and-conquer
// eigensolver, which is loaded with dlopen on the first call so that the
// rest of the library does not depend on it.
#include <dlfcn.h>

#include <cmath>
#include <mutex>

#include <cusolverDn.h>

#include "krylov.h"

namespace edk {
namespace {

constexpr int kGT = 64;  // output tile (rows and columns)
constexpr int kGK = 16;  // contraction depth staged per step

// G[i][j] = sum_l X(i,l) X(j,l) over the tiles (ti, tj) with ti <= tj, with
// X(i,l) = x[i*si + l*sl], 0 <= i < m, 0 <= l < L; G row-major, leading
// dimension m.  Its row-major upper triangle is the column-major lower
// triangle that the eigensolver reads.
__global__ void __launch_bounds__(256) k_gram(const double* __restrict__ x, long long si, long long sl, int m,
                                              long long L, double* __restrict__ G, int T) {
  __shared__ double As[kGK][kGT + 1];
  __shared__ double Bs[kGK][kGT + 1];
  int t = blockIdx.x, ti = 0;
  while (t >= T - ti) {
    t -= T - ti;
    ++ti;
  }
  const int tj = ti + t;
  const long long i0 = (long long)ti * kGT, j0 = (long long)tj * kGT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const bool lfast = sl == 1;  // the contraction index is the contiguous one
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
  for (long long l0 = 0; l0 < L; l0 += kGK) {
    for (int e = threadIdx.x; e < kGT * kGK; e += blockDim.x) {
      const int r = lfast ? e / kGK : e % kGT;
      const int l = lfast ? e % kGK : e / kGT;
      const long long gl = l0 + l, gi = i0 + r, gj = j0 + r;
      As[l][r] = (gi < m && gl < L) ? x[gi * si + gl * sl] : 0.0;
      Bs[l][r] = (gj < m && gl < L) ? x[gj * si + gl * sl] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kGK; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[k][ty + 16 * u];
        b[u] = Bs[k][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const long long i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
      if (i < m && j < m) G[i * m + j] = acc[u][v];
    }
}

// the five cuSOLVER entry points used here, resolved once
struct Solver {
  using create_t = cusolverStatus_t (*)(cusolverDnHandle_t*);
  using destroy_t = cusolverStatus_t (*)(cusolverDnHandle_t);
  using stream_t = cusolverStatus_t (*)(cusolverDnHandle_t, cudaStream_t);
  using bufsize_t = cusolverStatus_t (*)(cusolverDnHandle_t, cusolverEigMode_t, cublasFillMode_t, int, const double*,
                                         int, const double*, int*);
  using syevd_t = cusolverStatus_t (*)(cusolverDnHandle_t, cusolverEigMode_t, cublasFillMode_t, int, double*, int,
                                       double*, double*, int, int*);
  create_t create = nullptr;
  destroy_t destroy = nullptr;
  stream_t set_stream = nullptr;
  bufsize_t bufsize = nullptr;
  syevd_t syevd = nullptr;
  bool ok = false;
  std::string why;
};

const Solver& solver() {
  static Solver s;
  static std::once_flag once;
  std::call_once(once, [] {
    void* h = nullptr;
    for (const char* name : {"libcusolver.so.12", "libcusolver.so.11", "libcusolver.so"}) {
      h = dlopen(name, RTLD_NOW | RTLD_LOCAL);
      if (h) break;
    }
    if (!h) {
      const char* e = dlerror();
      s.why = std::string("cannot load cuSOLVER: ") + (e ? e : "unknown");
      return;
    }
    s.create = (Solver::create_t)dlsym(h, "cusolverDnCreate");
    s.destroy = (Solver::destroy_t)dlsym(h, "cusolverDnDestroy");
    s.set_stream = (Solver::stream_t)dlsym(h, "cusolverDnSetStream");
    s.bufsize = (Solver::bufsize_t)dlsym(h, "cusolverDnDsyevd_bufferSize");
    s.syevd = (Solver::syevd_t)dlsym(h, "cusolverDnDsyevd");
    s.ok = s.create && s.destroy && s.set_stream && s.bufsize && s.syevd;
    if (!s.ok) s.why = "cuSOLVER lacks the dense symmetric eigensolver entry points";
  });
  return s;
}

struct DevMem {
  std::vector<void*> p;
  ~DevMem() {
    for (void* q : p) cudaFree(q);
  }
  ed_status get(void** out, size_t bytes) {
    cudaError_t e = cudaMalloc(out, bytes < 16 ? 16 : bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMalloc(%zu) for the entanglement spectrum failed: %s", bytes, cudaGetErrorString(e));
      return ED_ENOMEM;
    }
    p.push_back(*out);
    return ED_OK;
  }
};

struct Handle {
  cusolverDnHandle_t h = nullptr;
  ~Handle() {
    if (h) solver().destroy(h);
  }
};

struct Events {
  cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
  ~Events() {
    for (cudaEvent_t x : e)
      if (x) cudaEventDestroy(x);
  }
};

}  // namespace
}  // namespace edk

using namespace edk;

extern "C" ed_status ed_entanglement_spectrum(ed_ctx* c, const double* psi, double* lambda, int64_t cap,
                                              int64_t* n_lambda, double* weight, double* entropy, double* stage_ms,
                                              void* stream) {
  if (!c || !n_lambda) {
    set_error("ctx or n_lambda is NULL");
    return ED_EINVAL;
  }
  int64_t need = 0, mmax = 0;
  for (const Block& b : c->blocks) {
    const int64_t m = std::min(b.dA, b.dB);
    need += m;
    mmax = std::max(mmax, m);
  }
  *n_lambda = need;
  if (!lambda) return ED_OK;  // size query
  if (!psi) {
    set_error("psi is NULL");
    return ED_EINVAL;
  }
  if (cap < need) {
    set_error("lambda holds %lld values, %lld needed", (long long)cap, (long long)need);
    return ED_EINVAL;
  }
  if (mmax > 46340) {  // m * m must fit the eigensolver's int sizes
    set_error("block Gram dimension %lld exceeds the dense eigensolver's limit", (long long)mmax);
    return ED_EUNSUPPORTED;
  }
  const Solver& S = solver();
  if (!S.ok) {
    set_error("%s", S.why.c_str());
    return ED_EUNSUPPORTED;
  }
  ED_DEVICE_SCOPE(c->device);
  ED_TRY(ensure_scratch(c));
  cudaStream_t st = (cudaStream_t)stream;
  Handle H;
  if (S.create(&H.h) != CUSOLVER_STATUS_SUCCESS || S.set_stream(H.h, st) != CUSOLVER_STATUS_SUCCESS) {
    set_error("cuSOLVER handle creation failed");
    return ED_ECUDA;
  }
  DevMem mem;
  double *G = nullptr, *W = nullptr, *work = nullptr;
  int* info = nullptr;
  ED_TRY(mem.get((void**)&G, (size_t)mmax * mmax * sizeof(double)));
  ED_TRY(mem.get((void**)&W, (size_t)mmax * sizeof(double)));
  ED_TRY(mem.get((void**)&info, sizeof(int)));
  int lwork = 0;
  if (S.bufsize(H.h, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, (int)mmax, G, (int)mmax, W, &lwork) !=
      CUSOLVER_STATUS_SUCCESS) {
    set_error("cuSOLVER workspace query failed");
    return ED_ECUDA;
  }
  ED_TRY(mem.get((void**)&work, (size_t)std::max(lwork, 1) * sizeof(double)));

  std::vector<double> w(mmax);
  std::vector<double> wt(c->blocks.size());
  Events ev;
  for (cudaEvent_t& x : ev.e) ED_CUDA_TRY(cudaEventCreate(&x));
  double t_gram = 0.0, t_eig = 0.0;
  int64_t pos = 0;
  for (size_t bi = 0; bi < c->blocks.size(); ++bi) {
    const Block& b = c->blocks[bi];
    const double* xb = psi + b.off;
    const int m = (int)std::min(b.dA, b.dB);
    // Gram matrix in the smaller dimension: Psi Psi^T (rows) or Psi^T Psi (columns)
    const bool rows = b.dA <= b.dB;
    const long long si = rows ? b.dB : 1, sl = rows ? 1 : b.dB, L = rows ? b.dB : b.dA;
    const int T = (m + kGT - 1) / kGT;
    const long long tiles = (long long)T * (T + 1) / 2;
    ED_CUDA_TRY(cudaEventRecord(ev.e[0], st));
    k_gram<<<(unsigned)tiles, 256, 0, st>>>(xb, si, sl, m, L, G, T);
    ED_CUDA_TRY(cudaGetLastError());
    ED_CUDA_TRY(cudaEventRecord(ev.e[1], st));
    int lw = 0;
    if (S.bufsize(H.h, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, m, G, m, W, &lw) !=
            CUSOLVER_STATUS_SUCCESS ||
        lw > lwork) {
      set_error("cuSOLVER workspace for dimension %d exceeds the one allocated", m);
      return ED_ECUDA;
    }
    if (S.syevd(H.h, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, m, G, m, W, work, lwork, info) !=
        CUSOLVER_STATUS_SUCCESS) {
      set_error("cuSOLVER eigensolver failed on block %zu (dimension %d)", bi, m);
      return ED_ECUDA;
    }
    ED_CUDA_TRY(cudaEventRecord(ev.e[2], st));
    int hinfo = 0;
    ED_CUDA_TRY(cudaMemcpyAsync(w.data(), W, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, st));
    ED_CUDA_TRY(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
    // ||Psi_s||^2 (the trace of rho_A(s)) with the library's FP64 reduction
    ED_TRY(dot_dev<double>(c, xb, xb, b.dA * b.dB, slot(c, 3), st, 0));
    ED_TRY(read_scalars(c, 3, 1, &wt[bi], st));  // synchronises the stream
    float t1 = 0.f, t2 = 0.f;
    ED_CUDA_TRY(cudaEventElapsedTime(&t1, ev.e[0], ev.e[1]));
    ED_CUDA_TRY(cudaEventElapsedTime(&t2, ev.e[1], ev.e[2]));
    t_gram += t1;
    t_eig += t2;
    if (hinfo != 0) {
      set_error("cuSOLVER eigensolver reported info=%d on block %zu", hinfo, bi);
      return ED_ECUDA;
    }
    for (int i = 0; i < m; ++i) lambda[pos + i] = w[m - 1 - i];  // descending
    pos += m;
  }
  if (stage_ms) {
    stage_ms[0] = t_gram;
    stage_ms[1] = t_eig;
  }
  double tot = 0.0;
  for (double v : wt) tot += v;
  if (weight)
    for (size_t bi = 0; bi < wt.size(); ++bi) weight[bi] = wt[bi];
  if (entropy) {
    // von Neumann entropy of the normalised spectrum; eigenvalues at or below
    // zero (rounding of a rank-deficient block) carry no weight
    double s = 0.0;
    if (tot > 0.0)
      for (int64_t i = 0; i < need; ++i) {
        const double p = lambda[i] / tot;
        if (p > 0.0) s -= p * std::log(p);
      }
    *entropy = s;
  }
  return ED_OK;
}
