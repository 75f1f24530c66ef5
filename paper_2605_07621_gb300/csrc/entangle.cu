// Entanglement spectrum across the cut: the spectrum xi = -log(lambda) of
// the entanglement Hamiltonian H_E = -log(rho_A), rho_A = Tr_B |psi><psi|,
// resolved by the conserved charge of side A (the paper's discussion of
// its figure "Distributed entanglement spectrum", with the sector weights W_q).
//
// In the block layout rho_A is block diagonal, rho_A(s) = Psi_s Psi_s^T, and
// its nonzero eigenvalues are those of the Gram matrix of Psi_s in the
// smaller of its two dimensions (the squared singular values of Psi_s).
// The Gram matrix is formed on the tensor cores by the FP64-accurate
// digit-split GEMM (ozaki.cu; one digit-plane buffer serves as both factors,
// only the tiles on or below the diagonal are computed: the matrix is
// symmetric); the eigenvalues of each Gram matrix come from cuSOLVER's dense
// symmetric divide-and-conquer eigensolver, which is loaded with dlopen on
// the first call so that the rest of the library does not depend on it.
#include <dlfcn.h>

#include <cmath>
#include <mutex>

#include <cusolverDn.h>

#include "krylov.h"
#include "ozaki.h"

namespace edk {
namespace {

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
  if (S.bufsize(H.h, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_UPPER, (int)mmax, G, (int)mmax, W, &lwork) !=
      CUSOLVER_STATUS_SUCCESS) {
    set_error("cuSOLVER workspace query failed");
    return ED_ECUDA;
  }
  ED_TRY(mem.get((void**)&work, (size_t)std::max(lwork, 1) * sizeof(double)));

  // digit planes of one block at a time (both factors of its Gram matrix),
  // tensor maps and launch lists of every block built up front
  OzContext oz;
  oz.device = c->device;
  OzOperand X;
  long long max_elems = 1;
  for (const Block& b : c->blocks) {
    const long long m = std::min(b.dA, b.dB), L = std::max(b.dA, b.dB);
    max_elems = std::max(max_elems, m * ((L + 7) / 8 * 8));
  }
  ED_TRY(oz_operand_buffer(&oz, max_elems, mmax, &X));
  std::vector<OzSliceJob> jobs;
  std::vector<OzProblem> probs;
  std::vector<long long> units, tiles;
  for (const Block& b : c->blocks) {
    const int m = (int)std::min(b.dA, b.dB), L = (int)std::max(b.dA, b.dB);
    int ma = 0, mb = 0;
    ED_TRY(oz_map(&oz, &X, m, L, true, &ma));
    ED_TRY(oz_map(&oz, &X, m, L, false, &mb));
    OzSliceJob j{};
    j.src = psi + b.off;
    j.sbase = 0;
    j.ld = b.dB;
    j.rows = (int)b.dA;
    j.cols = (int)b.dB;
    j.dst = X.slices;
    j.exps = X.exps;
    j.Kpad = (L + 7) / 8 * 8;
    j.first = 0;
    jobs.push_back(j);
    // Psi Psi^T (rows, dA <= dB) or Psi^T Psi (columns)
    units.push_back(b.dA <= b.dB ? (long long)b.dA : (b.dB + 31) / 32);
    OzProblem p{};
    p.mapA = ma;
    p.mapB = mb;
    p.ea = X.exps;
    p.eb = X.exps;
    p.C = G;
    p.cbase = 0;
    p.ldc = m;
    p.M = p.N = m;
    p.K = L;
    p.acc = 0;
    p.tiles_n = (m + kOzBN - 1) / kOzBN;
    p.tri = 1;
    p.tile0 = 0;
    probs.push_back(p);
    tiles.push_back(oz_tiles(m, m, 1));
  }
  ED_TRY(oz_finish(&oz));
  OzSliceJob* d_jobs = nullptr;
  OzProblem* d_probs = nullptr;
  ED_TRY(oz_alloc(&oz, (void**)&d_jobs, jobs.size() * sizeof(OzSliceJob)));
  ED_TRY(oz_alloc(&oz, (void**)&d_probs, probs.size() * sizeof(OzProblem)));
  ED_CUDA_TRY(cudaMemcpy(d_jobs, jobs.data(), jobs.size() * sizeof(OzSliceJob), cudaMemcpyHostToDevice));
  ED_CUDA_TRY(cudaMemcpy(d_probs, probs.data(), probs.size() * sizeof(OzProblem), cudaMemcpyHostToDevice));

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
    ED_CUDA_TRY(cudaEventRecord(ev.e[0], st));
    ED_TRY(oz_slice(&oz, d_jobs + bi, 1, units[bi], b.dA > b.dB, nullptr, st));
    ED_TRY(oz_gemm(&oz, d_probs + bi, 1, tiles[bi], nullptr, st));
    ED_CUDA_TRY(cudaEventRecord(ev.e[1], st));
    int lw = 0;
    if (S.bufsize(H.h, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_UPPER, m, G, m, W, &lw) !=
            CUSOLVER_STATUS_SUCCESS ||
        lw > lwork) {
      set_error("cuSOLVER workspace for dimension %d exceeds the one allocated", m);
      return ED_ECUDA;
    }
    if (S.syevd(H.h, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_UPPER, m, G, m, W, work, lwork, info) !=
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
