// Entanglement spectrum across the cut: the spectrum xi = -log(lambda) of
// the entanglement Hamiltonian H_E = -log(rho_A), rho_A = Tr_B |psi><psi|,
// resolved by the conserved charge of side A (the paper's discussion of
// its figure "Distributed entanglement spectrum", with the sector weights W_q).
//
// In the block layout rho_A is block diagonal, rho_A(s) = Psi_s Psi_s^T, and
// its nonzero eigenvalues are those of the Gram matrix of Psi_s in the
// smaller of its two dimensions (the squared singular values of Psi_s).
// The Gram matrix is formed on the tensor cores by the FP64-accurate
// digit-split GEMM (ozaki.cu; one digit-plane buffer serves as both
// factors, only the tiles on or below the diagonal), reduced to tridiagonal form on the GPU by Householder
// reflections, and its eigenvalues come from implicit-shift QL on the host,
// one thread per block while the GPU reduces the next block (eigsym.cu).
#include <cmath>
#include <algorithm>
#include <chrono>
#include <thread>

#include "krylov.h"
#include "eigsym.h"
#include "ozaki.h"

namespace edk {
namespace {

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
  if (mmax > 46340) {  // m * m must fit 32-bit index arithmetic of the reduction
    set_error("block Gram dimension %lld exceeds the dense eigensolver's limit", (long long)mmax);
    return ED_EUNSUPPORTED;
  }
  ED_DEVICE_SCOPE(c->device);
  ED_TRY(ensure_scratch(c));
  cudaStream_t st = (cudaStream_t)stream;
  DevMem mem;
  double *G = nullptr, *work = nullptr;
  ED_TRY(mem.get((void**)&G, (size_t)mmax * mmax * sizeof(double)));
  ED_TRY(mem.get((void**)&work, (size_t)std::max(tridiag_work_doubles((int)mmax),
                                                  tridiag_blocked_work_doubles((int)mmax)) *
                                     sizeof(double)));

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
    p.tri = 1;  // the lower triangle: all the reduction reads
    p.tile0 = 0;
    probs.push_back(p);
    tiles.push_back(oz_tiles(m, m, 1));
  }
  // the blocked reduction's trailing updates: panel buffers, digit planes,
  // and per block its panels' slicing jobs and products
  double *NVW = nullptr, *WV = nullptr;
  float2 *F = nullptr, *WVf = nullptr;
  OzOperand opA, opB;
  ED_TRY(mem.get((void**)&WVf, (size_t)mmax * 2 * kTriNb * sizeof(float2)));
  ED_TRY(mem.get((void**)&F, (size_t)mmax * tridiag_ldF((int)mmax) * sizeof(float2)));
  ED_CUDA_TRY(cudaMemsetAsync(F, 0, (size_t)mmax * tridiag_ldF((int)mmax) * sizeof(float2), st));
  ED_TRY(oz_alloc(&oz, (void**)&NVW, (size_t)mmax * 2 * kTriNb * sizeof(double)));
  ED_TRY(oz_alloc(&oz, (void**)&WV, (size_t)mmax * 2 * kTriNb * sizeof(double)));
  ED_TRY(oz_operand_buffer(&oz, mmax * 2 * kTriNb, mmax, &opA));
  ED_TRY(oz_operand_buffer(&oz, mmax * 2 * kTriNb, mmax, &opB));
  std::vector<OzSliceJob> tjobs;
  std::vector<OzProblem> tprobs;
  std::vector<size_t> toff(c->blocks.size());
  for (size_t bi = 0; bi < c->blocks.size(); ++bi) {
    const Block& b = c->blocks[bi];
    toff[bi] = tprobs.size();
    ED_TRY(tridiag_blocked_setup(&oz, G, (int)std::min(b.dA, b.dB), opA, opB, NVW, WV, tjobs, tprobs));
  }
  ED_TRY(oz_finish(&oz));
  OzSliceJob* d_tjobs = nullptr;
  OzProblem* d_tprobs = nullptr;
  if (!tprobs.empty()) {
    ED_TRY(oz_alloc(&oz, (void**)&d_tjobs, tjobs.size() * sizeof(OzSliceJob)));
    ED_TRY(oz_alloc(&oz, (void**)&d_tprobs, tprobs.size() * sizeof(OzProblem)));
    ED_CUDA_TRY(cudaMemcpy(d_tjobs, tjobs.data(), tjobs.size() * sizeof(OzSliceJob), cudaMemcpyHostToDevice));
    ED_CUDA_TRY(cudaMemcpy(d_tprobs, tprobs.data(), tprobs.size() * sizeof(OzProblem), cudaMemcpyHostToDevice));
  }
  OzSliceJob* d_jobs = nullptr;
  OzProblem* d_probs = nullptr;
  ED_TRY(oz_alloc(&oz, (void**)&d_jobs, jobs.size() * sizeof(OzSliceJob)));
  ED_TRY(oz_alloc(&oz, (void**)&d_probs, probs.size() * sizeof(OzProblem)));
  ED_CUDA_TRY(cudaMemcpy(d_jobs, jobs.data(), jobs.size() * sizeof(OzSliceJob), cudaMemcpyHostToDevice));
  ED_CUDA_TRY(cudaMemcpy(d_probs, probs.data(), probs.size() * sizeof(OzProblem), cudaMemcpyHostToDevice));

  std::vector<double> wt(c->blocks.size());
  // per block: its tridiagonal matrix, handed to a host thread for the QL
  // steps while the GPU forms and reduces the next block
  std::vector<std::vector<double>> dd(c->blocks.size()), ee(c->blocks.size());
  std::vector<char> ok(c->blocks.size(), 1);
  std::vector<std::thread> qr;
  struct Joiner {
    std::vector<std::thread>* t;
    ~Joiner() {
      for (auto& x : *t)
        if (x.joinable()) x.join();
    }
  } joiner{&qr};
  Events ev;
  for (cudaEvent_t& x : ev.e) ED_CUDA_TRY(cudaEventCreate(&x));
  double t_gram = 0.0, t_red = 0.0;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    cudaGetLastError();
    sms = 148;
  }
  // largest blocks first: their host QL runs while the GPU handles the rest
  std::vector<size_t> order(c->blocks.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t u, size_t v) {
    return std::min(c->blocks[u].dA, c->blocks[u].dB) > std::min(c->blocks[v].dA, c->blocks[v].dB);
  });
  for (size_t bi : order) {
    const Block& b = c->blocks[bi];
    const double* xb = psi + b.off;
    const int m = (int)std::min(b.dA, b.dB);
    // Gram matrix in the smaller dimension: Psi Psi^T (rows) or Psi^T Psi (columns)
    ED_CUDA_TRY(cudaEventRecord(ev.e[0], st));
    ED_TRY(oz_slice(&oz, d_jobs + bi, 1, units[bi], b.dA > b.dB, nullptr, st));
    ED_TRY(oz_gemm(&oz, d_probs + bi, 1, tiles[bi], nullptr, st));
    ED_CUDA_TRY(cudaEventRecord(ev.e[1], st));
    dd[bi].assign(m, 0.0);
    ee[bi].assign(std::max(m - 1, 1), 0.0);
    TriBlocked tb{&oz, NVW, WV, WVf, F, tridiag_ldF(m), {}, oz.d_err, d_tjobs + 2 * toff[bi], d_tprobs + toff[bi]};
    if (m >= 3) ED_TRY(tmap_8b_2d(&tb.tmF, F, m, m, tb.ldF, 34, 32));
    ED_TRY(tridiag_reduce_blocked(G, m, work, dd[bi].data(), ee[bi].data(), st, sms, tb));
    ED_CUDA_TRY(cudaEventRecord(ev.e[2], st));
    // ||Psi_s||^2 (the trace of rho_A(s)) with the library's FP64 reduction
    ED_TRY(dot_dev<double>(c, xb, xb, b.dA * b.dB, slot(c, 3), st, 0));
    ED_TRY(read_scalars(c, 3, 1, &wt[bi], st));  // synchronises the stream
    ED_TRY(oz_status(&oz, st));                   // no bounded wait of the block's kernels ran out
    float t1 = 0.f, t2 = 0.f;
    ED_CUDA_TRY(cudaEventElapsedTime(&t1, ev.e[0], ev.e[1]));
    ED_CUDA_TRY(cudaEventElapsedTime(&t2, ev.e[1], ev.e[2]));
    t_gram += t1;
    t_red += t2;
    ee[bi].resize(std::max(m - 1, 0));
    qr.emplace_back([&dd, &ee, &ok, bi] { ok[bi] = tridiag_eigenvalues(dd[bi], ee[bi]) ? 1 : 0; });
  }
  const auto tq = std::chrono::steady_clock::now();
  for (auto& x : qr) x.join();
  const double t_qr = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tq).count();
  int64_t pos = 0;
  for (size_t bi = 0; bi < c->blocks.size(); ++bi) {
    if (!ok[bi]) {
      set_error("tridiagonal QL did not converge on block %zu", bi);
      return ED_ENOCONV;
    }
    std::vector<double>& w = dd[bi];
    std::sort(w.begin(), w.end(), [](double u, double v) { return u > v; });  // descending
    for (size_t i = 0; i < w.size(); ++i) lambda[pos + i] = w[i];
    pos += (int64_t)w.size();
  }
  if (stage_ms) {
    stage_ms[0] = t_gram;
    stage_ms[1] = t_red + t_qr;  // GPU reduction plus the host QL left after the last block
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
