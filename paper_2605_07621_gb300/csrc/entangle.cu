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
// factors, only the tiles on or below the diagonal), reduced to tridiagonal
// form on the GPU by Householder reflections (eigsym.cu), and its eigenvalues
// come from implicit-shift QL on the host, one thread per block as soon as
// its tridiagonal matrix is ready.  Blocks run concurrently on a few streams.
#include <cmath>
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <string>
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
  const size_t nb = c->blocks.size();
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    cudaGetLastError();
    sms = 148;
  }

  // The blocks are reduced concurrently on up to kLanes streams ("lanes"):
  // a column's kernels are short and leave most of the GPU idle on all but
  // the largest blocks, so other blocks' columns fill it.  The largest block
  // goes first and alone (its host QL is the longest and overlaps everything
  // after it); the others go, largest first, to the lane with the least work
  // so far (cost ~ m^3 / 3 for the products plus a fixed cost per column);
  // each lane has its own buffers, sized for its largest block.
  constexpr int kLanes = 3;
  std::vector<size_t> order(nb);
  for (size_t i = 0; i < nb; ++i) order[i] = i;
  auto bm = [&](size_t i) { return (long long)std::min(c->blocks[i].dA, c->blocks[i].dB); };
  auto bl = [&](size_t i) { return (long long)std::max(c->blocks[i].dA, c->blocks[i].dB); };
  std::stable_sort(order.begin(), order.end(), [&](size_t u, size_t v) { return bm(u) > bm(v); });
  // device bytes of a lane sized for blocks up to (m, m x Lpad elements)
  auto lane_bytes = [&](long long m, long long xel) {
    const long long ldF = tridiag_ldF((int)m);
    return (double)m * m * 8 + (double)m * ldF * 8 + 3.0 * m * 2 * kTriNb * 8 +
           8.0 * tridiag_blocked_work_doubles((int)m) +
           2.0 * kOzDigits * xel + 2.0 * 2 * kOzDigits * m * 2 * kTriNb + 4.0 * m;
  };
  int lanes = kLanes;
  {
    size_t fr = 0, tot_mem = 0;
    if (cudaMemGetInfo(&fr, &tot_mem) != cudaSuccess) {
      cudaGetLastError();
      fr = 0;
    }
    long long m0 = nb ? bm(order[0]) : 1, x0 = 1;
    for (size_t i = 0; i < nb; ++i) x0 = std::max(x0, bm(i) * ((bl(i) + 7) / 8 * 8));
    const double one = lane_bytes(m0, x0);
    while (lanes > 1 && one * lanes > 0.8 * (double)fr) --lanes;
  }
  std::vector<int> lane_of(nb, 0);
  std::vector<std::vector<size_t>> lane_blocks(lanes);
  {
    // the largest block first, alone (lane 0; the other lanes start when it
    // is done), so that its host QL, the longest, overlaps all the rest
    std::vector<double> load(lanes, 0.0);
    if (nb) lane_blocks[0].push_back(order[0]);
    for (size_t oi = 1; oi < nb; ++oi) {
      const size_t bi = order[oi];
      const double m = (double)bm(bi);
      const double cost = m * m * m / 3.0 + 4e7 * m;
      const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      lane_of[bi] = k;
      load[k] += cost;
      lane_blocks[k].push_back(bi);
    }
  }
  while (lanes > 1 && lane_blocks[lanes - 1].empty()) --lanes;

  DevMem mem;
  OzContext oz;
  oz.device = c->device;
  struct Lane {
    long long mmax = 1, xel = 1;
    double *G = nullptr, *work = nullptr, *NVW = nullptr, *WV = nullptr;
    float2 *F = nullptr, *WVf = nullptr;
    OzOperand X, opA, opB;
    cudaStream_t s = nullptr;
  };
  std::vector<Lane> L(lanes);
  for (int k = 0; k < lanes; ++k) {
    for (size_t bi : lane_blocks[k]) {
      L[k].mmax = std::max(L[k].mmax, bm(bi));
      L[k].xel = std::max(L[k].xel, bm(bi) * ((bl(bi) + 7) / 8 * 8));
    }
    const long long mk = L[k].mmax;
    ED_TRY(mem.get((void**)&L[k].G, (size_t)mk * mk * sizeof(double)));
    ED_TRY(mem.get((void**)&L[k].work, (size_t)tridiag_blocked_work_doubles((int)mk) * sizeof(double)));
    ED_TRY(mem.get((void**)&L[k].F, (size_t)mk * tridiag_ldF((int)mk) * sizeof(float2)));
    ED_TRY(mem.get((void**)&L[k].WVf, (size_t)mk * 2 * kTriNb * sizeof(float2)));
    ED_TRY(oz_alloc(&oz, (void**)&L[k].NVW, (size_t)mk * 2 * kTriNb * sizeof(double)));
    ED_TRY(oz_alloc(&oz, (void**)&L[k].WV, (size_t)mk * 2 * kTriNb * sizeof(double)));
    ED_TRY(oz_operand_buffer(&oz, L[k].xel, mk, &L[k].X));
    ED_TRY(oz_operand_buffer(&oz, mk * 2 * kTriNb, mk, &L[k].opA));
    ED_TRY(oz_operand_buffer(&oz, mk * 2 * kTriNb, mk, &L[k].opB));
  }

  // per block: its Gram matrix (digit planes of Psi_s as both factors, the
  // tiles on or below the diagonal) and the trailing updates of its
  // reduction, in its lane's buffers; tensor maps and launch lists up front
  std::vector<OzSliceJob> jobs(nb);
  std::vector<OzProblem> probs(nb);
  std::vector<long long> units(nb), tiles(nb);
  std::vector<OzSliceJob> tjobs;
  std::vector<OzProblem> tprobs;
  std::vector<size_t> toff(nb);
  for (size_t bi = 0; bi < nb; ++bi) {
    const Block& b = c->blocks[bi];
    Lane& ln = L[lane_of[bi]];
    const int m = (int)bm(bi), Lg = (int)bl(bi);
    int ma = 0, mb = 0;
    ED_TRY(oz_map(&oz, &ln.X, m, Lg, true, &ma));
    ED_TRY(oz_map(&oz, &ln.X, m, Lg, false, &mb));
    OzSliceJob j{};
    j.src = psi + b.off;
    j.sbase = 0;
    j.ld = b.dB;
    j.rows = (int)b.dA;
    j.cols = (int)b.dB;
    j.dst = ln.X.slices;
    j.exps = ln.X.exps;
    j.Kpad = (Lg + 7) / 8 * 8;
    j.first = 0;
    jobs[bi] = j;
    // Psi Psi^T (rows, dA <= dB) or Psi^T Psi (columns)
    units[bi] = b.dA <= b.dB ? (long long)b.dA : (b.dB + 31) / 32;
    OzProblem p{};
    p.mapA = ma;
    p.mapB = mb;
    p.ea = ln.X.exps;
    p.eb = ln.X.exps;
    p.C = ln.G;
    p.cbase = 0;
    p.ldc = m;
    p.M = p.N = m;
    p.K = Lg;
    p.acc = 0;
    p.tiles_n = (m + kOzBN - 1) / kOzBN;
    p.tri = 1;  // the lower triangle: all the reduction reads
    p.tile0 = 0;
    probs[bi] = p;
    tiles[bi] = oz_tiles(m, m, 1);
    toff[bi] = tprobs.size();
    ED_TRY(tridiag_blocked_setup(&oz, ln.G, m, ln.opA, ln.opB, ln.NVW, ln.WV, tjobs, tprobs));
  }
  ED_TRY(oz_finish(&oz));
  OzSliceJob *d_tjobs = nullptr, *d_jobs = nullptr;
  OzProblem *d_tprobs = nullptr, *d_probs = nullptr;
  if (!tprobs.empty()) {
    ED_TRY(oz_alloc(&oz, (void**)&d_tjobs, tjobs.size() * sizeof(OzSliceJob)));
    ED_TRY(oz_alloc(&oz, (void**)&d_tprobs, tprobs.size() * sizeof(OzProblem)));
    ED_CUDA_TRY(cudaMemcpy(d_tjobs, tjobs.data(), tjobs.size() * sizeof(OzSliceJob), cudaMemcpyHostToDevice));
    ED_CUDA_TRY(cudaMemcpy(d_tprobs, tprobs.data(), tprobs.size() * sizeof(OzProblem), cudaMemcpyHostToDevice));
  }
  ED_TRY(oz_alloc(&oz, (void**)&d_jobs, nb * sizeof(OzSliceJob)));
  ED_TRY(oz_alloc(&oz, (void**)&d_probs, nb * sizeof(OzProblem)));
  ED_CUDA_TRY(cudaMemcpy(d_jobs, jobs.data(), nb * sizeof(OzSliceJob), cudaMemcpyHostToDevice));
  ED_CUDA_TRY(cudaMemcpy(d_probs, probs.data(), nb * sizeof(OzProblem), cudaMemcpyHostToDevice));

  // pinned host arrays for every block's tridiagonal matrix
  std::vector<size_t> hoff(nb + 1, 0);
  for (size_t bi = 0; bi < nb; ++bi) hoff[bi + 1] = hoff[bi] + 2 * (size_t)std::max(bm(bi), 1LL);
  struct Pinned {
    double* p = nullptr;
    ~Pinned() {
      if (p) cudaFreeHost(p);
    }
  } hde;
  ED_CUDA_TRY(cudaHostAlloc((void**)&hde.p, std::max<size_t>(hoff[nb], 1) * sizeof(double), cudaHostAllocDefault));
  struct EventSet {
    std::vector<cudaEvent_t> e;
    ~EventSet() {
      for (cudaEvent_t x : e)
        if (x) cudaEventDestroy(x);
    }
    ed_status make(size_t n) {
      e.assign(n, nullptr);
      for (cudaEvent_t& x : e) ED_CUDA_TRY(cudaEventCreate(&x));
      return ED_OK;
    }
  } ev_g0, ev_g1, ev_done, ev_lane, ev_se;
  ED_TRY(ev_g0.make(nb));
  ED_TRY(ev_g1.make(nb));
  ED_TRY(ev_done.make(nb));
  ED_TRY(ev_lane.make(lanes));
  ED_TRY(ev_se.make(3));
  struct Streams {
    std::vector<cudaStream_t> s;
    ~Streams() {
      for (cudaStream_t x : s) cudaStreamDestroy(x);
    }
  } own;
  ED_CUDA_TRY(cudaEventRecord(ev_se.e[0], st));
  for (int k = 0; k < lanes; ++k) {
    cudaStream_t s = nullptr;
    ED_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    own.s.push_back(s);
    L[k].s = s;
    ED_CUDA_TRY(cudaStreamWaitEvent(s, ev_se.e[0], 0));  // after the caller's work on its stream
  }
  // the reduction reads entries of F outside the trailing triangle (times
  // zero): every value must be finite
  for (int k = 0; k < lanes; ++k)
    ED_CUDA_TRY(cudaMemsetAsync(L[k].F, 0, (size_t)L[k].mmax * tridiag_ldF((int)L[k].mmax) * sizeof(float2), L[k].s));

  // per lane one host thread enqueues its blocks; per block one host thread
  // waits for its tridiagonal matrix and runs the QL steps
  std::vector<std::vector<double>> dd(nb), ee(nb);
  std::vector<char> ok(nb, 1);
  std::vector<std::thread> qr[kLanes];
  std::vector<std::thread> workers;
  struct Joiner {
    std::vector<std::thread>* t;
    int n;
    ~Joiner() {
      for (int i = 0; i < n; ++i)
        for (auto& x : t[i])
          if (x.joinable()) x.join();
    }
  };
  Joiner jq{qr, kLanes};
  Joiner jw{&workers, 1};
  std::vector<ed_status> lst(lanes, ED_OK);
  std::vector<std::string> lmsg(lanes);
  // lane 0 records first_done after the largest block; the other lanes'
  // streams wait for it (the host threads wait until it is recorded)
  std::mutex fm;
  std::condition_variable fcv;
  int first_state = 0;  // 0: not yet, 1: recorded, 2: lane 0 failed before it
  auto first_set = [&](int v) {
    {
      std::lock_guard<std::mutex> lk(fm);
      first_state = v;
    }
    fcv.notify_all();
  };
  auto lane_fn = [&](int k) {
    auto fail = [&](ed_status s) {
      lst[k] = s;
      lmsg[k] = ed_last_error();
      if (k == 0) first_set(2);
    };
    DeviceGuard dg(c->device);
    if (dg.status() != ED_OK) return fail(ED_ECUDA);
    Lane& ln = L[k];
    if (k > 0) {
      std::unique_lock<std::mutex> lk(fm);
      fcv.wait(lk, [&] { return first_state != 0; });
      if (first_state == 2) return;
      lk.unlock();
      if (cudaStreamWaitEvent(ln.s, ev_se.e[2], 0) != cudaSuccess) return fail(ED_ECUDA);
    }
    for (size_t bi : lane_blocks[k]) {
      const Block& b = c->blocks[bi];
      const int m = (int)bm(bi);
      double* hd = hde.p + hoff[bi];
      double* he = hd + std::max(m, 1);
      ed_status s = ED_OK;
      if (cudaEventRecord(ev_g0.e[bi], ln.s) != cudaSuccess) return fail(ED_ECUDA);
      if ((s = oz_slice(&oz, d_jobs + bi, 1, units[bi], b.dA > b.dB, nullptr, ln.s)) != ED_OK) return fail(s);
      if ((s = oz_gemm(&oz, d_probs + bi, 1, tiles[bi], nullptr, ln.s)) != ED_OK) return fail(s);
      if (cudaEventRecord(ev_g1.e[bi], ln.s) != cudaSuccess) return fail(ED_ECUDA);
      TriBlocked tb{&oz, ln.NVW, ln.WV, ln.WVf, ln.F, tridiag_ldF(m), {}, oz.d_err, d_tjobs + 2 * toff[bi],
                    d_tprobs + toff[bi]};
      if (m >= 3 && (s = tmap_8b_2d(&tb.tmF, ln.F, m, m, tb.ldF, 34, 32)) != ED_OK) return fail(s);
      if ((s = tridiag_reduce_blocked(ln.G, m, ln.work, hd, he, ln.s, sms, tb)) != ED_OK) return fail(s);
      if (cudaEventRecord(ev_done.e[bi], ln.s) != cudaSuccess) return fail(ED_ECUDA);
      if (k == 0 && bi == lane_blocks[0][0]) {
        if (cudaEventRecord(ev_se.e[2], ln.s) != cudaSuccess) return fail(ED_ECUDA);
        first_set(1);
      }
      cudaEvent_t done = ev_done.e[bi];
      auto ql = [&dd, &ee, &ok, hd, he, m, bi, done] {
        if (cudaEventSynchronize(done) != cudaSuccess) {
          ok[bi] = 2;
          return;
        }
        dd[bi].assign(hd, hd + m);
        ee[bi].assign(he, he + std::max(m - 1, 0));
        ok[bi] = tridiag_eigenvalues(dd[bi], ee[bi]) ? 1 : 0;
      };
      try {
        qr[k].emplace_back(ql);
      } catch (...) {
        ql();  // no thread to be had: wait for the block and reduce it here
      }
    }
    if (cudaEventRecord(ev_lane.e[k], ln.s) != cudaSuccess) return fail(ED_ECUDA);
  };
  for (int k = 0; k < lanes; ++k) {
    try {
      workers.emplace_back(lane_fn, k);
    } catch (...) {
      lane_fn(k);  // no thread to be had: enqueue this lane from here
    }
  }
  for (auto& x : workers) x.join();
  for (int k = 0; k < lanes; ++k)
    if (lst[k] != ED_OK) {
      for (int i = 0; i < lanes; ++i) cudaStreamSynchronize(L[i].s);  // nothing of this call left in flight
      set_error("%s", lmsg[k].c_str());
      return lst[k];
    }
  for (int k = 0; k < lanes; ++k) ED_CUDA_TRY(cudaStreamWaitEvent(st, ev_lane.e[k], 0));
  ED_CUDA_TRY(cudaEventRecord(ev_se.e[1], st));
  // ||Psi_s||^2 (the trace of rho_A(s)) with the library's FP64 reduction
  std::vector<double> wt(nb);
  for (size_t bi = 0; bi < nb; ++bi) {
    const Block& b = c->blocks[bi];
    ED_TRY(dot_dev<double>(c, psi + b.off, psi + b.off, b.dA * b.dB, slot(c, 3), st, 0));
    ED_TRY(read_scalars(c, 3, 1, &wt[bi], st));  // synchronises the stream
  }
  ED_TRY(oz_status(&oz, st));  // no bounded wait of the reduction's kernels ran out
  const auto tq = std::chrono::steady_clock::now();
  for (int k = 0; k < lanes; ++k)
    for (auto& x : qr[k]) x.join();
  const double t_qr = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tq).count();
  double t_gram = 0.0;
  float t_all = 0.f;
  for (size_t bi = 0; bi < nb; ++bi) {
    float t1 = 0.f;
    ED_CUDA_TRY(cudaEventElapsedTime(&t1, ev_g0.e[bi], ev_g1.e[bi]));
    t_gram += t1;
  }
  ED_CUDA_TRY(cudaEventElapsedTime(&t_all, ev_se.e[0], ev_se.e[1]));
  int64_t pos = 0;
  for (size_t bi = 0; bi < nb; ++bi) {
    if (ok[bi] != 1) {
      set_error(ok[bi] == 2 ? "waiting for block %zu's reduction failed" : "tridiagonal QL did not converge on block %zu",
                bi);
      return ED_ENOCONV;
    }
    std::vector<double>& w = dd[bi];
    std::sort(w.begin(), w.end(), [](double u, double v) { return u > v; });  // descending
    for (size_t i = 0; i < w.size(); ++i) lambda[pos + i] = w[i];
    pos += (int64_t)w.size();
  }
  if (stage_ms) {
    // with the blocks on several streams the Gram products overlap other
    // blocks' reductions: [0] = the Gram products' own device time, [1] =
    // the rest of the call's device time plus the host QL left at its end
    stage_ms[0] = t_gram;
    stage_ms[1] = std::max(0.0, (double)t_all - t_gram) + t_qr;
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
