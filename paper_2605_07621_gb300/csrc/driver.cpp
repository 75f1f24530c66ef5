// Lanczos ground-state and Green's-function drivers (host orchestration of
// the device kernels).  The paper uses H|psi> as the kernel of Krylov
// solvers (exact diagonalisation by Lanczos) and of dynamical correlations;
// it prints no solver, so these are the textbook three-term recurrence
// (Lanczos 1950), the lowest Ritz pair of the tridiagonal matrix, and the
// continued-fraction resolvent.  Every vector operation runs on the GPU; the
// host only keeps the alpha/beta scalars and solves the small tridiagonal
// eigenproblem.
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "krylov.h"

using namespace edk;

namespace {

template <typename T>
constexpr ed_dtype dtype_of();
template <>
constexpr ed_dtype dtype_of<double>() { return ED_F64; }
template <>
constexpr ed_dtype dtype_of<float>() { return ED_F32; }

// device buffers freed at scope exit
struct DevBuf {
  std::vector<void*> ptrs;
  ~DevBuf() {
    for (void* p : ptrs) cudaFree(p);
  }
  ed_status get(void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes < 16 ? 16 : bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMalloc(%zu) for Lanczos work failed: %s", bytes, cudaGetErrorString(e));
      return ED_ENOMEM;
    }
    ptrs.push_back(*p);
    return ED_OK;
  }
};

enum BasisKind { BASIS_NONE = 0, BASIS_SAME = 1, BASIS_BF16 = 2 };

// relative Ritz-residual target when an eigenvector is returned
constexpr double kVecResid = 1e-10;
// mixed precision: Ritz residual estimate (relative) at which the FP32 run
// hands over, and the FP64 refinement's convergence-check interval
constexpr double kLowResid = 3e-6;
constexpr int kRefineCheck = 3;
// Lanczos runs on sectors up to this size replay pairs of steps from a
// captured CUDA graph (their steps are bound by launch latency)
constexpr long long kGraphStates = 1ll << 22;
// Green's function runs re-orthogonalise only sectors up to this size
constexpr long long kGfReorthStates = 1ll << 22;

// Lanczos basis kept on the device as one contiguous array of `cap`
// vectors (same type as the recurrence, or BF16 when only a restart vector
// is needed).  When it does not fit the budget the vectors are recomputed
// in a second pass instead.
struct Basis {
  BasisKind kind = BASIS_NONE;
  size_t elem = 0;
  long long n = 0;
  int cap = 0, count = 0;
  bool complete = false;
  void* base = nullptr;
  ~Basis() {
    if (base) cudaFree(base);
  }
  bool init(BasisKind k, size_t e, long long len, int capacity, size_t budget) {
    kind = k;
    elem = e;
    n = len;
    cap = capacity;
    count = 0;
    complete = false;
    if (k == BASIS_NONE || capacity <= 0 || len <= 0) return false;
    // as many vectors as fit the budget; a longer run falls back to a second pass
    const size_t per = (size_t)len * e;
    if ((size_t)capacity * per > budget) capacity = (int)(budget / per);
    if (capacity < 2) return false;
    cap = capacity;
    size_t bytes = (size_t)capacity * per;
    if (cudaMalloc(&base, bytes) != cudaSuccess) {
      cudaGetLastError();
      base = nullptr;
      return false;
    }
    complete = true;
    return true;
  }
  void* at(int j) const { return (char*)base + (size_t)j * (size_t)n * elem; }
  void release() {
    if (base) cudaFree(base);
    base = nullptr;
    complete = false;
    count = 0;
  }
};

template <typename T>
void basis_store(ed_ctx* c, Basis* B, const T* v, long long n, cudaStream_t st) {
  if (!B || !B->complete) return;
  if (B->count >= B->cap) {
    B->complete = false;
    return;
  }
  void* p = B->at(B->count++);
  if (B->kind == BASIS_SAME)
    cudaMemcpyAsync(p, v, (size_t)n * sizeof(T), cudaMemcpyDeviceToDevice, st);
  else
    launch_cvt<float, __nv_bfloat16>(c, (const float*)v, (__nv_bfloat16*)p, n, st);
}

struct RunOut {
  std::vector<double> alpha, beta;  // beta[j] = beta_{j+1}
  bool converged = false;
  double theta = 0.0;
  int orthogonalised = 0;  // steps whose vector was orthogonalised against the basis
};

// Three-term Lanczos recurrence from the normalised v0 (device, type T).
// resid_tol > 0 additionally requires the Ritz residual estimate
// beta_m |s_m| <= resid_tol (used when an eigenvector is wanted).
//
// alpha_j, beta_{j+1} stay on the device (a history array) and are read
// back only every `check_every` steps (every kReadEvery in fixed-length
// runs), so the host does not synchronise with the GPU at every step.  A
// breakdown (beta ~ 0) is found at the next read; the steps run after it
// (on an invalid vector) are discarded, and the run ends at the breakdown.
constexpr int kReadEvery = 16;

// Partial reorthogonalisation (Simon 1984): the level of orthogonality
// omega_{j,k} = v_j . v_k is estimated by its own recurrence, obtained by
// projecting the three-term recurrence on v_k,
//   b_j w_{j+1,k} = b_k w_{j,k+1} + (a_k - a_j) w_{j,k} + b_{k-1} w_{j,k-1}
//                   - b_{j-1} w_{j-1,k}  (+ a rounding term of order eps |H|),
// with b_j = beta_{j+1}.  When some |w_{j+1,k}| exceeds sqrt(eps) the new
// vector, and the one after it, are orthogonalised against the whole basis
// (classical Gram-Schmidt twice) and their estimates reset to eps.  This
// keeps the basis semi-orthogonal, which leaves the tridiagonal matrix (and
// so the Ritz values and continued fractions) accurate to rounding, at a
// fraction of the cost of orthogonalising every step.
struct OmegaPRO {
  std::vector<double> a, b;       // alpha_k, beta_{k+1} of the steps so far
  std::vector<double> cur, prev;  // omega_{j,k}, omega_{j-1,k}
  bool force = false;             // orthogonalise the next vector as well
  int count = 0;                  // steps orthogonalised
  static constexpr double kEps = 2.220446049250313e-16;
  // step j gave alpha_j and b_j (before any correction); true when w
  // (the next vector) must be orthogonalised
  bool need(double aj, double bj, double anorm) {
    const int j = (int)a.size();
    a.push_back(aj);
    b.push_back(bj);
    std::vector<double> nw(j + 2, 0.0);
    if (j == 0) {
      cur.assign(1, 1.0);
    }
    double mx = 0.0;
    for (int k = 0; k < j && bj > 0.0; ++k) {
      double num = b[k] * cur[k + 1] + (a[k] - aj) * cur[k] - (j > 0 ? b[j - 1] * prev[k] : 0.0);
      if (k > 0) num += b[k - 1] * cur[k - 1];
      num += (num >= 0.0 ? 1.0 : -1.0) * 2.0 * kEps * anorm;
      nw[k] = num / bj;
      mx = std::max(mx, std::fabs(nw[k]));
    }
    nw[j] = bj > 0.0 ? kEps * anorm / bj : kEps;
    nw[j + 1] = 1.0;
    prev = cur;
    cur = nw;
    const bool r = force || mx > std::sqrt(kEps);
    force = r && !force;
    return r;
  }
  // the vector was orthogonalised: its estimates are back at rounding level
  void reset(double bj_new) {
    b.back() = bj_new;
    for (size_t k = 0; k + 1 < cur.size(); ++k) cur[k] = kEps;
    ++count;
  }
};

template <typename T>
ed_status lz_run(ed_ctx* c, cudaStream_t st, T* bufs[3], const T* v0, int max_iter, double tol, int check_every,
                 bool fixed, bool reorth, Basis* basis, RunOut& out, double resid_tol = 0.0, bool partial = false) {
  const long long n = c->D;
  T* vprev = bufs[0];
  T* v = bufs[1];
  T* w = bufs[2];
  DevBuf mem;
  double* hist = nullptr;  // [max_iter][2]: alpha_j, beta_{j+1}
  ED_TRY(mem.get((void**)&hist, (size_t)max_iter * 2 * sizeof(double)));
  std::vector<double> hbuf;
  ED_CUDA_TRY(cudaMemcpyAsync(v, v0, (size_t)n * sizeof(T), cudaMemcpyDeviceToDevice, st));
  basis_store<T>(c, basis, v, n, st);
  out.alpha.clear();
  out.beta.clear();
  out.converged = false;
  double theta_prev = NAN;
  double scale = 0.0;
  const int every = fixed ? kReadEvery : check_every;
  int read = 0;  // steps whose scalars the host holds
  bool done = false;
  // FP64 on the exact fixed-point path without reorthogonalisation: lz_c
  // writes the next step's fixed-point input and its scale, so the apply
  // skips its own exponent and conversion passes
  bool fuse = false, prepared = false;
  if constexpr (std::is_same<T, double>::value) fuse = !reorth && fixed_path(c, v);
  int* ew = c->d_exp + 1;
  const bool pro = partial && !reorth && basis && basis->kind == BASIS_SAME && basis->complete;
  OmegaPRO om;
  double anorm = 0.0;
  int* hcount = nullptr;  // device index of the next history entry
  ED_TRY(mem.get((void**)&hcount, sizeof(int)));
  ED_CUDA_TRY(cudaMemsetAsync(hcount, 0, sizeof(int), st));
  // one step up to its history entry (apply, alpha, beta, orthogonalisation)
  auto head = [&](int j, bool& ortho_now) -> ed_status {
    ortho_now = false;
    if constexpr (std::is_same<T, double>::value) {
      if (prepared)
        ED_TRY(apply_prepared_fixed(c, v, w, st));
      else
        ED_TRY(apply_H_impl(c, v, w, dtype_of<T>(), st));
    } else {
      ED_TRY(apply_H_impl(c, v, w, dtype_of<T>(), st));
    }
    launch_lz_a<T>(c, w, v, vprev, j > 0 ? 1 : 0, n, st);
    if constexpr (std::is_same<T, double>::value) {
      if (fuse)
        launch_lz_b_emax(c, w, v, n, ew, st);
      else
        launch_lz_b<T>(c, w, v, n, st);
    } else {
      launch_lz_b<T>(c, w, v, n, st);
    }
    if (reorth && basis && basis->kind == BASIS_SAME && basis->complete && basis->count <= kMaxBasis) {
      // classical Gram-Schmidt against all kept vectors, applied twice
      for (int pass = 0; pass < 2; ++pass)
        launch_reorth<T>(c, (const T*)basis->base, n, basis->count, w, n, hcoef(c), st);
      ED_TRY(dot_dev<T>(c, w, w, n, slot(c, 1), st, 1));
    }
    if (pro && basis->complete && basis->count <= kMaxBasis) {
      double ab[2];
      ED_TRY(read_scalars(c, 0, 2, ab, st));  // alpha_j, beta_{j+1} (synchronises)
      anorm = std::max(anorm, std::fabs(ab[0]) + ab[1]);
      if (om.need(ab[0], ab[1], anorm)) {
        for (int pass = 0; pass < 2; ++pass)
          launch_reorth<T>(c, (const T*)basis->base, n, basis->count, w, n, hcoef(c), st);
        ED_TRY(dot_dev<T>(c, w, w, n, slot(c, 1), st, 1));
        double bn;
        ED_TRY(read_scalars(c, 1, 1, &bn, st));
        om.reset(bn);
        ortho_now = true;
      }
    }
    launch_hist_push(c, hist, hcount, st);
    ED_CUDA_TRY(cudaGetLastError());
    return ED_OK;
  };
  // the rest of the step: the next Lanczos vector (and its fixed-point copy)
  auto tail = [&](bool ortho_now) {
    if constexpr (std::is_same<T, double>::value) {
      // (after an orthogonalisation the exponent lz_b recorded may be stale)
      if (fuse && c->d_fixed && !ortho_now) {
        launch_lz_c_fixed(c, w, vprev, c->d_fixed, ew, c->d_exp, n, st);
        prepared = true;
      } else {
        launch_lz_c<T>(c, w, vprev, n, st);
        prepared = false;
      }
    } else {
      launch_lz_c<T>(c, w, vprev, n, st);
    }
    std::swap(vprev, v);
    basis_store<T>(c, basis, v, n, st);
  };
  // read the scalars of the steps since the last read and examine them in order
  auto examine = [&](int m) -> ed_status {
    hbuf.resize((size_t)(m - read) * 2);
    ED_CUDA_TRY(cudaMemcpyAsync(hbuf.data(), hist + 2 * read, hbuf.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                st));
    ED_CUDA_TRY(cudaStreamSynchronize(st));
    for (int k = read; k < m && !done; ++k) {
      const double a = hbuf[2 * (k - read)], b = hbuf[2 * (k - read) + 1];
      out.alpha.push_back(a);
      out.beta.push_back(b);
      scale = std::max(scale, std::fabs(a) + b);
      const int mk = k + 1;
      const bool breakdown = !(b > 1e-13 * (scale > 0 ? scale : 1.0));
      if (!fixed && (mk % check_every == 0 || breakdown)) {
        double th = tridiag_lowest(out.alpha.data(), out.beta.data(), mk);
        bool ok = std::fabs(th - theta_prev) <= tol * std::fabs(th);
        if (ok && resid_tol > 0.0 && !breakdown) {
          std::vector<double> sv;
          tridiag_vector(out.alpha.data(), out.beta.data(), mk, th, sv);
          ok = std::fabs(b * sv[mk - 1]) <= resid_tol * std::max(1.0, std::fabs(th));
        }
        if (ok) {
          out.converged = true;
          done = true;
        }
        theta_prev = th;
      }
      if (breakdown) {
        out.converged = true;  // invariant subspace: T is exact
        done = true;
      }
    }
    read = m;
    return ED_OK;
  };
  // small sectors: pairs of steps (the v / vprev roles alternate, so a pair
  // returns them to where they started) captured once and replayed
  // (captured on the context's private stream and fenced with events
  // against the caller's stream, which may be the legacy default stream)
  bool graphs = n <= kGraphStates && !reorth && !pro && !(basis && basis->complete) && !c->prof && max_iter > 3;
  struct GraphState {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t fence[2] = {nullptr, nullptr};
    void release() {
      if (exec) cudaGraphExecDestroy(exec);
      if (graph) cudaGraphDestroy(graph);
      exec = nullptr;
      graph = nullptr;
    }
    ~GraphState() {
      release();
      for (auto& e : fence)
        if (e) cudaEventDestroy(e);
    }
  } gs;
  cudaGraph_t& graph = gs.graph;
  cudaGraphExec_t& gexec = gs.exec;
  cudaEvent_t* fence = gs.fence;
  if (graphs) {
    if (!c->lz_stream && cudaStreamCreateWithFlags(&c->lz_stream, cudaStreamNonBlocking) != cudaSuccess)
      c->lz_stream = nullptr;
    for (int q = 0; q < 2; ++q)
      if (cudaEventCreateWithFlags(&fence[q], cudaEventDisableTiming) != cudaSuccess) fence[q] = nullptr;
    graphs = c->lz_stream && fence[0] && fence[1];
    cudaGetLastError();
  }
  auto release = [&]() { gs.release(); };
  int j = 0;
  while (j < max_iter && !done) {
    if (graphs && j >= 1 && j + 2 < max_iter) {
      const cudaStream_t user = st, ps = c->lz_stream;
      if (!gexec) {
        st = ps;
        bool ok = cudaStreamBeginCapture(ps, cudaStreamCaptureModeRelaxed) == cudaSuccess;
        ed_status es = ED_OK;
        if (ok) {
          for (int q = 0; q < 2 && es == ED_OK; ++q) {
            bool on = false;
            es = head(j + q, on);
            if (es == ED_OK) tail(on);
          }
          ok = cudaStreamEndCapture(ps, &graph) == cudaSuccess && es == ED_OK &&
               cudaGraphInstantiate(&gexec, graph, 0) == cudaSuccess;
        }
        st = user;
        if (!ok) {
          // nothing captured has run: continue step by step
          cudaGetLastError();
          release();
          graphs = false;
          continue;
        }
      }
      ED_CUDA_TRY(cudaEventRecord(fence[0], st));
      ED_CUDA_TRY(cudaStreamWaitEvent(ps, fence[0], 0));
      const cudaError_t le = cudaGraphLaunch(gexec, ps);
      if (le != cudaSuccess) {
        release();
        ED_CUDA_TRY(le);
      }
      ED_CUDA_TRY(cudaEventRecord(fence[1], ps));
      ED_CUDA_TRY(cudaStreamWaitEvent(st, fence[1], 0));
      j += 2;
    } else {
      bool on = false;
      ED_TRY(head(j, on));
      ++j;
      if (j < max_iter) tail(on);
    }
    if (j - read >= every || j == max_iter) ED_TRY(examine(j));
  }
  // stop at the step the host examined last (later steps, if any, came
  // after a breakdown or convergence inside a read batch)
  const int steps = (int)out.alpha.size();
  out.theta = tridiag_lowest(out.alpha.data(), out.beta.data(), steps);
  out.orthogonalised = pro ? om.count : (reorth ? steps : 0);
  if (basis && basis->count > steps) basis->count = steps;
  bufs[0] = vprev;
  bufs[1] = v;
  return ED_OK;
}

// Ritz vector x = sum_j s_j v_j (FP64, normalised) from a stored basis or,
// when none was kept, from a second pass of the same recurrence.
template <typename T>
ed_status lz_vector(ed_ctx* c, cudaStream_t st, T* bufs[3], const T* v0, const RunOut& r, Basis* basis, double* x) {
  const long long n = c->D;
  const int m = (int)r.alpha.size();
  std::vector<double> s;
  tridiag_vector(r.alpha.data(), r.beta.data(), m, r.theta, s);
  const bool combine = std::is_same<T, float>::value && basis && basis->complete && basis->count >= m &&
                       basis->kind == BASIS_SAME && m <= kMaxBasis;
  if (!combine) ED_CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)n * sizeof(double), st));
  if (combine) {
    // one pass over the stored FP32 vectors, float-float sums
    ED_TRY(launch_combine_f32(c, (const float*)basis->base, n, s.data(), m, x, st));
  } else if (basis && basis->complete && basis->count >= m) {
    for (int j = 0; j < m; ++j) {
      if (basis->kind == BASIS_BF16)
        launch_axpy_basis<__nv_bfloat16, double>(c, (const __nv_bfloat16*)basis->at(j), x, s[j], n, st);
      else
        launch_axpy_basis<T, double>(c, (const T*)basis->at(j), x, s[j], n, st);
    }
  } else {
    T* vprev = bufs[0];
    T* v = bufs[1];
    T* w = bufs[2];
    ED_CUDA_TRY(cudaMemcpyAsync(v, v0, (size_t)n * sizeof(T), cudaMemcpyDeviceToDevice, st));
    launch_axpy_basis<T, double>(c, v, x, s[0], n, st);
    for (int j = 0; j + 1 < m; ++j) {
      ED_TRY(apply_H_impl(c, v, w, dtype_of<T>(), st));
      const double bj = j > 0 ? r.beta[j - 1] : 0.0;
      launch_lz_rerun<T>(c, w, v, j > 0 ? vprev : nullptr, r.alpha[j], bj, 1.0 / r.beta[j], vprev, n, st);
      std::swap(vprev, v);
      launch_axpy_basis<T, double>(c, v, x, s[j + 1], n, st);
    }
  }
  ED_TRY(dot_dev<double>(c, x, x, n, slot(c, 3), st, 1));
  double nrm;
  ED_TRY(read_scalars(c, 3, 1, &nrm, st));
  if (nrm > 0) launch_scale_cvt<double, double>(c, x, x, 1.0 / nrm, n, st);
  ED_CUDA_TRY(cudaGetLastError());
  return ED_OK;
}

// ||H x - theta x|| in FP64 (tmp: D doubles)
ed_status residual64(ed_ctx* c, cudaStream_t st, const double* x, double theta, double* tmp, double* res) {
  const long long n = c->D;
  ED_TRY(apply_H_impl(c, x, tmp, ED_F64, st));
  launch_axpy_basis<double, double>(c, x, tmp, -theta, n, st);
  ED_TRY(dot_dev<double>(c, tmp, tmp, n, slot(c, 3), st, 1));
  return read_scalars(c, 3, 1, res, st);
}

size_t free_device_bytes() {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return fr;
}

}  // namespace

extern "C" void ed_lanczos_default_opts(ed_lanczos_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->mode = ED_LZ_F64;
  o->max_iter = 400;
  o->tol = 1e-12;
  o->check_every = 5;
  o->fixed_iter = 0;
  o->reorth = 0;
  o->seed = 20260507ULL;
  o->v0 = nullptr;
  o->refine_block = 30;
  o->stream = nullptr;
}

extern "C" ed_status ed_lanczos_ground(ed_ctx* c, const ed_lanczos_opts* opts_in, double* e0, void* psi0,
                                       ed_report* rep) {
  auto t0 = std::chrono::steady_clock::now();
  if (!c || !e0) { set_error("ctx or e0 is NULL"); return ED_EINVAL; }
  if (!c->ops_built) { set_error("ed_build_local_ops has not been called"); return ED_EINVAL; }
  ed_lanczos_opts o;
  ed_lanczos_default_opts(&o);
  if (opts_in) o = *opts_in;
  if (o.mode < ED_LZ_F64 || o.mode > ED_LZ_MIXED || o.max_iter < 1 || o.check_every < 1 || !(o.tol >= 0.0)) {
    set_error("bad Lanczos options");
    return ED_EINVAL;
  }
  if (c->D < 1) { set_error("empty sector"); return ED_EINVAL; }
  ED_DEVICE_SCOPE(c->device);
  ED_TRY(ensure_scratch(c));
  cudaStream_t st = (cudaStream_t)o.stream;
  const long long n = c->D;
  const int max_iter = (int)std::min<long long>(o.max_iter, o.fixed_iter ? o.max_iter : n + 1);
  DevBuf mem;
  double *v0 = nullptr, *x = nullptr, *tmp = nullptr;
  ED_TRY(mem.get((void**)&v0, n * sizeof(double)));
  if (o.v0) {
    ED_CUDA_TRY(cudaMemcpyAsync(v0, o.v0, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  } else {
    ED_TRY(random_vector_impl(c, o.seed, v0, ED_F64, st));
  }
  ED_TRY(dot_dev<double>(c, v0, v0, n, slot(c, 3), st, 1));
  double nrm;
  ED_TRY(read_scalars(c, 3, 1, &nrm, st));
  if (!(nrm > 0)) { set_error("start vector is zero"); return ED_EINVAL; }
  launch_scale_cvt<double, double>(c, v0, v0, 1.0 / nrm, n, st);

  ed_report R;
  std::memset(&R, 0, sizeof(R));
  if (rep) {
    R.alpha = rep->alpha;
    R.beta = rep->beta;
    R.ab_capacity = rep->ab_capacity;
  }
  auto record_ab = [&](const RunOut& r) {
    if (!R.alpha || R.ab_capacity <= 0) return;
    int k = std::min<int>((int)r.alpha.size(), R.ab_capacity);
    for (int i = 0; i < k; ++i) {
      R.alpha[i] = r.alpha[i];
      if (R.beta) R.beta[i] = r.beta[i];
    }
    R.n_ab = k;
  };
  const size_t budget = free_device_bytes() / 2;
  const bool want_vec = psi0 != nullptr;
  double energy = 0.0;
  bool converged = false;

  if (o.mode == ED_LZ_F64) {
    double* bufs[3];
    for (auto& b : bufs) ED_TRY(mem.get((void**)&b, n * sizeof(double)));
    Basis B;
    if (o.reorth || want_vec) B.init(BASIS_SAME, sizeof(double), n, max_iter + 1, budget);
    RunOut r;
    ED_TRY(lz_run<double>(c, st, bufs, v0, max_iter, o.tol, o.check_every, o.fixed_iter != 0, o.reorth != 0, &B, r,
                          want_vec ? kVecResid : 0.0));
    record_ab(r);
    R.iterations = (int)r.alpha.size();
    energy = r.theta;
    converged = r.converged || o.fixed_iter;
    if (want_vec) {
      ED_TRY(mem.get((void**)&tmp, n * sizeof(double)));
      ED_TRY(lz_vector<double>(c, st, bufs, v0, r, &B, (double*)psi0));
      ED_TRY(residual64(c, st, (const double*)psi0, energy, tmp, &R.residual));
    }
  } else {
    // FP32-storage Lanczos (FP64 reductions)
    float* bufs32[3];
    for (auto& b : bufs32) ED_TRY(mem.get((void**)&b, n * sizeof(float)));
    float* v0f;
    ED_TRY(mem.get((void**)&v0f, n * sizeof(float)));
    launch_cvt<double, float>(c, v0, v0f, n, st);
    const bool mixed = o.mode == ED_LZ_MIXED;
    Basis B;
    if (mixed || want_vec || o.reorth) {
      // keep the basis in FP32 when it fits, else in BF16 (a restart vector
      // needs only a few digits), else recompute it in a second pass.  The
      // basis may take all free memory but what the steps after this run
      // allocate (the FP64 vectors of the refinement, or the result and a
      // residual vector); it is released before the refinement starts
      const size_t later = (size_t)n * sizeof(double) * (mixed ? 6 : 2) + ((size_t)1 << 30);
      const size_t fr = free_device_bytes();
      const size_t budget32 = fr > later ? fr - later : 0;
      if (!B.init(BASIS_SAME, sizeof(float), n, max_iter + 1, budget32) && !o.reorth)
        B.init(BASIS_BF16, 2, n, max_iter + 1, budget32);
    }
    // mixed: the FP32 run goes on until its Ritz vector is close to the
    // FP32 floor (residual estimate), so that the FP64 refinement starts
    // from a vector that needs only a few steps
    const double tol_low = mixed ? std::max(o.tol, 2e-7) : o.tol;
    RunOut r;
    ED_TRY(lz_run<float>(c, st, bufs32, v0f, max_iter, tol_low, o.check_every, o.fixed_iter != 0, o.reorth != 0, &B,
                         r, mixed ? kLowResid : 0.0));
    record_ab(r);
    R.iterations = R.iterations_low = (int)r.alpha.size();
    R.e_low = r.theta;
    energy = r.theta;
    converged = r.converged || o.fixed_iter;
    if (mixed || want_vec) {
      ED_TRY(mem.get((void**)&x, n * sizeof(double)));
      ED_TRY(lz_vector<float>(c, st, bufs32, v0f, r, &B, x));
      B.release();
    }
    if (mixed) {
      // FP64 refinement: Lanczos restarted from the FP32 Ritz vector until
      // the energy is stable to tol (relative)
      double* bufs[3];
      for (auto& b : bufs) ED_TRY(mem.get((void**)&b, n * sizeof(double)));
      double* xnew;
      ED_TRY(mem.get((void**)&xnew, n * sizeof(double)));
      double e_prev = r.theta;
      converged = false;
      const int ce = std::min(o.check_every, kRefineCheck);
      const int blk = std::max(o.refine_block, 2 * ce);
      for (int rs = 0; rs < 20; ++rs) {
        Basis B64;
        if (want_vec) B64.init(BASIS_SAME, sizeof(double), n, blk + 1, free_device_bytes() / 2);
        RunOut r2;
        ED_TRY(lz_run<double>(c, st, bufs, x, blk, o.tol, ce, false, false, &B64, r2, want_vec ? kVecResid : 0.0));
        R.iterations += (int)r2.alpha.size();
        R.restarts += 1;
        energy = r2.theta;
        const bool done = r2.converged || std::fabs(energy - e_prev) <= o.tol * std::fabs(energy);
        if (!done || want_vec) {
          ED_TRY(lz_vector<double>(c, st, bufs, x, r2, &B64, xnew));
          std::swap(x, xnew);
        }
        e_prev = energy;
        if (done) {
          converged = true;
          break;
        }
      }
      if (want_vec) {
        ED_CUDA_TRY(cudaMemcpyAsync(psi0, x, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        ED_TRY(mem.get((void**)&tmp, n * sizeof(double)));
        ED_TRY(residual64(c, st, (const double*)psi0, energy, tmp, &R.residual));
      }
    } else if (want_vec) {
      ED_CUDA_TRY(cudaMemcpyAsync(psi0, x, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      ED_TRY(mem.get((void**)&tmp, n * sizeof(double)));
      ED_TRY(residual64(c, st, (const double*)psi0, energy, tmp, &R.residual));
    }
  }
  ED_CUDA_TRY(cudaStreamSynchronize(st));
  R.converged = converged ? 1 : 0;
  R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  *e0 = energy;
  if (rep) *rep = R;
  if (!converged) {
    set_error("Lanczos did not meet tol=%g within %d steps", o.tol, R.iterations);
    return ED_ENOCONV;
  }
  return ED_OK;
}

namespace {

struct CtxGuard {
  ed_ctx* c = nullptr;
  ~CtxGuard() {
    if (c) ed_destroy(c);
  }
};

// phi = c^dag_{site,spin} psi0 (create) or c_{site,spin} psi0 in the shifted
// sector context c2.  The spin cut puts up electrons on side A (rows) and
// down electrons on side B (columns); with all up operators ordered before
// all down operators the sign is (-1)^(electrons of the same spin below the
// site) times (-1)^N_up for a down operator.
ed_status fermion_apply(ed_ctx* c, ed_ctx* c2, const double* psi0, int site, int spin, bool create, double* phi,
                        cudaStream_t st) {
  const Side& src = spin == 0 ? c->A : c->B;
  const Side& dst = spin == 0 ? c2->A : c2->B;
  const int ksrc = spin == 0 ? c->n_up : c->n_dw;
  const int kdst = spin == 0 ? c2->n_up : c2->n_dw;
  std::vector<int> map(dst.dim(kdst), -1);
  std::vector<signed char> sg(dst.dim(kdst), 0);
  const uint32_t bit = 1u << site;
  const uint32_t below = bit - 1u;
  for (int64_t r = 0; r < dst.dim(kdst); ++r) {
    uint32_t xd = dst.states[dst.start[kdst] + r];
    bool occ = (xd & bit) != 0;
    if (occ != create) continue;
    uint32_t xs = xd ^ bit;
    int64_t rs = combinadic_rank(xs);
    if (rs < 0 || rs >= src.dim(ksrc) || src.states[src.start[ksrc] + rs] != xs) {
      set_error("internal: fermion remap left the sector");
      return ED_EINVAL;
    }
    int par = __builtin_popcount(xs & below) + (spin == 1 ? c->n_up : 0);
    map[r] = (int)rs;
    sg[r] = (par & 1) ? -1 : 1;
  }
  DevBuf mem;
  int* dmap;
  signed char* dsg;
  ED_TRY(mem.get((void**)&dmap, map.size() * sizeof(int)));
  ED_TRY(mem.get((void**)&dsg, sg.size()));
  ED_CUDA_TRY(cudaMemcpyAsync(dmap, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  ED_CUDA_TRY(cudaMemcpyAsync(dsg, sg.data(), sg.size(), cudaMemcpyHostToDevice, st));
  const Block& b1 = c->blocks[0];
  const Block& b2 = c2->blocks[0];
  launch_fermion_remap(c2, psi0, b1.dA, b1.dB, phi, b2.dA, b2.dB, dmap, dsg, spin, st);
  ED_CUDA_TRY(cudaGetLastError());
  ED_CUDA_TRY(cudaStreamSynchronize(st));
  return ED_OK;
}

}  // namespace

extern "C" ed_status ed_lanczos_gf(ed_ctx* c, const void* psi0, double e0, int site, int spin, int n_iter,
                                   const double* omega, int n_omega, double eta, double* G, double* a_p, double* b_p,
                                   double* a_h, double* b_h, double* w_p, double* w_h, int reorth, void* stream) {
  if (!c || !psi0 || (n_omega > 0 && (!omega || !G))) { set_error("NULL argument"); return ED_EINVAL; }
  if (reorth < ED_GF_REORTH_AUTO || reorth > ED_GF_REORTH_PARTIAL) { set_error("bad reorth mode %d", reorth); return ED_EINVAL; }
  if (c->kind != ED_HUBBARD) { set_error("the Green's function needs a Hubbard context"); return ED_EINVAL; }
  if (!c->ops_built) { set_error("ed_build_local_ops has not been called"); return ED_EINVAL; }
  if (site < 0 || site >= c->n_sites || (spin != 0 && spin != 1) || n_iter < 1 || n_omega < 0 || !(eta >= 0.0)) {
    set_error("bad Green's function arguments");
    return ED_EINVAL;
  }
  ED_DEVICE_SCOPE(c->device);
  ED_TRY(ensure_scratch(c));
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf mem;
  std::vector<double> hp_a, hp_b, hh_a, hh_b;
  double wp = 0.0, wh = 0.0;
  for (int part = 0; part < 2; ++part) {
    const bool create = part == 0;
    const int d = create ? 1 : -1;
    const int nu = c->n_up + (spin == 0 ? d : 0);
    const int nd = c->n_dw + (spin == 1 ? d : 0);
    if (nu < 0 || nd < 0 || nu > c->n_sites || nd > c->n_sites) continue;
    ed_model_desc m{};
    m.kind = ED_HUBBARD;
    m.n_sites = c->n_sites;
    m.n_bonds = (int)c->bi.size();
    m.bi = c->bi.data();
    m.bj = c->bj.data();
    m.t = c->t.data();
    m.U = c->U.data();
    m.eps = c->eps.data();
    m.n_up = nu;
    m.n_dw = nd;
    m.spin_cut = 1;
    CtxGuard g;
    ED_TRY(ed_build_sectors(&m, &g.c));
    ED_TRY(ed_build_local_ops(g.c, c->ops_flags));
    ed_ctx* c2 = g.c;
    ED_TRY(ensure_scratch(c2));
    const long long n2 = c2->D;
    double* bufs[4];
    for (auto& b : bufs) ED_TRY(mem.get((void**)&b, n2 * sizeof(double)));
    double* phi = bufs[3];
    ED_TRY(fermion_apply(c, c2, (const double*)psi0, site, spin, create, phi, st));
    ED_TRY(dot_dev<double>(c2, phi, phi, n2, slot(c2, 3), st, 0));
    double w0;
    ED_TRY(read_scalars(c2, 3, 1, &w0, st));
    if (!(w0 > 0.0)) continue;
    launch_scale_cvt<double, double>(c2, phi, phi, 1.0 / std::sqrt(w0), n2, st);
    // re-orthogonalisation against the kept Krylov basis: full (every step)
    // for sectors of at most kGfReorthStates states, partial (when the
    // estimated loss of orthogonality reaches sqrt(eps)) above; both need
    // the whole basis in half of the free device memory, otherwise the plain
    // three-term recurrence runs.  Full classical Gram-Schmidt twice costs
    // about 4 j n FP64 FMAs at step j on the slow FP64 pipe and reads the
    // basis four times, so above a few million states it outweighs H|psi>
    // many times (41 M states, 300 steps: 24 s against 2.5 s)
    const int steps = (int)std::min<long long>(n_iter, n2);
    Basis B;
    // (a partial basis would only re-orthogonalise the first steps, at O(j n)
    // cost each, so it is used only when every step's vector fits)
    const bool want = reorth != ED_GF_REORTH_NONE;
    const bool fits = want && steps <= kMaxBasis &&
                      (size_t)(steps + 1) * (size_t)n2 * sizeof(double) <= free_device_bytes() / 2 &&
                      B.init(BASIS_SAME, sizeof(double), n2, steps + 1, free_device_bytes() / 2) &&
                      B.cap >= steps + 1;
    if (!fits && (reorth == ED_GF_REORTH_FULL || reorth == ED_GF_REORTH_PARTIAL)) {
      set_error("the Krylov basis (%d x %lld states) does not fit in half of the free device memory", steps + 1,
                (long long)n2);
      return ED_ENOMEM;
    }
    const bool full = fits && (reorth == ED_GF_REORTH_FULL || (reorth == ED_GF_REORTH_AUTO && n2 <= kGfReorthStates));
    const bool partial = fits && !full;
    RunOut r;
    ED_TRY(lz_run<double>(c2, st, bufs, phi, steps, 0.0, 1, true, full, fits ? &B : nullptr, r, 0.0, partial));
    ED_CUDA_TRY(cudaStreamSynchronize(st));
    if (create) { hp_a = r.alpha; hp_b = r.beta; wp = w0; }
    else { hh_a = r.alpha; hh_b = r.beta; wh = w0; }
  }
  auto out_coef = [&](const std::vector<double>& src, double* dst) {
    if (!dst) return;
    for (int i = 0; i < n_iter; ++i) dst[i] = i < (int)src.size() ? src[i] : 0.0;
  };
  out_coef(hp_a, a_p);
  out_coef(hp_b, b_p);
  out_coef(hh_a, a_h);
  out_coef(hh_b, b_h);
  if (w_p) *w_p = wp;
  if (w_h) *w_h = wh;
  if (n_omega == 0) return ED_OK;
  // continued fractions on the device, one thread per frequency
  double *d_om, *d_G, *d_ap, *d_bp, *d_ah, *d_bh;
  const int mp = (int)hp_a.size(), mh = (int)hh_a.size();
  ED_TRY(mem.get((void**)&d_om, n_omega * sizeof(double)));
  ED_TRY(mem.get((void**)&d_G, 2 * (size_t)n_omega * sizeof(double)));
  ED_TRY(mem.get((void**)&d_ap, (mp + 1) * sizeof(double)));
  ED_TRY(mem.get((void**)&d_bp, (mp + 1) * sizeof(double)));
  ED_TRY(mem.get((void**)&d_ah, (mh + 1) * sizeof(double)));
  ED_TRY(mem.get((void**)&d_bh, (mh + 1) * sizeof(double)));
  ED_CUDA_TRY(cudaMemcpyAsync(d_om, omega, n_omega * sizeof(double), cudaMemcpyHostToDevice, st));
  if (mp) {
    ED_CUDA_TRY(cudaMemcpyAsync(d_ap, hp_a.data(), mp * sizeof(double), cudaMemcpyHostToDevice, st));
    ED_CUDA_TRY(cudaMemcpyAsync(d_bp, hp_b.data(), mp * sizeof(double), cudaMemcpyHostToDevice, st));
  }
  if (mh) {
    ED_CUDA_TRY(cudaMemcpyAsync(d_ah, hh_a.data(), mh * sizeof(double), cudaMemcpyHostToDevice, st));
    ED_CUDA_TRY(cudaMemcpyAsync(d_bh, hh_b.data(), mh * sizeof(double), cudaMemcpyHostToDevice, st));
  }
  launch_green_cf(d_om, n_omega, eta, e0, d_ap, d_bp, mp, wp, d_ah, d_bh, mh, wh, d_G, st);
  ED_CUDA_TRY(cudaGetLastError());
  ED_CUDA_TRY(cudaMemcpyAsync(G, d_G, 2 * (size_t)n_omega * sizeof(double), cudaMemcpyDeviceToHost, st));
  ED_CUDA_TRY(cudaStreamSynchronize(st));
  return ED_OK;
}
