/*
 * ed.h -- C ABI of the GB300 bipartite H|psi> / Lanczos engine.
 *
 * The wavefunction of one symmetry sector of a K-local lattice model
 * (paper Eq. (1)) is stored in the entanglement-cut representation of
 * Eq. (3): a set of symmetry-resolved blocks Psi_s, one per value s of the
 * conserved charge on side A of the cut, each a d_A(s) x d_B(s) matrix.  The
 * Hamiltonian has the block form of Eq. (2):
 *     (H psi)_s = H_A,s Psi_s + Psi_s H_B,s^T + V_s o Psi_s
 *                 + sum_k c_k P^A_k Psi_s' (P^B_k)^T
 * (side Hamiltonians, a diagonal, and the cross-cut terms evaluated through
 * the paper's Vec/Kronecker identity [L (x) R] Vec(Psi) = Vec(R Psi L^T)).
 *
 * Vector layout (every x, y, psi pointer below): blocks concatenated in
 * ascending s; block s is row-major d_A(s) x d_B(s) (B index contiguous),
 * starting at element offset off[s] (ed_blocks).  Rows are the side-A
 * states of charge s in ascending order of their side-local bit strings
 * (combinadic / colex rank), columns the side-B states likewise.  Which
 * lattice site each side-local bit stands for is reported by ed_side_sites:
 * for spin models side A lists its sites on a cross-cut bond first, side B
 * lists them last, each group in ascending site order; for the Hubbard spin
 * cut bit p is site p on both sides (side A = spin-up occupations, side B =
 * spin-down occupations).
 *
 * Ownership: the caller owns every vector it passes (device pointers unless
 * stated); the context owns all operator tables, maps and work buffers.
 * Errors: every call returns an ed_status and never aborts; ed_last_error()
 * gives a message for the calling thread.  Streams: the caller's stream is
 * used; no call synchronises the device except where it returns host
 * scalars (noted per call).  Devices: a context lives on the device that
 * was current when it was built; every call runs there and puts the calling
 * thread's current device back before it returns.
 */
#ifndef ED_H
#define ED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ed_ctx ed_ctx;

typedef enum {
  ED_OK = 0,
  ED_EINVAL = 1,       /* malformed model, bad argument or size */
  ED_ENOMEM = 2,       /* device or host allocation failed */
  ED_ECUDA = 3,        /* a CUDA runtime call failed */
  ED_ENOCONV = 4,      /* Lanczos stopped at max_iter without meeting tol */
  ED_ETIMEOUT = 5,     /* a bounded wait ran out */
  ED_EUNSUPPORTED = 6, /* valid request outside what the library supports */
  ED_ECANCELLED = 7    /* a served request was cancelled */
} ed_status;

typedef enum { ED_F64 = 0, ED_F32 = 1 } ed_dtype;

typedef enum { ED_SPIN = 0, ED_HUBBARD = 1 } ed_kind;

/* One lattice model, its target sector and its entanglement cut.
 * Spin (ED_SPIN): H = sum_b [ jz_b S^z_i S^z_j + jxy_b/2 (S^+_i S^-_j + h.c.) ],
 *   n_up = number of up spins; cut_mask = bit mask of side-A sites.
 * Hubbard (ED_HUBBARD): H = -sum_{b,sigma} t_b (c^dag_i c_j + h.c.)
 *   + sum_i U_i n_i,up n_i,dw + sum_i eps_i n_i; sector (n_up, n_dw); the cut
 *   separates spin up (side A) from spin down (side B), spin_cut must be 1.
 *   Fermion order: all up sites ascending, then all down sites ascending.
 * All arrays are host memory, read during ed_build_sectors only. */
typedef struct {
  int kind;
  int n_sites;             /* 1 .. 64 (spin), 1 .. 32 (Hubbard) */
  int n_bonds;
  const int* bi;           /* bond endpoints, length n_bonds */
  const int* bj;
  const double* jxy;       /* spin, per bond (NULL = 0) */
  const double* jz;        /* spin, per bond (NULL = 0) */
  const double* t;         /* Hubbard, per bond (NULL = 0) */
  const double* U;         /* Hubbard, per site (NULL = 0) */
  const double* eps;       /* Hubbard, per site (NULL = 0) */
  int n_up;
  int n_dw;
  uint64_t cut_mask;       /* spin: side-A sites; each side at most 30 sites */
  int spin_cut;            /* Hubbard: 1 */
} ed_model_desc;

/* Build the sector/block structure (paper Eqs. (2)-(3): charges q_l + q_r
 * = q, block dimensions and offsets, combinadic ranks).  Selects the
 * current CUDA device for the context.  *out is set on success. */
ed_status ed_build_sectors(const ed_model_desc* model, ed_ctx** out);

/* Build the side operators of Eq. (2) on the device: CSR of H_A,s and
 * H_B,s off-diagonals, side diagonals, the cross-cut maps.
 * flags: ED_OPS_DEFAULT, or ED_OPS_FORCE_CSR / ED_OPS_FORCE_DENSE to pin the
 * per-sector choice instead of autotuning it.  Synchronises the device. */
#define ED_OPS_DEFAULT 0
#define ED_OPS_FORCE_CSR 1
#define ED_OPS_FORCE_DENSE 2
ed_status ed_build_local_ops(ed_ctx* ctx, int flags);

/* y = H x over the whole sector (all blocks), device pointers of ed_dim
 * elements of `dtype`, x and y must not overlap.  ED_F64: FP64 storage,
 * FP64-accurate result; ED_F32: FP32 storage and accumulation.  Enqueued on
 * `stream` (cudaStream_t, NULL = legacy default stream); no sync.  The
 * context's scratch (fixed-point copy of x, work counter) serves one call at
 * a time: calls on one context must not overlap on the GPU. */
ed_status ed_apply_H(ed_ctx* ctx, const void* x, void* y, ed_dtype dtype, void* stream);

/* y = H x like ed_apply_H with ED_F64, for callers that cannot allocate
 * device memory (for example code that runs inside another framework's
 * memory pool, under a capture that forbids allocation, or with the whole
 * device already handed out): this call never calls cudaMalloc, cudaFree or
 * any allocating library routine.  The paper has no counterpart; it exists
 * for such callers.  The exact fixed-point path needs a scratch copy of x
 * (8 bytes per state); here that scratch is a fixed device array compiled
 * into the library (32 MiB, held by every GPU that loads the library until
 * the process exits), so a context whose dimension (ed_dim: all blocks
 * together) exceeds 4,194,272 states is rejected with ED_EINVAL.  Models
 * whose couplings are not dyadic use the FP64 kernels, which need no
 * scratch.  The first call on a device looks up the array's device address
 * and keeps it for the life of the process; make that first call before
 * any stream capture, and do not reset the device (cudaDeviceReset) between
 * calls: the kept address would then be stale.  All calls share the array
 * and it keeps the last call's contents: two calls that overlap on the GPU
 * (different streams, or different contexts) race and give wrong results.
 * x, y: device FP64, not overlapping, x 16-byte aligned; enqueued on
 * `stream`. */
ed_status ed_apply_H_noalloc(ed_ctx* ctx, const void* x, void* y, void* stream);

/* Lanczos options / report (paper: H|psi> as the kernel of a Krylov
 * solver).  mode: ED_LZ_F64 plain FP64; ED_LZ_F32 FP32 storage with FP64
 * reductions; ED_LZ_MIXED FP32 Lanczos then FP64 restarted refinement until
 * the energy is stable to tol. */
typedef enum { ED_LZ_F64 = 0, ED_LZ_F32 = 1, ED_LZ_MIXED = 2 } ed_lz_mode;

typedef struct {
  int mode;              /* ed_lz_mode */
  int max_iter;          /* Lanczos steps cap (per phase); default 400 */
  double tol;            /* relative change of the lowest Ritz value; default 1e-12 */
  int check_every;       /* convergence test period in steps; default 5 */
  int fixed_iter;        /* 1: run exactly max_iter steps, no convergence stop */
  int reorth;            /* 1: full reorthogonalisation when the basis fits */
  uint64_t seed;         /* start vector = key-indexed SplitMix64 values */
  const double* v0;      /* optional FP64 device start vector (overrides seed) */
  int refine_block;      /* mixed mode: steps per FP64 restart; default 30 */
  void* stream;          /* cudaStream_t */
} ed_lanczos_opts;

typedef struct {
  int iterations;        /* total Lanczos steps (all phases) */
  int iterations_low;    /* steps taken in FP32 storage (mixed / f32) */
  int restarts;          /* FP64 restarts (mixed) */
  int converged;         /* 1 if tol was met */
  double e_low;          /* energy after the FP32 phase (mixed) */
  double residual;       /* ||H psi - E psi|| in FP64 (when a vector was formed) */
  double seconds;        /* wall time of the call */
  double* alpha;         /* optional host buffers (capacity ab_capacity) for */
  double* beta;          /*   the first-phase coefficients alpha_j, beta_{j+1} */
  int ab_capacity;
  int n_ab;              /* number of alpha written */
} ed_report;

void ed_lanczos_default_opts(ed_lanczos_opts* o);

/* Lowest eigenvalue E0 of the sector (and optionally its FP64 eigenvector
 * into psi0, device, ed_dim doubles).  Convergence: the lowest Ritz value
 * changes by at most tol (relative) over check_every steps; when psi0 is
 * requested the Ritz residual estimate beta_m |s_m| must also be at most
 * 1e-10 max(1, |E0|).  Synchronises the stream.  Returns ED_ENOCONV (with
 * *e0 and the report filled) when this was not met within max_iter. */
ed_status ed_lanczos_ground(ed_ctx* ctx, const ed_lanczos_opts* opts, double* e0, void* psi0, ed_report* rep);

/* Zero-temperature Green's function of a Hubbard context:
 *   G(w) = <psi0| c (z - (H - E0))^-1 c^dag |psi0> + <psi0| c^dag (z + (H - E0))^-1 c |psi0>,
 * z = w + i eta, c = c_{site,spin} (spin 0 = up), from n_iter-step FP64
 * Lanczos continued fractions started from c^dag psi0 and c psi0 (built on
 * the device in the shifted sectors).  reorth selects how the Krylov
 * vectors are kept orthogonal (ED_GF_REORTH_*): FULL orthogonalises every
 * step against the whole basis (classical Gram-Schmidt twice); PARTIAL only
 * the steps at which the estimated loss of orthogonality (Simon's
 * recurrence) reaches sqrt(eps), and the step after; both need all n_iter+1
 * basis vectors in half of the free device memory (ED_ENOMEM otherwise).
 * AUTO: FULL for shifted sectors of at most 2^22 states, PARTIAL above, and
 * the plain three-term recurrence when the basis does not fit (above that
 * size full orthogonalisation costs many times the H|psi> of a step).  psi0: device FP64 ground state of
 * ctx; omega: host, n_omega; G: host, 2*n_omega doubles (re, im pairs).
 * a_p, b_p, a_h, b_h: optional host outputs (n_iter each) of the particle
 * and hole coefficients; w_p, w_h: optional norms ||c^dag psi0||^2,
 * ||c psi0||^2.  Synchronises the stream. */
enum {
  ED_GF_REORTH_AUTO = -1,   /* full up to 2^22 states, partial above (when the basis fits) */
  ED_GF_REORTH_NONE = 0,    /* plain three-term recurrence */
  ED_GF_REORTH_FULL = 1,    /* every step against the whole basis */
  ED_GF_REORTH_PARTIAL = 2  /* when the estimated loss of orthogonality reaches sqrt(eps) */
};
ed_status ed_lanczos_gf(ed_ctx* ctx, const void* psi0, double e0, int site, int spin, int n_iter,
                        const double* omega, int n_omega, double eta, double* G, double* a_p, double* b_p,
                        double* a_h, double* b_h, double* w_p, double* w_h, int reorth, void* stream);

/* Entanglement spectrum of a state across the cut (the paper's discussion
 * of its figure "Distributed entanglement spectrum"): the eigenvalues lambda of the
 * reduced density matrix rho_A = Tr_B |psi><psi|, whose logarithms give the
 * spectrum xi = -log(lambda) of the entanglement Hamiltonian, resolved by the
 * charge s of side A, with the sector weights W_s = sum_i lambda_{s,i} /
 * sum_{s,i} lambda_{s,i}.  rho_A is block diagonal, rho_A(s) = Psi_s Psi_s^T;
 * its nonzero eigenvalues are those of the Gram matrix of Psi_s in the
 * smaller of d_A(s), d_B(s), formed on the device by this library; its
 * eigenvalues come from a blocked Householder reduction to tridiagonal form
 * on the device (float-float panel arithmetic, FP64-accurate tensor-core
 * trailing updates) and implicit QL steps on the host (one host thread per
 * block as soon as its tridiagonal matrix is ready; ED_ENOCONV if a QL
 * iteration does not converge).  The largest block is reduced first and
 * alone, the others concurrently on up to three internal streams that start
 * after the caller's prior work on `stream`.
 *   psi      device FP64 vector of ctx (not normalised by the call)
 *   lambda   host, capacity cap: for every block in ed_blocks order, its
 *            min(d_A, d_B) eigenvalues in descending order (rounding can
 *            leave eigenvalues of a rank-deficient block slightly negative)
 *   n_lambda receives sum_s min(d_A(s), d_B(s)); with lambda NULL the call
 *            only returns this count; cap smaller than it is ED_EINVAL
 *   weight   host, one per block (nullable): ||Psi_s||^2 = trace rho_A(s),
 *            summed on the device in FP64
 *   entropy  host (nullable): -sum p ln p over p = lambda / sum(weight) > 0
 *   stage_ms host (nullable), 2 doubles: the Gram kernels' own device time
 *            (summed over blocks; they overlap other blocks' reductions),
 *            and the rest of the call's device time plus the host QL time
 *            left after the device work (milliseconds)
 * The Gram matrices are formed on the tensor cores in FP64-accurate
 * digit-split form (8 BF16 digit planes per value, exact FP32 sums per digit
 * order, FP64 combination).  Device memory, per stream sized for its largest
 * block m = min(dA,dB) with the larger dimension L: the Gram matrix
 * (8 m^2 bytes; only its lower triangle is formed and reduced), its
 * float-float copy (8 m^2 bytes), the digit planes of Psi_s (16 m L bytes)
 * and the panel and work arrays (about 7 KB x m plus m^2 / 4 bytes); fewer
 * streams are used when device memory is short.  Blocks with
 * min(dA,dB) > 46340 are ED_EUNSUPPORTED.  Synchronises the stream. */
ed_status ed_entanglement_spectrum(ed_ctx* ctx, const double* psi, double* lambda, int64_t cap, int64_t* n_lambda,
                                   double* weight, double* entropy, double* stage_ms, void* stream);

/* The last stage of ed_entanglement_spectrum on its own: all eigenvalues of
 * the n x n symmetric tridiagonal matrix with diagonal d[0..n-1] and
 * off-diagonal e[0..n-2] (e[i] couples i and i+1), by the root-free implicit
 * QL iteration on the host (Pal, Walker and Kahan; Reinsch 1971), into
 * lambda[0..n-1] in ascending order; each within a few eps of the matrix
 * norm.  Host arrays, owned by the caller; d and e are not modified; lambda
 * may not alias them.  n = 0 is a no-op.  ED_EINVAL for n < 0 or a NULL
 * array (e may be NULL for n <= 1); ED_ENOCONV if a block needs more than 60
 * QL sweeps.  Needs no device. */
ed_status ed_tridiag_eigenvalues(const double* d, const double* e, int64_t n, double* lambda);

/* ---- dense-block form -----------------------------------------------------
 * The bipartite operator of paper Eq. (2) with dense side operators on
 * symmetry blocks (its DMRG setting): blocks q = 0..nq-1 of dimension
 * chi[q] x chi[q] (left x right index), the state the concatenation of the
 * row-major blocks Psi_q (dimension sum_q chi_q^2), and
 *   (H psi)_q' = H_L,q' Psi_q' + Psi_q' H_R,q'^T + sum_m L_m,q Psi_q R_m,q^T
 * over the cross terms m with q' = q + delta[m] (the Vec identity
 * [L (x) R] Vec(Psi) = Vec(L Psi R^T), row-major).  Every product runs on
 * the tensor cores in FP64-accurate digit-split form (each FP64 row scaled
 * by a power of two and split into 8 BF16 digits; digit products summed
 * exactly in FP32 per digit order, combined in FP64), one launch per stage.
 * A tensor-core wait that runs out (it should not) sets an error flag the
 * library keeps, and the apply's output is then incomplete.
 *   HL, HR   host pointers, one per block: chi_q x chi_q row-major
 *   delta    per cross term, nonzero
 *   Lm, Rm   host pointers [m * nq + q]: chi_{q+delta} x chi_q row-major for
 *            the source blocks q with q + delta inside 0..nq-1, NULL otherwise
 * The matrices are copied to the device; the caller keeps its own.
 * ed_dense_apply: x, y device FP64 vectors of ed_dense_dim elements, not
 * overlapping; asynchronous on the stream.  One operator holds one scratch
 * buffer for its partial products: applies of the same operator must not
 * overlap on the GPU (use one stream, or synchronise between them). */
typedef struct ed_dense ed_dense;
ed_status ed_dense_create(int nq, const int64_t* chi, const double* const* HL, const double* const* HR, int n_terms,
                          const int* delta, const double* const* Lm, const double* const* Rm, ed_dense** out);
int64_t ed_dense_dim(const ed_dense* d);
ed_status ed_dense_apply(ed_dense* d, const double* x, double* y, void* stream);
void ed_dense_destroy(ed_dense* d);

/* ---- batched form -------------------------------------------------------
 * Many independent single-block instances (Hubbard models with the spin
 * cut) packed into one device arena and stepped together: every kernel is
 * one persistent launch over all (instance, row), (instance, tile) or
 * (instance, chunk) work items of the active instances, and the whole
 * Lanczos step (apply, FP64 reductions, vector update) is one captured CUDA
 * graph replayed each step.  Eq. (2) for one block with the spin cut (no
 * cross terms): H psi = H_A Psi + Psi H_B^T + V o Psi.  Per instance, H psi
 * runs in one of three modes:
 *   0  CSR: the side operators as sparse rows, one warp per row of Psi;
 *   1  dense on the tensor cores, 128 x 64 output tiles;
 *   2  dense on the tensor cores, 128 x 128 output tiles.
 * The dense modes (instances with d_A, d_B <= 1024) hold H_A and H_B as
 * dense matrices and form both products with BF16 tcgen05 MMAs and FP32
 * accumulation, every FP32 operand split into three BF16 pieces (24
 * significant bits; piece products of order <= 2 kept), so the result has
 * FP32 accuracy.  flags: ED_OPS_DEFAULT times every mode on each instance
 * shape (d_A, d_B, nonzeros of H_A and H_B) and keeps the fastest, cached
 * per process (so a shape is timed once); ED_OPS_FORCE_CSR uses mode 0 and
 * allocates no dense tables; ED_OPS_FORCE_DENSE uses mode 1 when d_B <= 64,
 * else 2, wherever the instance has a dense form.
 * Vectors are FP32; reductions are FP64-accurate.  A tensor-core wait that
 * runs out (it should not) sets an error flag; the next ed_batch_lanczos
 * or ed_batch_create then returns ED_ETIMEOUT. */
typedef struct ed_batch ed_batch;
ed_status ed_batch_create(const ed_model_desc* models, int n, int flags, ed_batch** out);
/* total elements of the concatenated layout (instance i at off[i]) */
int64_t ed_batch_dim(const ed_batch* b);
ed_status ed_batch_offsets(const ed_batch* b, int64_t* off /* n+1, host */);
/* modes: host n ints (nullable), the mode of each instance (0, 1, 2 above);
 * tune_ms: host 4 floats (nullable), device time of one batched H psi with
 * every instance in mode 0, in mode 1, in mode 2 (where it has a dense
 * form), and with the chosen modes; under a forced flag only the last is
 * measured, the others are 0 */
ed_status ed_batch_info(const ed_batch* b, int* modes, float* tune_ms);
/* y = H x for all instances (device FP32 vectors in the concatenated layout) */
ed_status ed_batch_apply(ed_batch* b, const void* x, void* y, ed_dtype dtype, void* stream);
/* ground-state energies of all instances (mode ED_LZ_F32; tol: relative
 * change of the lowest Ritz value between checks every check_every steps).
 * e0: host n doubles; iters: host n ints (nullable).  Synchronises. */
ed_status ed_batch_lanczos(ed_batch* b, const ed_lanczos_opts* opts, double* e0, int* iters, ed_report* rep);
void ed_batch_destroy(ed_batch* b);

/* ---- serving form -------------------------------------------------------
 * A request loop with continuous batching over the batched engine: a worker
 * thread admits queued requests in arrival order whenever a slot is free
 * and the request's tables plus three FP32 Krylov vectors fit in the
 * device budget (one arena allocated at creation), keeps their Krylov state
 * resident, steps all admitted requests together, and completes each one
 * when its lowest Ritz value is stable to tol at a multiple of check_every
 * steps since its admission (so a result does not depend on the other
 * requests in the mix).  Requests: Hubbard models with the spin cut. */
typedef struct ed_server ed_server;
typedef struct {
  int64_t device_bytes;       /* arena for tables and Krylov vectors */
  int max_slots;              /* requests on the device at once (<= 4096) */
  int max_iter;               /* Lanczos steps per request */
  int check_every;            /* steps between convergence checks */
  double tol;                 /* relative change of the lowest Ritz value */
  uint64_t seed;              /* start vectors (key-indexed SplitMix64) */
  int inject_alloc_failures;  /* test hook: fail this many admissions with ED_ENOMEM */
} ed_server_opts;
typedef struct {
  double e0;
  int iterations;
  int converged;
  int status;                 /* ed_status of the request */
  double latency_s;           /* submit -> done */
  double queue_s;             /* submit -> admitted */
  double run_s;               /* admitted -> done */
} ed_result;
typedef struct {
  int64_t submitted, completed, failed, queued, running;
  double p50_s, p99_s, mean_s;    /* latency of completed requests */
  double throughput_rps;          /* completed / (last completion - first submit) */
  int64_t device_bytes, device_bytes_free;
} ed_server_stats;
void ed_server_default_opts(ed_server_opts* o);
ed_status ed_server_create(const ed_server_opts* opts, ed_server** out);
/* queue a request (model arrays are copied); *ticket identifies it */
ed_status ed_server_submit(ed_server* s, const ed_model_desc* model, uint64_t* ticket);
/* wait at most timeout_ms for the request: ED_ETIMEOUT if it has not
 * finished, otherwise the request's status with *res filled */
ed_status ed_server_wait(ed_server* s, uint64_t ticket, int timeout_ms, ed_result* res);
/* cancel a queued or running request (it leaves between steps) */
ed_status ed_server_cancel(ed_server* s, uint64_t ticket);
ed_status ed_server_get_stats(ed_server* s, ed_server_stats* out);
/* stops the worker after its current step and frees the device arena */
void ed_server_destroy(ed_server* s);

/* ---- tracing ------------------------------------------------------------
 * Per-stage CUDA-event timing of ed_apply_H.  While enabled, every apply
 * records events on the caller's stream around its stages: 0 = exponent of
 * max|x|, 1 = fixed-point copy (both only on the exact FP64 path), 2 = row
 * pass (diagonal, H_B, cross terms), 3 = H_A panel pass.  ed_profile_read
 * waits for the recorded applies and returns the accumulated milliseconds
 * per stage (ms: host array of 4) and the number of applies; reset != 0
 * clears the totals.  Applies that do not use the class-sorted kernels
 * record nothing. */
ed_status ed_profile_enable(ed_ctx* ctx, int enable);
ed_status ed_profile_read(ed_ctx* ctx, double* ms, int64_t* count, int reset);
/* Which row pass ed_apply_H runs for `dtype` on this context: 0 = the
 * plain per-row kernel (the class-sorted kernels do not apply), 1 = the
 * class-sorted row pass (k_row5); negative: ed_build_local_ops has not run. */
int ed_row_pass(const ed_ctx* ctx, ed_dtype dtype);
/* Arithmetic of the FP64 apply on this context (Eq. (2) evaluated on a
 * fixed-point copy of x unless 0): 0 = FP64 arithmetic per matrix element;
 * 1 = every coupling dyadic: exact 64-bit integer sums, rounded once;
 * 2 = couplings not dyadic: class sums weighted by 64-bit integers (every
 *     FP64 coupling and diagonal term as an integer multiple of one power of
 *     two) into exact 128-bit sums, rounded once per pass;
 * 3 = value range too wide for 2: class sums weighted in FP64.
 * Negative: ed_build_local_ops has not run. */
int ed_fp64_mode(const ed_ctx* ctx);

/* ---- queries ---------------------------------------------------------- */
int64_t ed_dim(const ed_ctx* ctx);
int ed_num_blocks(const ed_ctx* ctx);
/* per block: charge s, d_A, d_B, element offset (host arrays of ed_num_blocks) */
ed_status ed_blocks(const ed_ctx* ctx, int* s, int64_t* dA, int64_t* dB, int64_t* off);
/* bit-string keys (oracle convention: spin key bit i = site i; Hubbard
 * key = up | dw << n_sites) of the global indices [start, start+count), host. */
ed_status ed_state_keys(const ed_ctx* ctx, int64_t start, int64_t count, uint64_t* keys);
/* lattice site of each side-local bit: side 0 = A, 1 = B; sites: host array
 * of at least n_sites ints, *n_bits: bits on that side. */
ed_status ed_side_sites(const ed_ctx* ctx, int side, int* sites, int* n_bits);
/* fill x (device, ed_dim elements of dtype) with the key-indexed SplitMix64
 * values U[-1,1) for `seed` (unnormalised); enqueued on stream. */
ed_status ed_random_vector(ed_ctx* ctx, uint64_t seed, void* x, ed_dtype dtype, void* stream);
/* device memory held by the context, bytes */
int64_t ed_device_bytes(const ed_ctx* ctx);
void ed_destroy(ed_ctx* ctx);
const char* ed_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ED_H */
