/*
 * ed_oracle.c -- plain CPU exact-diagonalisation oracle (TEST INFRASTRUCTURE).
 *
 * This file is test infrastructure: only the tests, the smoke check and the
 * bench's CPU-baseline leg may load it.  It shares no code with the CUDA path.
 *
 * It builds nothing in the bipartite (entanglement-cut) representation.  It
 * works in the full, unsplit symmetry sector of the paper's K-local model
 * (Eq. (1)): the basis is the ascending list of bit-string keys with fixed
 * particle numbers, and H is applied term by term to each full bit string.
 * By Eqs. (2)-(3) the bipartite H|psi> is the same linear map up to a
 * permutation of basis states, so this is the definition the GPU path must
 * reproduce.
 *
 * Models (the paper names them but prints no normalisation; these are the
 * readings used throughout):
 *   spin-1/2 XXZ:  H = sum_b [ jz_b S^z_i S^z_j + jxy_b/2 (S^+_i S^-_j + S^-_i S^+_j) ]
 *                  key bit i = 1 <=> site i spin up.
 *   Hubbard:       H = -sum_{b,sigma} t_b (c^dag_{i sigma} c_{j sigma} + h.c.)
 *                      + sum_i U_i n_{i up} n_{i dw} + sum_i eps_i (n_{i up} + n_{i dw})
 *                  key = up | (dw << S); fermionic operator order is the bit
 *                  order of the key (all up sites ascending, then all down
 *                  sites ascending), so a hop between key bits p and q picks
 *                  up (-1)^(number of set key bits strictly between p and q).
 *
 * Plain C99 + OpenMP; index lookup is a binary search in the sorted key list
 * (narrowed by a bucket table of the leading key bits).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_SPIN 0
#define OR_HUBBARD 1

typedef struct {
  int kind;          /* OR_SPIN or OR_HUBBARD */
  int n_sites;
  int n_bonds;
  const int *bi, *bj;
  const double *jxy, *jz; /* spin: per bond */
  const double *t;        /* Hubbard: per bond */
  const double *U, *eps;  /* Hubbard: per site */
} or_model;

static int popc64(uint64_t x) { return __builtin_popcountll(x); }

/* number of k-subsets of n */
static int64_t binom(int n, int k) {
  if (k < 0 || k > n) return 0;
  int64_t r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

int64_t or_sector_dim(const or_model* m, int n_up, int n_dw) {
  if (m->kind == OR_SPIN) return binom(m->n_sites, n_up);
  return binom(m->n_sites, n_up) * binom(m->n_sites, n_dw);
}

/* next larger integer with the same popcount (Gosper) */
static uint64_t next_comb(uint64_t v) {
  uint64_t t = v | (v - 1);
  return (t + 1) | (((~t & -~t) - 1) >> (__builtin_ctzll(v) + 1));
}

/* all n-bit strings with popcount k, ascending; returns count */
static int64_t list_comb(int n, int k, uint64_t* out) {
  int64_t c = 0;
  if (k == 0) { out[0] = 0; return 1; }
  uint64_t v = (k == 64) ? ~0ULL : ((1ULL << k) - 1);
  uint64_t lim = (n == 64) ? 0 : (1ULL << n);
  for (;;) {
    out[c++] = v;
    if (k == n) break;
    uint64_t w = next_comb(v);
    if (w >= lim || w <= v) break;
    v = w;
  }
  return c;
}

/* Sector keys in ascending order.  Returns the count, or -1 if cap is too small. */
int64_t or_sector_keys(const or_model* m, int n_up, int n_dw, uint64_t* keys, int64_t cap) {
  int n = m->n_sites;
  int64_t d = or_sector_dim(m, n_up, n_dw);
  if (d > cap) return -1;
  if (m->kind == OR_SPIN) return list_comb(n, n_up, keys);
  int64_t du = binom(n, n_up), dd = binom(n, n_dw);
  uint64_t* up = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)du);
  uint64_t* dw = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)dd);
  list_comb(n, n_up, up);
  list_comb(n, n_dw, dw);
  /* key = up | dw << n ascends with dw (outer) then up (inner) */
  for (int64_t j = 0; j < dd; ++j)
    for (int64_t i = 0; i < du; ++i) keys[j * du + i] = up[i] | (dw[j] << n);
  free(up);
  free(dw);
  return d;
}

/* Matrix elements of row `key`: H|key'> components <key|H|key'>.
 * Writes the diagonal element to *diag and the off-diagonal (key', value)
 * pairs to nk/nv; returns the number of off-diagonal entries (<= cap). */
int or_row(const or_model* m, uint64_t key, double* diag, uint64_t* nk, double* nv, int cap) {
  int n = m->n_sites, c = 0;
  double d = 0.0;
  if (m->kind == OR_SPIN) {
    for (int b = 0; b < m->n_bonds; ++b) {
      int i = m->bi[b], j = m->bj[b];
      int si = (int)((key >> i) & 1), sj = (int)((key >> j) & 1);
      /* S^z_i S^z_j = +1/4 for parallel, -1/4 for antiparallel spins */
      d += m->jz[b] * ((si == sj) ? 0.25 : -0.25);
      /* (S^+_i S^-_j + S^-_i S^+_j)/2 swaps antiparallel spins with element 1/2 */
      if (si != sj && m->jxy[b] != 0.0) {
        if (c >= cap) return -1;
        nk[c] = key ^ ((1ULL << i) | (1ULL << j));
        nv[c] = 0.5 * m->jxy[b];
        ++c;
      }
    }
  } else {
    uint64_t up = key & ((n == 64) ? ~0ULL : ((1ULL << n) - 1));
    uint64_t dw = key >> n;
    for (int s = 0; s < n; ++s) {
      int nu = (int)((up >> s) & 1), nd = (int)((dw >> s) & 1);
      d += m->U[s] * nu * nd + m->eps[s] * (nu + nd);
    }
    for (int b = 0; b < m->n_bonds; ++b) {
      if (m->t[b] == 0.0) continue;
      for (int sp = 0; sp < 2; ++sp) {
        int p = m->bi[b] + sp * n, q = m->bj[b] + sp * n;
        int op = (int)((key >> p) & 1), oq = (int)((key >> q) & 1);
        if (op == oq) continue; /* c^dag_p c_q + c^dag_q c_p needs exactly one occupied */
        int lo = p < q ? p : q, hi = p < q ? q : p;
        uint64_t between = (hi - lo > 1) ? (((1ULL << hi) - 1) & ~((1ULL << (lo + 1)) - 1)) : 0ULL;
        int sign = (popc64(key & between) & 1) ? -1 : 1;
        if (c >= cap) return -1;
        nk[c] = key ^ ((1ULL << p) | (1ULL << q));
        nv[c] = -m->t[b] * sign;
        ++c;
      }
    }
  }
  *diag = d;
  return c;
}

/* ---------------------------------------------------------------- index lookup */

typedef struct {
  const uint64_t* keys;
  int64_t D;
  int shift;        /* bucket = key >> shift */
  int64_t* bucket;  /* size nb + 1 */
  int64_t nb;
} or_index;

static int key_bits(const or_model* m) { return m->kind == OR_SPIN ? m->n_sites : 2 * m->n_sites; }

static void index_build(or_index* ix, const or_model* m, const uint64_t* keys, int64_t D) {
  int nbits = key_bits(m);
  int bb = nbits < 22 ? nbits : 22;
  ix->keys = keys;
  ix->D = D;
  ix->shift = nbits - bb;
  ix->nb = (int64_t)1 << bb;
  ix->bucket = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ix->nb + 1));
  if (!ix->bucket) return;
  int64_t p = 0;
  for (int64_t h = 0; h < ix->nb; ++h) {
    while (p < D && (keys[p] >> ix->shift) < (uint64_t)h) ++p;
    ix->bucket[h] = p;
  }
  ix->bucket[ix->nb] = D;
}

static void index_free(or_index* ix) { free(ix->bucket); }

/* position of key in the sorted list, or -1 */
static int64_t index_find(const or_index* ix, uint64_t key) {
  uint64_t h = key >> ix->shift;
  if (h >= (uint64_t)ix->nb) return -1;
  int64_t lo = ix->bucket[h], hi = ix->bucket[h + 1] - 1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    uint64_t k = ix->keys[mid];
    if (k == key) return mid;
    if (k < key) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

/* position of each key (or -1) */
int or_find(const or_model* m, const uint64_t* keys, int64_t D, const uint64_t* q, int64_t nq, int64_t* pos) {
  or_index ix;
  index_build(&ix, m, keys, D);
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < nq; ++r) pos[r] = index_find(&ix, q[r]);
  index_free(&ix);
  return 0;
}

#define ROW_CAP 512

/* (H x)[r] for one row r of the sorted basis: the diagonal term plus every
 * off-diagonal term, in the order or_row lists them.  Sets *bad if a
 * connected state is missing from the basis. */
static double row_value(const or_model* m, const or_index* ix, const uint64_t* keys, const double* x, int64_t r,
                        uint64_t* nk, double* nv, int* bad) {
  double diag;
  int c = or_row(m, keys[r], &diag, nk, nv, ROW_CAP);
  if (c < 0) { *bad = 1; return 0.0; }
  double acc = diag * x[r];
  for (int e = 0; e < c; ++e) {
    int64_t col = index_find(ix, nk[e]);
    if (col < 0) { *bad = 1; continue; }
    acc += nv[e] * x[col];
  }
  return acc;
}

/* Rows [r0, r1) of y = H x on the full sector with sorted basis `keys`
 * (length D); y has r1 - r0 entries.  Returns 0, or -1 if a connected state
 * is missing from the basis (which would mean H leaves the sector). */
int or_apply_range(const or_model* m, const uint64_t* keys, int64_t D, const double* x, int64_t r0, int64_t r1,
                   double* y, int nthreads) {
  or_index ix;
  index_build(&ix, m, keys, D);
  int bad = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel reduction(| : bad)
  {
    uint64_t nk[ROW_CAP];
    double nv[ROW_CAP];
#pragma omp for schedule(static)
    for (int64_t r = r0; r < r1; ++r) y[r - r0] = row_value(m, &ix, keys, x, r, nk, nv, &bad);
  }
  index_free(&ix);
  return bad ? -1 : 0;
}

/* A lookup index built once and kept (for repeated row evaluations of one
 * large sector): or_index_new returns NULL on allocation failure. */
void* or_index_new(const or_model* m, const uint64_t* keys, int64_t D) {
  or_index* ix = (or_index*)malloc(sizeof(or_index));
  if (!ix) return NULL;
  index_build(ix, m, keys, D);
  if (!ix->bucket) { free(ix); return NULL; }
  return ix;
}

void or_index_delete(void* h) {
  if (!h) return;
  index_free((or_index*)h);
  free(h);
}

/* y[i] = (H x)[rows[i]] for n listed rows, with an index from or_index_new
 * over the same sorted keys; same arithmetic per row as or_apply_range. */
int or_apply_rows_ix(const or_model* m, const void* h, const double* x, const int64_t* rows, int64_t n, double* y,
                     int nthreads) {
  const or_index* ix = (const or_index*)h;
  int bad = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel reduction(| : bad)
  {
    uint64_t nk[ROW_CAP];
    double nv[ROW_CAP];
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      int64_t r = rows[i];
      if (r < 0 || r >= ix->D) { bad = 1; y[i] = 0.0; continue; }
      y[i] = row_value(m, ix, ix->keys, x, r, nk, nv, &bad);
    }
  }
  return bad ? -1 : 0;
}

/* y = H x on the full sector (all rows). */
int or_apply(const or_model* m, const uint64_t* keys, int64_t D, const double* x, double* y, int nthreads) {
  return or_apply_range(m, keys, D, x, 0, D, y, nthreads);
}

/* Dense H (row-major D x D) for small sectors. */
int or_dense(const or_model* m, const uint64_t* keys, int64_t D, double* H) {
  or_index ix;
  index_build(&ix, m, keys, D);
  int bad = 0;
  memset(H, 0, sizeof(double) * (size_t)D * (size_t)D);
#pragma omp parallel reduction(| : bad)
  {
    uint64_t nk[ROW_CAP];
    double nv[ROW_CAP];
#pragma omp for schedule(static)
    for (int64_t r = 0; r < D; ++r) {
      double diag;
      int c = or_row(m, keys[r], &diag, nk, nv, ROW_CAP);
      if (c < 0) { bad = 1; continue; }
      H[r * D + r] += diag;
      for (int e = 0; e < c; ++e) {
        int64_t col = index_find(&ix, nk[e]);
        if (col < 0) { bad = 1; continue; }
        H[r * D + col] += nv[e];
      }
    }
  }
  index_free(&ix);
  return bad ? -1 : 0;
}

/* Row terms of many keys at once (for sampled-row checks of huge sectors):
 * for query r, entries [off[r], off[r+1]) of (nk, nv) hold its off-diagonal
 * terms and diag[r] its diagonal.  off must have nq+1 slots and nk/nv
 * capacity cap.  Returns the total number of entries, or -1 on overflow. */
int64_t or_rows(const or_model* m, const uint64_t* q, int64_t nq, double* diag, int64_t* off, uint64_t* nk,
                double* nv, int64_t cap) {
  int64_t tot = 0;
  uint64_t tk[ROW_CAP];
  double tv[ROW_CAP];
  for (int64_t r = 0; r < nq; ++r) {
    off[r] = tot;
    int c = or_row(m, q[r], &diag[r], tk, tv, ROW_CAP);
    if (c < 0 || tot + c > cap) return -1;
    memcpy(nk + tot, tk, sizeof(uint64_t) * (size_t)c);
    memcpy(nv + tot, tv, sizeof(double) * (size_t)c);
    tot += c;
  }
  off[nq] = tot;
  return tot;
}

/* Fermion operator on Hubbard keys: c^dag_{site,spin} (create=1) or
 * c_{site,spin} (create=0) applied to psi (basis `src`, length Ds) gives phi
 * in basis `dst` (length Dd).  Sign (-1)^(set key bits below the operator's
 * bit position), from the operator order stated above.  Returns 0 or -1. */
int or_fermion_op(const or_model* m, int site, int spin, int create, const uint64_t* src, int64_t Ds,
                  const double* psi, const uint64_t* dst, int64_t Dd, double* phi) {
  int p = site + (spin ? m->n_sites : 0);
  or_index ix;
  index_build(&ix, m, src, Ds);
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int64_t r = 0; r < Dd; ++r) {
    uint64_t k = dst[r];
    int occ = (int)((k >> p) & 1);
    /* c^dag_p |k'> = sign |k> needs k' = k with bit p cleared and bit p set in k */
    if ((create && !occ) || (!create && occ)) { phi[r] = 0.0; continue; }
    uint64_t kp = k ^ (1ULL << p);
    int64_t col = index_find(&ix, kp);
    if (col < 0) { bad = 1; phi[r] = 0.0; continue; }
    uint64_t below = (p == 0) ? 0ULL : ((1ULL << p) - 1);
    int sign = (popc64(kp & below) & 1) ? -1 : 1;
    phi[r] = sign * psi[col];
  }
  index_free(&ix);
  return bad ? -1 : 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
