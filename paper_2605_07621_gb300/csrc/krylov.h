// Internal declarations shared by the Krylov kernels and drivers.
#pragma once

#include <cuda_bf16.h>

#include <vector>

#include "ed_internal.h"

namespace edk {

constexpr int kMaxPartials = 4096;
constexpr int kMaxBasis = 2048;  // reorthogonalisation coefficients kept on the device

ed_status apply_H_impl(ed_ctx* c, const void* x, void* y, ed_dtype dt, cudaStream_t st);
ed_status random_vector_impl(const ed_ctx* c, uint64_t seed, void* x, ed_dtype dt, cudaStream_t st);

int grid_for(const ed_ctx* c, long long n);
ed_status ensure_scratch(ed_ctx* c);
double* slot(ed_ctx* c, int k);
double* hcoef(ed_ctx* c);
template <typename T>
ed_status dot_dev(ed_ctx* c, const T* a, const T* b, long long n, double* out, cudaStream_t st, int op);
ed_status read_scalars(ed_ctx* c, int first, int count, double* out, cudaStream_t st);
double tridiag_lowest(const double* a, const double* b, int m);
void tridiag_vector(const double* a, const double* b, int m, double theta, std::vector<double>& s);

// kernel launchers (krylov_launch.cu)
template <typename T>
void launch_lz_a(ed_ctx* c, T* w, const T* v, const T* vprev, int use_beta, long long n, cudaStream_t st);
template <typename T>
void launch_lz_b(ed_ctx* c, T* w, const T* v, long long n, cudaStream_t st);
template <typename T>
void launch_lz_c(ed_ctx* c, const T* w, T* out, long long n, cudaStream_t st);
// FP64 Lanczos steps that hand the next H|psi> its fixed-point input:
// lz_b also records the largest exponent of w in *ew; lz_c also writes the
// fixed-point copy X of w / beta and its scale (biased exponent) to *ex
void launch_lz_b_emax(ed_ctx* c, double* w, const double* v, long long n, int* ew, cudaStream_t st);
void launch_lz_c_fixed(ed_ctx* c, const double* w, double* out, long long* X, const int* ew, int* ex, long long n,
                       cudaStream_t st);
// H|psi> of the exact fixed-point path from an input already converted
// (c->d_fixed with the scale in c->d_exp[0]); y receives FP64.  x is the
// FP64 input itself (read only when the diagonal is added in FP64)
ed_status apply_prepared_fixed(ed_ctx* c, const double* x, double* y, cudaStream_t st);
// the fixed-point FP64 path applies to x on this context
bool fixed_path(const ed_ctx* c, const void* x);
template <typename T>
void launch_lz_rerun(ed_ctx* c, const T* w, const T* v, const T* vprev, double alpha, double beta, double inv_next,
                     T* out, long long n, cudaStream_t st);
template <typename TI, typename TO>
void launch_scale_cvt(ed_ctx* c, const TI* x, TO* y, double s, long long n, cudaStream_t st);
template <typename TB, typename TO>
void launch_axpy_basis(ed_ctx* c, const TB* v, TO* x, double s, long long n, cudaStream_t st);
// hist[2j], hist[2j+1] = alpha_j, beta_{j+1} from the scalar slots, j = *counter (incremented)
void launch_hist_push(ed_ctx* c, double* hist, int* counter, cudaStream_t st);
template <typename TI, typename TO>
void launch_cvt(ed_ctx* c, const TI* x, TO* y, long long n, cudaStream_t st);
// x = sum_j s_j V_j over m <= kMaxBasis FP32 vectors V_j = V + j n (float-float sums)
ed_status launch_combine_f32(ed_ctx* c, const float* V, long long n, const double* s, int m, double* x,
                             cudaStream_t st);
template <typename T>
void launch_axpy_dev(ed_ctx* c, const T* x, T* y, const double* s, double sign, long long n, cudaStream_t st);
template <typename T>
void launch_reorth(ed_ctx* c, const T* V, long long ldv, int m, T* w, long long n, double* h, cudaStream_t st);
void launch_green_cf(const double* omega, int n_omega, double eta, double e0, const double* ap, const double* bp, int mp,
                     double wp, const double* ah, const double* bh, int mh, double wh, double* G, cudaStream_t st);
void launch_fermion_remap(ed_ctx* c, const double* psi, long long dA_src, long long dB_src, double* phi,
                          long long dA_dst, long long dB_dst, const int* map, const signed char* sgn, int side,
                          cudaStream_t st);

}  // namespace edk
