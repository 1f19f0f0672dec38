// Internal declarations shared by the CUDA translation units of librpa.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/rpa.h"

namespace rpa {

// Record the message that rpa_last_error(NULL) returns for plan-less calls.
void set_call_error(const char* msg);

struct cplx {
  double re, im;
};

// Transitions of a q-point: k-points x valence x conduction.
inline long n_transitions(const rpa_qpoint& q) {
  return (long)(q.n_k > 1 ? q.n_k : 1) * q.n_v * q.n_c;
}

// ---- mixed-precision subspace of chi~(0) (rpa_eig.cu) ---------------------

namespace tc {
struct Workspace;
}

namespace eig {
// Extra vectors carried beyond N_eig through the start and the FP64 step.
int extra_vectors(int n_eig);
// Whether the mixed path takes the subspace this way (opt-in with RPA_EIG_MIXED=1;
// N_G >= 1024 and room for the extra vectors).
bool applies(int n, int n_eig);
// Whether its chi~ X products run on the tensor-core GEMM (RPA_EIG_TC, default on).
bool products_on_tc();
struct Refine {
  void* blas = nullptr;               // cublasHandle_t
  float2* h32 = nullptr;              // chi~ / max|chi~| in complex64, n x n (then reflectors)
  float *d32 = nullptr, *e32 = nullptr;  // FP32 tridiagonal T: diagonal, off-diagonal
  float2* tau32 = nullptr;            // its Householder scalars
  double *d64 = nullptr, *e64 = nullptr, *e2 = nullptr;  // T in FP64, e^2
  float* e2f = nullptr;               // e^2 in FP32 (the FP32 bisection phase)
  double* wt = nullptr;               // m' + 1 smallest eigenvalues of T
  int* first = nullptr;               // cluster starts of those eigenvalues
  double* zt = nullptr;               // eigenvectors of T, n x m' row-major
  double* lanes = nullptr;            // inverse-iteration scratch, 6 n x m'
  float2* c32 = nullptr;              // T's eigenvectors, then chi~'s, n x m' complex64
  cplx* bt = nullptr;                 // conj-transposed block, a tensor-core GEMM operand
  cplx* yb = nullptr;                 // conj-transposed Ritz coefficients, m' x m'
  double* dinv = nullptr;             // inverse column norms (Cholesky-QR)
  cplx *x0 = nullptr, *x1 = nullptr, *x2 = nullptr;  // n x m' blocks (column-major)
  cplx* tau = nullptr;                // Householder scalars
  cplx* g = nullptr;                  // m' x m' Rayleigh quotient
  double* theta = nullptr;            // its eigenvalues
  unsigned long long* absmax = nullptr;
  int* info = nullptr;
  void* dwork = nullptr;
  size_t dbytes = 0;
  void* hwork = nullptr;
  size_t hbytes = 0;
  int max_n = 0, max_mp = 0;
  rpa_status alloc(void* sol, void* params, int n_max, int mp_max, std::string& err);
  void release();
  // lam_out[0 .. n_eig) and the column-major n x n_eig vec_out: the N_eig most
  // negative eigenpairs of the column-major view hc (n x n, Hermitian, not modified).
  // With a tensor-core workspace the chi~ X products run on its digit-sliced
  // projection GEMM (sized for N_eig + extra_vectors columns), else in cuBLAS FP64.
  rpa_status subspace(void* sol, void* params, const cplx* hc, int n, int n_eig,
                      double* lam_out, cplx* vec_out, tc::Workspace* tcw, cudaStream_t st,
                      std::string& err, int* launches);
};
}  // namespace eig

// ---- FP64 SIMT contractions (rpa_fp64.cu) ---------------------------------

// chi[g][h] (+)= -(1/Omega) sum_vc conj(X[vc,g]) X[vc,h],  X = sf[vc] sv[g] A[vc,g].
// Upper block-triangle only; zero `chi` first when split_k > 1.
cudaError_t launch_herk_fp64(const void* A, int a_dtype, int n_vc, int n_g, const double* sf,
                             const double* sv, double scale, cplx* chi, cudaStream_t st);

// mt[i][vc] = conj(sum_g A[vc][g] B[g][i]), B = [n_g][n_eig].
cudaError_t launch_project_fp64(const void* A, int a_dtype, int n_vc, int n_g, const cplx* B,
                                int n_eig, cplx* mt, cudaStream_t st);

// chis[k][i][j] (+)= scale sum_vc f_k(vc) mt[i][vc] conj(mt[j][vc]) for all k; upper triangle;
// f_k(vc) = ow[vc] 4 D/(D^2 + w_k^2).
cudaError_t launch_chis_fp64(const cplx* mt, int n_eig, int n_vc, const double* delta,
                             const double* ow, const double* omega, int n_freq, double scale,
                             cplx* chis, cudaStream_t st);

// Fill the strictly lower triangle of `batch` n x n Hermitian matrices from the upper one,
// and zero the imaginary part of the diagonal.
cudaError_t launch_mirror_hermitian(cplx* m, int n, int batch, cudaStream_t st);

// ---- small kernels (rpa_small.cu) -------------------------------------------

// Per q-point scalars: sv[g] = sqrt(v(G)) (bare or slab-truncated), and per
// transition delta = e_c - e_v, pair weight ow = g_k (f_v - f_c), sf0 = sqrt(f(0)).
// bad |= 1 (|q+G|^2), 2 (transition energy), 4 (pair weight sign), 8 (slab kernel).
cudaError_t launch_prepare_scalars(const rpa_qpoint& q, double* sv, double* delta, double* ow,
                                   double* sf0, int* bad, cudaStream_t st);
cudaError_t launch_freq_grid(int n_freq, double s, double* omega, double* weight,
                             cudaStream_t st);
// C = conj(U) in canonical gauge; B = sv * C.  U column-major [n_g x n_eig] (ld = ldu).
cudaError_t launch_gauge(const cplx* U, int ldu, int n_g, int n_eig, const double* sv, cplx* C,
                         cplx* B, cudaStream_t st);
// w[vc] = sum_i |mt[i][vc]|^2 ; trace[k] = scale sum_vc f_k(vc) w[vc]
cudaError_t launch_trace(const cplx* mt, int n_eig, int n_vc, const double* delta,
                         const double* ow, const double* omega, int n_freq, double scale,
                         double* w, double* trace, cudaStream_t st);
// f[k][vc] = ow[vc] 4 D/(D^2 + w_k^2) for every frequency.
cudaError_t launch_all_freq_weights(const double* delta, const double* ow, int n_vc,
                                    const double* omega, int n_freq, double* f, cudaStream_t st);
// chis[k][i][i] := (scale sum_vc f[k][vc] |mt[i][vc]|^2, 0) in FP64: the exact diagonal of
// every chi_s(w_k), so that the tensor-core rounding leaves Tr chi_s untouched.
cudaError_t launch_chis_diagonal(const cplx* mt, int n_eig, int n_vc, const double* f,
                                 int n_freq, double scale, cplx* chis, cudaStream_t st);
// chi[g][g] = scale sv[g]^2 sum_vc sf0[vc]^2 |A[vc][g]|^2 in FP64 (the mixed path's
// chi~ diagonal); scratch holds up to 64 n_g doubles (fewer chunks if smaller).
cudaError_t launch_chi0_diagonal(const void* A, int dtype, long n_vc, int n_g, const double* sf0,
                                 const double* sv, double scale, double* scratch,
                                 size_t scratch_doubles, cplx* chi, cudaStream_t st);
// ec = (1/2pi) sum_k weight_k [sum_i log1p(-lam[k][i]) + trace_k]; bad |= 1 if 1 - lam <= 0.
cudaError_t launch_logsum(const double* lam, int n_eig, int ld_lam, int n_freq,
                          const double* trace, const double* weight, double* ec, int* bad,
                          cudaStream_t st);
// ec = (1/2pi) sum_k weight_k [logdet_k + trace_k]
cudaError_t launch_logdet_sum(const double* logdet, int n_freq, const double* trace,
                              const double* weight, double* ec, int* bad, cudaStream_t st);
// ---- tiled FP64 Cholesky (rpa_chol.cu) ----------------------------------------

// Complex elements of the scratch `inv` that a factorisation of `batch` matrices needs.
size_t cholesky_scratch_count(int batch);
// In-place Cholesky A = L L^H of `batch` Hermitian positive definite n x n matrices
// (row-major, stride n*n; the lower triangle is read and overwritten by L, the upper
// triangle is not touched).  logdet[b] += 2 sum_i ln L_ii when logdet is not NULL;
// bad |= 16 where a pivot is not > 0 (it is then taken as 1).  *launches += kernels.
cudaError_t launch_cholesky_tiled(cplx* a, int n, int batch, double* logdet, int* bad, cplx* inv,
                                  cudaStream_t st, int* launches);
// work[k] = I - chis[k] (lower triangle), then its Cholesky factor and
// logdet[k] = ln det(I - chis[k]) = 2 sum ln L_ii.
cudaError_t launch_cholesky_logdet(cplx* work, const cplx* chis, int n, int batch,
                                   double* logdet, int* bad, cplx* inv, cudaStream_t st,
                                   int* launches);
cudaError_t launch_generate_m(const rpa_qpoint* q, int v0, int nv, int c0, int nc, void* out,
                              int dtype, cudaStream_t st);

}  // namespace rpa
