// Dense Hermitian eigensolver building blocks written for GB300 (rpa_dense.cu):
// the subspace of chi~(0) (step a3) without a vendor solver.
//
//  * hetrd: Householder reduction of an n x n Hermitian matrix (column-major,
//    full storage) to a real symmetric tridiagonal T = Q^H A Q, in FP32 or FP64.
//    One persistent cooperative kernel walks the columns; the rank-2 updates of
//    a panel of 32 columns are deferred and applied to the trailing matrix at
//    the end of the panel (the blocked scheme of Dongarra, Sorensen and
//    Hammarling 1989), with grid-wide barriers between the steps that need all
//    of a column.  The reflectors v_k (leading 1 explicit) overwrite
//    A(k+1:n, k); Q = H_0 H_1 ... H_{n-2}, H_k = I - tau_k v_k v_k^H.
//  * apply_q: X <- Q X for an n x m block X, reflectors applied in blocks of 32
//    in the compact WY form I - V T V^H (Schreiber and Van Loan 1989).
//  * jacobi: all eigenpairs of a small Hermitian matrix by cyclic two-sided
//    Jacobi rotations in FP64 (round-robin pairing, one persistent kernel).  On
//    the nearly diagonal Rayleigh quotients of the subspace refinement it
//    converges in a few sweeps and returns eigenvectors orthonormal to FP64
//    rounding.
//  * gemm_z: complex FP64 C = alpha op(A) op(B) + beta C on the FP64 pipe (the
//    FP64 path's block products).
//  * trinv: inverse of a lower-triangular matrix in FP64 (Cholesky-QR).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "rpa_internal.h"

namespace rpa {
namespace dense {

// Scratch of hetrd for matrices up to n_max (device pointers).
struct HetrdWork {
  void* vp = nullptr;    // [n_max][32] complex panel V (row-major)
  void* wp = nullptr;    // [n_max][32] complex panel W
  void* xcol = nullptr;  // [n_max] complex
  void* ycol = nullptr;  // [n_max] complex
  void* part = nullptr;  // [grid][65] complex partial sums
  void* part2 = nullptr; // [grid] complex
  unsigned* bar = nullptr;  // barrier words
  int* status = nullptr;    // nonzero: a barrier wait ran out
  int n_max = 0, grid = 0;
  size_t elem = 0;          // bytes of one complex element (8 or 16)
};

// Allocate for matrices up to n_max with complex elements of `elem` bytes (8: FP32
// reduction, 16: FP64).  grid: persistent CTAs (0: one per SM).
rpa_status hetrd_alloc(HetrdWork& w, int n_max, size_t elem, std::string& err);
void hetrd_free(HetrdWork& w);

// Reduce the n x n Hermitian column-major A (complex of T, full storage; float2 for
// T = float, double2 for T = double) to tridiagonal form: d[n], e[n-1] (real T),
// tau[n-1] (complex T); the reflectors overwrite A's strictly lower part (A(k+1, k)
// holds 1).  Returns RPA_ETIMEOUT if a grid barrier ran out.
template <typename T>
rpa_status hetrd(HetrdWork& w, void* a, int n, T* d, T* e, void* tau, cudaStream_t st,
                 std::string& err, int* launches);

// X <- Q X, X n x m column-major (ld n), complex of T; a and tau as left by hetrd.
// tfac: scratch of ceil((n-1)/32) * 32 * 32 complex of T.
template <typename T>
rpa_status apply_q(const void* a, const void* tau, int n, void* x, int m, void* tfac,
                   cudaStream_t st, std::string& err, int* launches);

// Scratch of the Jacobi eigensolver for matrices up to m_max.
struct JacobiWork {
  double* prm = nullptr;   // rotation parameters [m_max/2 + 1][4]
  double* part = nullptr;  // per-CTA convergence measures
  unsigned* bar = nullptr;
  int* status = nullptr;
  int* perm = nullptr;     // [m_max] ascending order of the eigenvalues
  int m_max = 0, grid = 0;
};
rpa_status jacobi_alloc(JacobiWork& w, int m_max, std::string& err);
void jacobi_free(JacobiWork& w);

// All eigenpairs of the m x m Hermitian column-major g (complex128, destroyed):
// theta[m] ascending, y (m x m column-major, ld m) the eigenvectors in that order.
// ywork: m x m complex128 scratch.  Returns RPA_ETIMEOUT if a barrier ran out.
rpa_status jacobi(JacobiWork& w, cplx* g, int m, double* theta, cplx* y, cplx* ywork,
                  cudaStream_t st, std::string& err, int* launches);

// C (m x n, ldc) = alpha op(A) op(B) + beta C, complex128 column-major; op = 'N',
// 'T' or 'C' (conjugate transpose).  op(A) is m x k, op(B) k x n.
rpa_status gemm_z(char opa, char opb, int m, int n, int k, cplx alpha, const cplx* a, int lda,
                  const cplx* b, int ldb, cplx beta, cplx* c, int ldc, cudaStream_t st,
                  std::string& err, int* launches);

// Overwrite the upper-triangular n x n R (complex128, column-major, leading
// dimension ld, strictly lower part zero) with R^-1 by recursive doubling:
// [R11 R12; 0 R22]^-1 = [X11, -X11 R12 X22; 0, X22], 32 x 32 diagonal tiles by
// back substitution.  work: n x n complex128 scratch.
rpa_status trinv_upper(cplx* r, int n, int ld, cplx* work, cudaStream_t st, std::string& err,
                       int* launches);

}  // namespace dense
}  // namespace rpa
