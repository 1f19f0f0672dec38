// Subspace of chi~(0) (step a3, Method: the N_eig eigenvectors of chi~(0) with the
// most negative eigenvalues), computed by this library's own kernels (rpa_eig.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "rpa_dense.h"
#include "rpa_internal.h"
#include "rpa_tc.h"

namespace rpa {
namespace eig {

// Extra vectors carried beyond N_eig through the start and the refinement.
int extra_vectors(int n_eig);
// Size of the refined block, m' = min(n, N_eig + extra_vectors(N_eig)).
int block_size(int n, int n_eig);
// Whether a mixed-precision plan starts from the FP32 reduction of chi~ (n >= 1024,
// room for the extra vectors, RPA_EIG_START32 not 0); otherwise the start is the
// FP64 reduction.
bool start32(int n, int n_eig);
// Whether the block products of an FP32 start run on the tensor-core GEMM
// (RPA_EIG_TC, default on); the FP64 start uses FP64 products.
bool products_on_tc();
// Whether the plans take the library solver (RPA_EIG=cusolver) instead.
bool use_library();

struct Refine {
  // FP32 start
  float2* h32 = nullptr;                 // chi~ / max|chi~| (n x n), then its reflectors
  float *d32 = nullptr, *e32 = nullptr;  // T in FP32
  float2* tau32 = nullptr;
  // FP64 start
  cplx* tau64 = nullptr;
  // T in FP64 (and e^2, FP32 copies for the bisection)
  double *d64 = nullptr, *e64 = nullptr, *e2 = nullptr;
  float *e2f = nullptr, *d32b = nullptr;
  double* wt = nullptr;                  // the m' (+1) most negative eigenvalues of T
  int* first = nullptr;                  // cluster starts
  double* zt = nullptr;                  // eigenvectors of T, n x m' row-major
  double* lanes = nullptr;               // inverse-iteration scratch, 6 n x m'
  float2* c32 = nullptr;                 // back-transformed start, complex64 n x m'
  void* tfac = nullptr;                  // compact WY factors
  cplx *x0 = nullptr, *x1 = nullptr, *x2 = nullptr, *x3 = nullptr, *x4 = nullptr;  // n x m' blocks
  cplx* bt = nullptr;                    // conjugate-transposed block (tensor-core operand)
  cplx *g = nullptr, *yv = nullptr, *yw = nullptr, *rw = nullptr;  // m' x m'
  double *theta = nullptr, *dinv = nullptr;
  cplx* chol_inv = nullptr;
  int* flags = nullptr;
  unsigned long long* absmax = nullptr;
  HostReader reader;                     // small host reads outside the copy engines
  dense::HetrdWork hw32, hw64;
  dense::JacobiWork jw;
  // tensor-core workspace of the FP32 start's block products (planes of its own, so
  // that the projection's operand planes can be cut on the side stream meanwhile)
  tc::Workspace tw;
  bool has_tw = false;
  int max_n = 0, max_mp = 0;
  bool has32 = false;
  rpa_status alloc(int n_max, int mp_max, bool with32, std::string& err);
  void release();
  // lam_out[0 .. n_eig) and the column-major n x n_eig vec_out: the N_eig most
  // negative eigenpairs of the column-major view hc (n x n, Hermitian, not
  // modified).  a64: n x n complex128 scratch (may be vec_out).  mixed: a
  // mixed-precision plan (FP32 start where start32(); its block products on the
  // tensor cores where products_on_tc(), in the workspace tw).  RPA_ENUMERIC: a degenerate spectrum (a cluster of more than
  // 64 eigenvalues of T within 1e-10 of the largest, or no interval to filter):
  // the caller takes the library solver.
  rpa_status subspace(const cplx* hc, int n, int n_eig, double* lam_out, cplx* vec_out,
                      cplx* a64, bool mixed, cudaStream_t st, std::string& err, int* launches);
};

}  // namespace eig
}  // namespace rpa
