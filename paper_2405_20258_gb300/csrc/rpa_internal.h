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

// ---- FP64 SIMT contractions (rpa_fp64.cu) ---------------------------------

// chi[g][h] (+)= -(1/Omega) sum_vc conj(X[vc,g]) X[vc,h],  X = sf[vc] sv[g] A[vc,g].
// Upper block-triangle only.  accumulate: added to chi with FP64 atomics (chunks of
// a q-point's transitions; the caller zeroes chi first); else chi is overwritten.
cudaError_t launch_herk_fp64(const void* A, int a_dtype, int n_vc, int n_g, const double* sf,
                             const double* sv, double scale, cplx* chi, cudaStream_t st,
                             bool accumulate = false);

// mt[i][vc] (row stride ld_mt, n_vc when <= 0) = conj(sum_g A[vc][g] B[g][i]),
// B = [n_g][n_eig].
cudaError_t launch_project_fp64(const void* A, int a_dtype, int n_vc, int n_g, const cplx* B,
                                int n_eig, cplx* mt, cudaStream_t st, long ld_mt = 0);

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
// Transition order of the tensor-core chi~(0) K-blocks: order[pos] = the transitions
// by decreasing |ow| / |delta| (0 where either is 0), equal keys by index, on the
// device (bitonic sort).  nvb > 0: sorted within segments of nvb valence bands of one
// k-point (the chunks of a streamed q-point), as indices local to the segment.
// items: order_items(n) 16-byte items of scratch.  *launches += the kernels launched.
long order_items(long n);
cudaError_t launch_transition_order(const double* delta, const double* ow, long n, int n_v,
                                    int n_c, int nvb, void* items, int* order, cudaStream_t st,
                                    int* launches);
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
// part / n_parts: the transitions of A are piece `part` of n_parts (a q-point drawn
// in chunks): the sums accumulate in the scratch and the diagonal is written with
// the last piece.
cudaError_t launch_chi0_diagonal(const void* A, int dtype, long n_vc, int n_g, const double* sf0,
                                 const double* sv, double scale, double* scratch,
                                 size_t scratch_doubles, cplx* chi, cudaStream_t st,
                                 int part = 0, int n_parts = 1);
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

// Small device-to-host reads that bypass the copy engines: one kernel stores the pieces
// into mapped pinned host memory, then the stream is synchronised.  A copy-engine read
// (cudaMemcpyAsync to the host) can wait behind a large host-to-device copy that another
// stream has in flight, such as the next q-point's inputs.
struct HostReader {
  char* host = nullptr;  // pinned, mapped
  char* dev = nullptr;   // its device address
  size_t bytes = 0;
};
struct ReadPiece {
  const void* src;  // device
  void* dst;        // host
  size_t bytes;     // a multiple of 4
};
cudaError_t reader_alloc(HostReader& r, size_t bytes);
void reader_free(HostReader& r);
// Reads up to four pieces and synchronises st; pieces that do not fit the reader (or a
// reader never allocated) go through cudaMemcpyAsync instead.
cudaError_t read_to_host(HostReader& r, const ReadPiece* p, int n, cudaStream_t st);

}  // namespace rpa
