// Tiled FP64 Cholesky factorisation of a batch of Hermitian positive definite
// matrices, and the log-determinant ln det(1 - chi_s(i w_k)) = 2 sum_i ln L_ii of
// Eq. (rpaE) that the paper evaluates through a factorisation instead of
// eigenvalues (Implementation and GPU Optimization: Tr ln = ln det).
//
// GB300 issues about two FP64 FMAs per SM per clock, so the factorisation is
// arithmetic bound and must keep every SM busy.  It is right-looking over
// 32 x 32 tiles, three launches per tile column k, every launch batched over
// the matrices (gridDim.y):
//   potrf  one CTA per matrix factors the diagonal tile in shared memory,
//          adds its pivots' logarithms, and writes the inverse of that tile;
//   panel  one CTA per tile below the diagonal: L_ik = A_ik L_kk^-H, a small
//          product with the stored inverse;
//   update one CTA per tile of the trailing lower triangle:
//          A_ij -= L_ik L_jk^H (the O(n^3) part, ~all of the FMAs).
// Every thread of an update or panel CTA holds a 2 x 2 block of outputs.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "rpa_internal.h"

namespace rpa {
namespace {

constexpr int NB = 32;       // tile edge
constexpr int THREADS = 256;  // 16 x 16 threads, 2 x 2 outputs each

__device__ __forceinline__ cplx cmul_conj_acc(cplx acc, cplx a, cplx b) {
  // acc + a * conj(b)
  acc.re = fma(a.re, b.re, fma(a.im, b.im, acc.re));
  acc.im = fma(a.im, b.re, fma(-a.re, b.im, acc.im));
  return acc;
}

// work[b] = I - chis[b] on and below the diagonal (row-major n x n); logdet[b] = 0
__global__ void one_minus_kernel(const cplx* chis, int n, int batch, cplx* work,
                                 double* logdet) {
  const long per = (long)n * n, tot = per * batch;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot;
       e += (long)gridDim.x * blockDim.x) {
    if (e < batch && logdet) logdet[e] = 0.0;
    const long r = e % per;
    const int i = (int)(r / n), j = (int)(r % n);
    if (j > i) continue;
    const cplx v = chis[e];
    work[e] = cplx{(i == j ? 1.0 : 0.0) - v.re, i == j ? 0.0 : -v.im};
  }
}

// Factor the diagonal tile (k0, k0) of matrix blockIdx.x; inverse of L_kk to
// inv[b] (NB x NB row-major, zero above the diagonal).
__global__ void __launch_bounds__(THREADS) potrf_tile_kernel(cplx* a, int n, int k0, int kb,
                                                             cplx* inv, double* logdet,
                                                             int* bad) {
  __shared__ cplx t[NB][NB + 1];
  __shared__ cplx u[NB][NB + 1];
  __shared__ double piv[NB];
  __shared__ double rpiv;
  const int b = blockIdx.x, tid = threadIdx.x;
  cplx* m = a + (size_t)b * n * n;
  for (int e = tid; e < NB * NB; e += THREADS) {
    const int i = e / NB, j = e % NB;
    t[i][j] = (i < kb && j <= i) ? m[(size_t)(k0 + i) * n + k0 + j] : cplx{0.0, 0.0};
    u[i][j] = cplx{(i == j && i < kb) ? 1.0 : 0.0, 0.0};
  }
  __syncthreads();
  // Column j: the pivot, then column j of L and row j of X = L^-1 scaled by 1 / L_jj,
  // then the trailing update of the tile and X(j+1:, 0:j] -= L(j+1:, j) X(j, 0:j]
  // (forward elimination of the identity: X is final when the loop ends).
  for (int j = 0; j < kb; ++j) {
    if (tid == 0) {
      double d = t[j][j].re;
      if (!(d > 0.0) || !isfinite(d)) {
        atomicOr(bad, 16);
        d = 1.0;
      }
      const double pj = sqrt(d);
      piv[j] = pj;
      rpiv = 1.0 / pj;
      t[j][j] = cplx{pj, 0.0};
    }
    __syncthreads();
    const double rp = rpiv;
    if (tid > j && tid < kb) {
      t[tid][j].re *= rp;
      t[tid][j].im *= rp;
    } else if (tid >= NB && tid - NB <= j) {
      const int c = tid - NB;
      u[j][c].re *= rp;
      u[j][c].im *= rp;
    }
    __syncthreads();
    const int rem = kb - j - 1;
    for (int e = tid; e < rem * rem; e += THREADS) {
      const int i = j + 1 + e / rem, c = j + 1 + e % rem;
      if (c > i) continue;
      const cplx li = t[i][j], lc = t[c][j];
      // t[i][c] -= li conj(lc)
      t[i][c].re -= li.re * lc.re + li.im * lc.im;
      t[i][c].im -= li.im * lc.re - li.re * lc.im;
    }
    for (int e = tid; e < rem * (j + 1); e += THREADS) {
      const int i = j + 1 + e / (j + 1), c = e % (j + 1);
      const cplx l = t[i][j], x = u[j][c];
      u[i][c].re -= l.re * x.re - l.im * x.im;
      u[i][c].im -= l.re * x.im + l.im * x.re;
    }
    __syncthreads();
  }
  for (int e = tid; e < NB * NB; e += THREADS) {
    const int i = e / NB, j = e % NB;
    if (i < kb && j <= i) m[(size_t)(k0 + i) * n + k0 + j] = t[i][j];
    inv[(size_t)b * NB * NB + e] = u[i][j];
  }
  // 2 sum_j ln L_jj of this tile (the logarithms in parallel, summed in a fixed order)
  if (logdet && tid < 32) {
    double l = tid < kb ? 2.0 * log(piv[tid]) : 0.0;
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if (tid == 0) logdet[b] += l;
  }
}

// L_ik = A_ik L_kk^-H for the tiles below the diagonal tile: blockIdx.x = tile row
// below k0 + kb, blockIdx.y = matrix.
__global__ void __launch_bounds__(THREADS) panel_kernel(cplx* a, int n, int k0, int kb,
                                                        const cplx* inv) {
  __shared__ cplx sa[NB][NB + 1];
  __shared__ cplx su[NB][NB + 1];
  const int b = blockIdx.y, tid = threadIdx.x;
  const int i0 = k0 + kb + blockIdx.x * NB, ib = min(NB, n - i0);
  cplx* m = a + (size_t)b * n * n;
  for (int e = tid; e < NB * NB; e += THREADS) {
    const int r = e / NB, c = e % NB;
    sa[r][c] = (r < ib && c < kb) ? m[(size_t)(i0 + r) * n + k0 + c] : cplx{0.0, 0.0};
    su[r][c] = inv[(size_t)b * NB * NB + e];
  }
  __syncthreads();
  const int tx = tid % 16, ty = tid / 16;
  cplx acc[2][2] = {};
  // out[r][c] = sum_q A[r][q] conj(X[c][q]), X lower (q <= c)
  for (int q = 0; q < NB; ++q) {
    const cplx a0 = sa[2 * ty][q], a1 = sa[2 * ty + 1][q];
    const cplx x0 = su[2 * tx][q], x1 = su[2 * tx + 1][q];
    acc[0][0] = cmul_conj_acc(acc[0][0], a0, x0);
    acc[0][1] = cmul_conj_acc(acc[0][1], a0, x1);
    acc[1][0] = cmul_conj_acc(acc[1][0], a1, x0);
    acc[1][1] = cmul_conj_acc(acc[1][1], a1, x1);
  }
  for (int y = 0; y < 2; ++y)
    for (int x = 0; x < 2; ++x) {
      const int r = 2 * ty + y, c = 2 * tx + x;
      if (r < ib && c < kb) m[(size_t)(i0 + r) * n + k0 + c] = acc[y][x];
    }
}

// A_ij -= L_ik L_jk^H over the trailing lower triangle of tiles: blockIdx.x =
// linear index of tile (ti, tj), tj <= ti, blockIdx.y = matrix.
__global__ void __launch_bounds__(THREADS) update_kernel(cplx* a, int n, int k0, int kb) {
  __shared__ cplx si[NB][NB + 1];
  __shared__ cplx sj[NB][NB + 1];
  const int b = blockIdx.y, tid = threadIdx.x;
  const int l = blockIdx.x;
  int ti = (int)((sqrtf(8.0f * l + 1.0f) - 1.0f) * 0.5f);
  while ((ti + 1) * (ti + 2) / 2 <= l) ++ti;
  while (ti * (ti + 1) / 2 > l) --ti;
  const int tj = l - ti * (ti + 1) / 2;
  const int base = k0 + kb;
  const int i0 = base + ti * NB, j0 = base + tj * NB;
  const int ib = min(NB, n - i0), jb = min(NB, n - j0);
  cplx* m = a + (size_t)b * n * n;
  for (int e = tid; e < NB * NB; e += THREADS) {
    const int r = e / NB, q = e % NB;
    si[r][q] = (r < ib && q < kb) ? m[(size_t)(i0 + r) * n + k0 + q] : cplx{0.0, 0.0};
    sj[r][q] = (r < jb && q < kb) ? m[(size_t)(j0 + r) * n + k0 + q] : cplx{0.0, 0.0};
  }
  __syncthreads();
  const int tx = tid % 16, ty = tid / 16;
  cplx acc[2][2] = {};
  for (int q = 0; q < kb; ++q) {
    const cplx a0 = si[2 * ty][q], a1 = si[2 * ty + 1][q];
    const cplx b0 = sj[2 * tx][q], b1 = sj[2 * tx + 1][q];
    acc[0][0] = cmul_conj_acc(acc[0][0], a0, b0);
    acc[0][1] = cmul_conj_acc(acc[0][1], a0, b1);
    acc[1][0] = cmul_conj_acc(acc[1][0], a1, b0);
    acc[1][1] = cmul_conj_acc(acc[1][1], a1, b1);
  }
  for (int y = 0; y < 2; ++y)
    for (int x = 0; x < 2; ++x) {
      const int r = 2 * ty + y, c = 2 * tx + x;
      if (r >= ib || c >= jb) continue;
      if (ti == tj && c > r) continue;  // the diagonal tile's upper half is never read
      cplx& o = m[(size_t)(i0 + r) * n + j0 + c];
      o.re -= acc[y][x].re;
      o.im -= acc[y][x].im;
    }
}

}  // namespace

size_t cholesky_scratch_count(int batch) { return (size_t)batch * NB * NB; }

cudaError_t launch_cholesky_tiled(cplx* a, int n, int batch, double* logdet, int* bad, cplx* inv,
                                  cudaStream_t st, int* launches) {
  if (n < 1 || batch < 1) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  const int T = (n + NB - 1) / NB;
  int nl = 0;
  for (int k = 0; k < T; ++k) {
    const int k0 = k * NB, kb = std::min(NB, n - k0), rem = T - k - 1;
    potrf_tile_kernel<<<batch, THREADS, 0, st>>>(a, n, k0, kb, inv, logdet, bad);
    ++nl;
    if (rem > 0) {
      panel_kernel<<<dim3(rem, batch), THREADS, 0, st>>>(a, n, k0, kb, inv);
      update_kernel<<<dim3(rem * (rem + 1) / 2, batch), THREADS, 0, st>>>(a, n, k0, kb);
      nl += 2;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (launches) *launches += nl;
  return cudaSuccess;
}

cudaError_t launch_cholesky_logdet(cplx* work, const cplx* chis, int n, int batch,
                                   double* logdet, int* bad, cplx* inv, cudaStream_t st,
                                   int* launches) {
  const long tot = (long)n * n * batch;
  const int grid = (int)std::min<long>((tot + 255) / 256, 8192);
  one_minus_kernel<<<grid, 256, 0, st>>>(chis, n, batch, work, logdet);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (launches) *launches += 1;
  return launch_cholesky_tiled(work, n, batch, logdet, bad, inv, st, launches);
}

}  // namespace rpa
