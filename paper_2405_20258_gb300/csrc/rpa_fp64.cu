// FP64 SIMT contractions of the static-subspace RPA path.
//
// GB300 issues very few FP64 operations per clock (about 2 DFMA per SM per
// cycle), so these kernels are bound by the FP64 pipe, not by memory: a plain
// 64x64 shared-memory tile with a 4x4 complex register micro-tile per thread
// keeps the FP64 units busy.  They are the reference-precision path and the
// fallback for shapes the tensor-core path does not take.
#include <cuda_runtime.h>

#include "rpa_internal.h"

namespace rpa {
namespace {

constexpr int TILE = 64;
constexpr int BK = 16;
constexpr int NT = 256;  // 16 x 16 threads

__device__ __forceinline__ cplx load_c(const void* p, int dtype, size_t idx) {
  if (dtype == RPA_C64) {
    float2 v = reinterpret_cast<const float2*>(p)[idx];
    return {(double)v.x, (double)v.y};
  }
  double2 v = reinterpret_cast<const double2*>(p)[idx];
  return {v.x, v.y};
}

// Upper block-triangle enumeration: linear t -> (bi, bj), bi <= bj < nb.
__device__ __forceinline__ void tri_index(int t, int nb, int& bi, int& bj) {
  int r = 0;
  while (t >= nb - r) {
    t -= nb - r;
    ++r;
  }
  bi = r;
  bj = r + t;
}

// chi[g][h] = scale * sum_vc conj(X[vc][g]) X[vc][h],  X[vc][g] = sf[vc] sv[g] A[vc][g]
// Eq. (chi0_partial_occs) at w = 0 with the v^1/2 symmetrisation folded into X.
__global__ void __launch_bounds__(NT) herk_fp64_kernel(const void* __restrict__ A, int dtype,
                                                       int n_vc, int n_g,
                                                       const double* __restrict__ sf,
                                                       const double* __restrict__ sv, double scale,
                                                       cplx* __restrict__ chi, int nb, int kchunk,
                                                       int atomic) {
  __shared__ cplx Xg[BK][TILE + 1];
  __shared__ cplx Xh[BK][TILE + 1];
  int bi, bj;
  tri_index(blockIdx.x, nb, bi, bj);
  const int g0 = bi * TILE, h0 = bj * TILE;
  const int k0 = blockIdx.y * kchunk;
  const int k1 = min(n_vc, k0 + kchunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double ar[4][4], ai[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) ar[i][j] = ai[i][j] = 0.0;

  for (int kb = k0; kb < k1; kb += BK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int idx = threadIdx.x + NT * r;
      int kk = idx / TILE, c = idx % TILE;
      int vc = kb + kk;
      cplx a = {0.0, 0.0}, b = {0.0, 0.0};
      if (vc < k1) {
        double s = sf[vc];
        int g = g0 + c, h = h0 + c;
        if (g < n_g) {
          a = load_c(A, dtype, (size_t)vc * n_g + g);
          double w = s * sv[g];
          a.re *= w;
          a.im *= w;
        }
        if (h < n_g) {
          b = load_c(A, dtype, (size_t)vc * n_g + h);
          double w = s * sv[h];
          b.re *= w;
          b.im *= w;
        }
      }
      Xg[kk][c] = a;
      Xh[kk][c] = b;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      cplx x[4], y[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) x[i] = Xg[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) y[j] = Xh[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          // conj(x) * y
          ar[i][j] = fma(x[i].re, y[j].re, ar[i][j]);
          ar[i][j] = fma(x[i].im, y[j].im, ar[i][j]);
          ai[i][j] = fma(x[i].re, y[j].im, ai[i][j]);
          ai[i][j] = fma(-x[i].im, y[j].re, ai[i][j]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int g = g0 + ty + 16 * i, h = h0 + tx + 16 * j;
      if (g < n_g && h < n_g) {
        cplx* o = chi + (size_t)g * n_g + h;
        if (atomic) {
          atomicAdd(&o->re, scale * ar[i][j]);
          atomicAdd(&o->im, scale * ai[i][j]);
        } else {
          o->re = scale * ar[i][j];
          o->im = scale * ai[i][j];
        }
      }
    }
}

// mt[i][vc] = conj(sum_g A[vc][g] B[g][i])   (M~ = (A v^1/2 C)^H, B = v^1/2 C)
__global__ void __launch_bounds__(NT) project_fp64_kernel(const void* __restrict__ A, int dtype,
                                                          int n_vc, int n_g,
                                                          const cplx* __restrict__ B, int n_eig,
                                                          cplx* __restrict__ mt, long ld_mt) {
  __shared__ cplx As[BK][TILE + 1];
  __shared__ cplx Bs[BK][TILE + 1];
  const int vc0 = blockIdx.x * TILE, i0 = blockIdx.y * TILE;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double ar[4][4], ai[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) ar[a][b] = ai[a][b] = 0.0;
  for (int gb = 0; gb < n_g; gb += BK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int idx = threadIdx.x + NT * r;
      int row = idx / BK, kk = idx % BK;  // A tile: 64 vc rows x 16 g
      int vc = vc0 + row, g = gb + kk;
      cplx a = {0.0, 0.0};
      if (vc < n_vc && g < n_g) a = load_c(A, dtype, (size_t)vc * n_g + g);
      As[kk][row] = a;
      int kr = idx / TILE, col = idx % TILE;  // B tile: 16 g rows x 64 i
      int g2 = gb + kr, i = i0 + col;
      cplx b = {0.0, 0.0};
      if (g2 < n_g && i < n_eig) b = B[(size_t)g2 * n_eig + i];
      Bs[kr][col] = b;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      cplx x[4], y[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) x[a] = As[kk][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) y[b] = Bs[kk][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          ar[a][b] = fma(x[a].re, y[b].re, ar[a][b]);
          ar[a][b] = fma(-x[a].im, y[b].im, ar[a][b]);
          ai[a][b] = fma(x[a].re, y[b].im, ai[a][b]);
          ai[a][b] = fma(x[a].im, y[b].re, ai[a][b]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int vc = vc0 + tx + 16 * a, i = i0 + ty + 16 * b;
      if (vc < n_vc && i < n_eig) {
        cplx o = {ar[a][b], -ai[a][b]};
        mt[(size_t)i * ld_mt + vc] = o;
      }
    }
}

// chis[k][i][j] = scale sum_vc f_k(vc) mt[i][vc] conj(mt[j][vc]),  f_k = 4D/(D^2 + w_k^2)
// (chi0_s = M_s^+ Delta M_s of the Method section, one launch for every frequency).
__global__ void __launch_bounds__(NT) chis_fp64_kernel(const cplx* __restrict__ mt, int n_eig,
                                                       int n_vc, const double* __restrict__ delta,
                                                       const double* __restrict__ ow,
                                                       const double* __restrict__ omega,
                                                       int n_freq, double scale,
                                                       cplx* __restrict__ chis, int nb,
                                                       int split, int kchunk, int atomic) {
  __shared__ cplx Mi[BK][TILE + 1];
  __shared__ cplx Mj[BK][TILE + 1];
  __shared__ double fk[BK];
  int bi, bj;
  tri_index(blockIdx.x, nb, bi, bj);
  const int k = blockIdx.y / split, sidx = blockIdx.y % split;
  const int i0 = bi * TILE, j0 = bj * TILE;
  const int v0 = sidx * kchunk, v1 = min(n_vc, v0 + kchunk);
  const double w2 = omega[k] * omega[k];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double ar[4][4], ai[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) ar[a][b] = ai[a][b] = 0.0;
  for (int vb = v0; vb < v1; vb += BK) {
    if (threadIdx.x < BK) {
      int vc = vb + threadIdx.x;
      double d = vc < v1 ? delta[vc] : 1.0;
      double o = vc < v1 ? ow[vc] : 0.0;
      fk[threadIdx.x] = o != 0.0 ? o * (4.0 * d / (d * d + w2)) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int idx = threadIdx.x + NT * r;
      int row = idx / BK, kk = idx % BK;
      int vc = vb + kk;
      cplx a = {0.0, 0.0}, b = {0.0, 0.0};
      if (vc < v1) {
        if (i0 + row < n_eig) {
          a = mt[(size_t)(i0 + row) * n_vc + vc];
          a.re *= fk[kk];
          a.im *= fk[kk];
        }
        if (j0 + row < n_eig) b = mt[(size_t)(j0 + row) * n_vc + vc];
      }
      Mi[kk][row] = a;
      Mj[kk][row] = b;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      cplx x[4], y[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) x[a] = Mi[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) y[b] = Mj[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          // x * conj(y)
          ar[a][b] = fma(x[a].re, y[b].re, ar[a][b]);
          ar[a][b] = fma(x[a].im, y[b].im, ar[a][b]);
          ai[a][b] = fma(x[a].im, y[b].re, ai[a][b]);
          ai[a][b] = fma(-x[a].re, y[b].im, ai[a][b]);
        }
    }
    __syncthreads();
  }
  cplx* out = chis + (size_t)k * n_eig * n_eig;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
      if (i < n_eig && j < n_eig) {
        cplx* o = out + (size_t)i * n_eig + j;
        if (atomic) {
          atomicAdd(&o->re, scale * ar[a][b]);
          atomicAdd(&o->im, scale * ai[a][b]);
        } else {
          o->re = scale * ar[a][b];
          o->im = scale * ai[a][b];
        }
      }
    }
}

// Lower triangle := conj(upper), via a 32x32 shared-memory transpose per tile pair.
__global__ void mirror_kernel(cplx* __restrict__ m, int n, int nb) {
  __shared__ cplx t[32][33];
  int bi, bj;
  tri_index(blockIdx.x, nb, bi, bj);  // source tile (bi, bj) in the upper block triangle
  cplx* mat = m + (size_t)blockIdx.y * n * n;
  const int r0 = bi * 32, c0 = bj * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    int r = r0 + y, c = c0 + threadIdx.x;
    if (r < n && c < n) t[y][threadIdx.x] = mat[(size_t)r * n + c];
  }
  __syncthreads();
  // destination (c, r) for every r < c of the source
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    int r = r0 + threadIdx.x, c = c0 + y;  // write row c, column r
    if (r < n && c < n) {
      cplx v = t[threadIdx.x][y];
      if (c > r) {
        mat[(size_t)c * n + r] = {v.re, -v.im};
      } else if (c == r) {
        mat[(size_t)c * n + r] = {v.re, 0.0};
      }
    }
  }
}

inline int ceil_div(long a, long b) { return (int)((a + b - 1) / b); }

}  // namespace

cudaError_t launch_herk_fp64(const void* A, int a_dtype, int n_vc, int n_g, const double* sf,
                             const double* sv, double scale, cplx* chi, cudaStream_t st,
                             bool accumulate) {
  int nb = ceil_div(n_g, TILE);
  int tiles = nb * (nb + 1) / 2;
  // split the vc sum so that a few waves of blocks cover the GPU
  int want = 152 * 6;
  int split = tiles >= want ? 1 : ceil_div(want, tiles);
  int kchunk = ceil_div(ceil_div(n_vc, split), BK) * BK;
  split = ceil_div(n_vc, kchunk);
  if (split > 1 && !accumulate) {
    cudaError_t e = cudaMemsetAsync(chi, 0, sizeof(cplx) * (size_t)n_g * n_g, st);
    if (e != cudaSuccess) return e;
  }
  dim3 grid(tiles, split);
  herk_fp64_kernel<<<grid, NT, 0, st>>>(A, a_dtype, n_vc, n_g, sf, sv, scale, chi, nb, kchunk,
                                        split > 1 || accumulate);
  return cudaGetLastError();
}

cudaError_t launch_project_fp64(const void* A, int a_dtype, int n_vc, int n_g, const cplx* B,
                                int n_eig, cplx* mt, cudaStream_t st, long ld_mt) {
  dim3 grid(ceil_div(n_vc, TILE), ceil_div(n_eig, TILE));
  project_fp64_kernel<<<grid, NT, 0, st>>>(A, a_dtype, n_vc, n_g, B, n_eig, mt,
                                           ld_mt > 0 ? ld_mt : n_vc);
  return cudaGetLastError();
}

cudaError_t launch_chis_fp64(const cplx* mt, int n_eig, int n_vc, const double* delta,
                             const double* ow, const double* omega, int n_freq, double scale,
                             cplx* chis, cudaStream_t st) {
  int nb = ceil_div(n_eig, TILE);
  int tiles = nb * (nb + 1) / 2;
  int want = 152 * 6;
  int per = tiles * n_freq;
  int split = per >= want ? 1 : ceil_div(want, per);
  int kchunk = ceil_div(ceil_div(n_vc, split), BK) * BK;
  split = ceil_div(n_vc, kchunk);
  if (split > 1) {
    cudaError_t e =
        cudaMemsetAsync(chis, 0, sizeof(cplx) * (size_t)n_freq * n_eig * n_eig, st);
    if (e != cudaSuccess) return e;
  }
  dim3 grid(tiles, n_freq * split);
  chis_fp64_kernel<<<grid, NT, 0, st>>>(mt, n_eig, n_vc, delta, ow, omega, n_freq, scale, chis,
                                        nb, split, kchunk, split > 1);
  return cudaGetLastError();
}

cudaError_t launch_mirror_hermitian(cplx* m, int n, int batch, cudaStream_t st) {
  int nb = ceil_div(n, 32);
  dim3 grid(nb * (nb + 1) / 2, batch);
  mirror_kernel<<<grid, dim3(32, 8), 0, st>>>(m, n, nb);
  return cudaGetLastError();
}

}  // namespace rpa
