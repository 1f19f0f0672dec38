// Subspace of chi~(0) (step a3, Method: the N_eig eigenvectors of chi~(0) with the
// most negative eigenvalues), with this library's own kernels.
//
// GB300 issues about two FP64 FMAs per SM per clock, so a dense FP64 eigensolve
// of chi~ would dominate a q-point.  Its O(n^3) part, the Householder reduction
// to a real tridiagonal T, runs in FP32 on mixed-precision plans; everything
// after it keeps FP64 accuracy:
//   1. start: chi~ / max|chi~| in complex64 reduced to T = Q^H (chi~/max) Q
//      (rpa_dense.cu hetrd<float>; FP64 plans and small n: hetrd<double> of chi~);
//      the m' + 1 most negative eigenvalues of T by Sturm bisection (an FP32
//      phase, then FP64 from the FP32 bracket once FP64 counts confirm it) and
//      m' eigenvectors by FP64 inverse iteration (rpa_tridiag.h), back-transformed
//      by Q in the reduction's precision (compact WY blocks).  The reduction keeps
//      chi~'s graded structure, so these m' = N_eig + p vectors span chi~'s
//      leading subspace to ~1e-5 (FP32) -- provided T's own eigenpairs are FP64;
//   2. (FP32 start) a degree-3 Chebyshev polynomial of chi~ that damps the
//      interval of the unwanted eigenvalues [lambda_{m'+1}, 0] (scaled at
//      lambda_1, after Zhou and Saad 2007), applied to the m' vectors;
//   3. an orthonormal basis by column-scaled Cholesky-QR2 (tiled FP64 Cholesky of
//      the Gram matrix, its triangular inverse, the products on the tensor cores
//      or the FP64 pipe); a Cholesky that meets a non-positive pivot is repeated
//      with a shift of 1e-12 of the unit diagonal and followed by a third pass
//      (shifted Cholesky-QR3, Fukaya et al. 2020);
//   4. Rayleigh-Ritz: G = Q^H chi~ Q, its eigenpairs by cyclic Jacobi in FP64
//      (nearly diagonal here: a few sweeps, eigenvectors orthonormal to FP64
//      rounding), the N_eig Ritz vectors Q Y and values.
// p = max(64, N_eig/4) extra vectors put the unwanted eigenvalues that the filter
// must damp well below |lambda_{N_eig}| on these spectra (0.55 of it at N_eig =
// 400), so one filtered step gains ~10-200x.
// The matrix is used as the column-major view of the row-major chi~ buffer, i.e.
// conj(chi~): same eigenvalues, conjugated eigenvectors (undone by the gauge
// kernel).
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "rpa_eig.h"
#include "rpa_tridiag.h"

namespace rpa {
namespace eig {
namespace {

__device__ __forceinline__ void atomic_max_abs(unsigned long long* a, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

__global__ void absmax_kernel(const cplx* h, long n2, unsigned long long* out) {
  double m = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n2;
       i += (long)gridDim.x * blockDim.x)
    m = fmax(m, fmax(fabs(h[i].re), fabs(h[i].im)));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomic_max_abs(out, m);
}

// h32 = h / max|h| in complex64
__global__ void to_c64_kernel(const cplx* h, long n2, const unsigned long long* mx,
                              float2* h32) {
  const double m = __longlong_as_double((long long)*mx);
  const double s = m > 0.0 ? 1.0 / m : 1.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n2;
       i += (long)gridDim.x * blockDim.x)
    h32[i] = make_float2((float)(h[i].re * s), (float)(h[i].im * s));
}

// x[:, 0:cols] = v32[:, 0:cols] in complex128 (column-major, leading dimension n)
__global__ void to_c128_kernel(const float2* v32, long n, int cols, cplx* x) {
  const long tot = n * cols;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < tot;
       i += (long)gridDim.x * blockDim.x)
    x[i] = cplx{(double)v32[i].x, (double)v32[i].y};
}

// T in FP64 (an exact promotion of the FP32 reduction) and its squared
// off-diagonal in FP64 and in FP32
// A few host integers written to the device as kernel arguments (4 KB at most per
// launch), not by a host-to-device copy: such a copy queues on the copy engine
// behind whatever large input copy another stream has in flight.
constexpr long kInvitSmemMax = 227L * 1024;  // dynamic shared memory a block may opt into

struct IntBatch {
  int off, cnt;
  int v[1000];
};

__global__ void put_ints_kernel(IntBatch b, int* dst) {
  for (int i = threadIdx.x; i < b.cnt; i += blockDim.x) dst[b.off + i] = b.v[i];
}

__global__ void promote_tri_kernel(const float* d32, const float* e32, int n, double* d,
                                   double* e, double* e2, float* e2f) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    d[i] = (double)d32[i];
    if (i + 1 < n) {
      const double x = (double)e32[i];
      e[i] = x;
      e2[i] = x * x;
      e2f[i] = e32[i] * e32[i];
    }
  }
}

// w[j] for j < k: eigenvalue j (ascending) of T by Sturm bisection, a thread each.
// mode 0: FP64 throughout; 1: FP32 bisection finished in FP64; 2: FP32 only (to 4
// FP32 ulps of the eigenvalue: the FP32 reduction's T is itself an FP32 object, and
// the refinement that follows restores FP64 accuracy).
__global__ void bisect_kernel(const double* d, const double* e, const double* e2, const float* d32,
                              const float* e2f, int n, int k, int mode, double* w) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  double lo, hi, pivmin;
  tri::bounds(d, e, n, &lo, &hi, &pivmin);
  if (mode == 2) {
    float flo = (float)lo, fhi = (float)hi;
    tri::bisect_f(d32, e2f, n, j, &flo, &fhi);
    w[j] = 0.5 * ((double)flo + (double)fhi);
    return;
  }
  const double abstol = 1e-8 * DBL_EPSILON * fmax(fabs(lo), fabs(hi));
  w[j] = mode == 1 ? tri::bisect_mixed(d, e2, d32, e2f, n, j, lo, hi, pivmin, abstol)
                   : tri::bisect(d, e2, n, j, lo, hi, pivmin, abstol);
}

// The k most negative eigenvalues of T for the FP32 start, to 4 FP32 ulps of each: a
// warp per eigenvalue, whose lanes place 32 shifts evenly inside its bracket and take
// FP32 Sturm counts at all of them at once (multisection: five bits of the bracket per
// pass over T instead of one).  The first lane whose count exceeds j closes the
// bracket from above, the lane before it from below.  The Gershgorin bracket comes from
// the FP64 T, computed by the warp.
__global__ void bisect32_warp_kernel(const double* d, const double* e, const float* d32,
                                     const float* e2f, int n, int k, double* w) {
  const int j = (int)((blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= k) return;  // whole warps
  double l = d[0], h = d[0];
  for (int i = lane; i < n; i += 32) {
    const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
    l = fmin(l, d[i] - r);
    h = fmax(h, d[i] + r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    l = fmin(l, __shfl_xor_sync(0xffffffffu, l, o));
    h = fmax(h, __shfl_xor_sync(0xffffffffu, h, o));
  }
  const double wd = fmax(h - l, DBL_MIN);
  float flo = __double2float_rd(l - 2.0 * DBL_EPSILON * wd * n - DBL_MIN);
  float fhi = __double2float_ru(h + 2.0 * DBL_EPSILON * wd * n + DBL_MIN);
  const float fpiv = 1.1754944e-38f;  // FLT_MIN
  for (int it = 0; it < 32; ++it) {
    if (fhi - flo <= 4.0f * 1.1920929e-7f * fmaxf(fabsf(flo), fabsf(fhi))) break;
    const float x =
        fminf(fmaxf(flo + (fhi - flo) * ((float)(lane + 1) * (1.0f / 33.0f)), flo), fhi);
    const int cnt = tri::sturm_count_f(d32, e2f, n, x, fpiv);
    const unsigned above = __ballot_sync(0xffffffffu, cnt > j);
    float nlo = flo, nhi = fhi;
    if (above == 0u) {
      nlo = __shfl_sync(0xffffffffu, x, 31);
    } else {
      const int f = __ffs(above) - 1;
      nhi = __shfl_sync(0xffffffffu, x, f);
      const float prev = __shfl_sync(0xffffffffu, x, f > 0 ? f - 1 : 0);
      if (f > 0) nlo = prev;
    }
    if (!(nhi - nlo < fhi - flo)) break;  // no progress at FP32 resolution
    flo = nlo;
    fhi = nhi;
  }
  if (lane == 0) w[j] = 0.5 * ((double)flo + (double)fhi);
}

// Eigenvectors of T for the clusters c < nc of w (cluster c = w[first[c] ..
// first[c+1])), a thread each; z is n x ldz row-major; lanes holds 6 n nc doubles,
// element i of a thread's lane q at q n nc + i nc + c.
__global__ void invit_kernel(const double* d, const double* e, int n, const double* w,
                             const int* first, int nc, double* z, int ldz, double* lanes) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  double lo, hi, pivmin;
  tri::bounds(d, e, n, &lo, &hi, &pivmin);
  const double tiny = DBL_EPSILON * fmax(fabs(lo), fabs(hi));
  const long plane = (long)n * nc;
  double* b = lanes + c;
  tri::cluster_vectors(d, e, n, w, first[c], first[c + 1], tiny, z, ldz,
                       tri::Lane{b, nc}, tri::Lane{b + plane, nc}, tri::Lane{b + 2 * plane, nc},
                       tri::Lane{b + 3 * plane, nc}, tri::Lane{b + 4 * plane, nc},
                       tri::Lane{b + 5 * plane, nc});
}

// The same in FP32 arithmetic for the FP32 start, whose T (d32, e32) is itself an FP32
// object: its eigenvectors are wanted to FP32 accuracy only (the filtered
// Rayleigh-Ritz refinement restores FP64).  tiny: the pivot floor, FLT_EPSILON |T|;
// lanes holds 6 n nc floats.
__global__ void invit32_kernel(const float* d, const float* e, int n, const double* w,
                               const int* first, int nc, float tiny, double* z, int ldz,
                               float* lanes) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const long plane = (long)n * nc;
  float* b = lanes + c;
  using LF = tri::LaneT<float>;
  tri::cluster_vectors<float>(d, e, n, w, first[c], first[c + 1], tiny, z, ldz, LF{b, nc},
                              LF{b + plane, nc}, LF{b + 2 * plane, nc}, LF{b + 3 * plane, nc},
                              LF{b + 4 * plane, nc}, LF{b + 5 * plane, nc});
}

// The same with each thread's six lanes in shared memory (`per` clusters a block, one
// warp, lanes interleaved with stride `per`): the factor and the solves walk a chain
// of dependent steps over n rows, so a step's latency sets the time, and a load from
// shared memory returns in a few tens of cycles where one that follows the thread's
// own global store to the same lanes goes to L2.  Same arithmetic, same results.
__global__ void invit32_smem_kernel(const float* d, const float* e, int n, const double* w,
                                    const int* first, int nc, float tiny, double* z, int ldz,
                                    int per) {
  extern __shared__ float lane_sm[];
  const int c = blockIdx.x * per + threadIdx.x;
  if (threadIdx.x >= per || c >= nc) return;
  const long plane = (long)n * per;
  float* b = lane_sm + threadIdx.x;
  using LF = tri::LaneT<float>;
  tri::cluster_vectors<float>(d, e, n, w, first[c], first[c + 1], tiny, z, ldz, LF{b, per},
                              LF{b + plane, per}, LF{b + 2 * plane, per}, LF{b + 3 * plane, per},
                              LF{b + 4 * plane, per}, LF{b + 5 * plane, per});
}

// c[i + n j] = z[i k + j] as complex64 (column-major n x k from row-major FP64)
__global__ void z_to_c64_kernel(const double* z, int n, int k, float2* c) {
  const long tot = (long)n * k;
  for (long o = blockIdx.x * (long)blockDim.x + threadIdx.x; o < tot;
       o += (long)gridDim.x * blockDim.x) {
    const long i = o % n, j = o / n;
    c[o] = make_float2((float)z[i * k + j], 0.f);
  }
}

// dinv[j] = 1 / ||x[:, j]|| in FP64 (1 for a zero column); one 256-thread block per
// column of the column-major n x cols block, grid = cols
__global__ void inv_colnorm_kernel(const cplx* x, int n, int cols, double* dinv) {
  __shared__ double red[8];
  const int j = blockIdx.x;
  if (j >= cols) return;  // whole blocks only
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const cplx v = x[(long)j * n + i];
    s += v.re * v.re + v.im * v.im;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    dinv[j] = t > 0.0 ? 1.0 / sqrt(t) : 1.0;
  }
}

// x[:, j] *= dinv[j]
__global__ void scale_cols_kernel(cplx* x, int n, int cols, const double* dinv) {
  const long tot = (long)n * cols;
  for (long o = blockIdx.x * (long)blockDim.x + threadIdx.x; o < tot;
       o += (long)gridDim.x * blockDim.x) {
    const double f = dinv[o / n];
    x[o].re *= f;
    x[o].im *= f;
  }
}

// zero the strictly lower triangle of the column-major m x m matrix g
__global__ void zero_lower_kernel(cplx* g, int m) {
  const long tot = (long)m * m;
  for (long o = blockIdx.x * (long)blockDim.x + threadIdx.x; o < tot;
       o += (long)gridDim.x * blockDim.x)
    if (o % m > o / m) g[o] = cplx{0.0, 0.0};
}


// T of the FP64 start: e^2 in FP64 and FP32, and FP32 copies of d (the FP32
// bisection phase)
__global__ void promote64_kernel(const double* d, const double* e, int n, double* e2, float* e2f,
                                 float* d32) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    d32[i] = (float)d[i];
    if (i + 1 < n) {
      e2[i] = e[i] * e[i];
      e2f[i] = (float)e2[i];
    }
  }
}

// x[i + n j] = z[i k + j] as complex128 (column-major n x k from row-major FP64)
__global__ void z_to_c128_kernel(const double* z, int n, int k, cplx* x) {
  const long tot = (long)n * k;
  for (long o = blockIdx.x * (long)blockDim.x + threadIdx.x; o < tot;
       o += (long)gridDim.x * blockDim.x) {
    const long i = o % n, j = o / n;
    x[o] = cplx{z[i * k + j], 0.0};
  }
}

// out (cols x rows, column-major) = X^H for the column-major rows x cols X, through
// 32 x 32 shared-memory tiles
__global__ void ctrans_kernel(const cplx* x, int rows, int cols, cplx* out) {
  __shared__ cplx t[32][33];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  for (int jj = threadIdx.y; jj < 32; jj += blockDim.y) {
    const int i = i0 + threadIdx.x, j = j0 + jj;
    if (i < rows && j < cols) t[jj][threadIdx.x] = x[(size_t)j * rows + i];
  }
  __syncthreads();
  for (int ii = threadIdx.y; ii < 32; ii += blockDim.y) {
    const int j = j0 + threadIdx.x, i = i0 + ii;
    if (i < rows && j < cols) {
      const cplx v = t[threadIdx.x][ii];
      out[(size_t)i * cols + j] = cplx{v.re, -v.im};
    }
  }
}

// out = a x + b y (real scalars), count elements
__global__ void axpby_kernel(long count, double a, const cplx* x, double b, const cplx* y,
                             cplx* out) {
  for (long o = blockIdx.x * (long)blockDim.x + threadIdx.x; o < count;
       o += (long)gridDim.x * blockDim.x) {
    const cplx u = x[o], v = y[o];
    out[o] = cplx{a * u.re + b * v.re, a * u.im + b * v.im};
  }
}

// g = (g + g^H) / 2 for the column-major m x m g, one thread per pair i <= j
__global__ void hermitise_kernel(cplx* g, int m) {
  const long tot = (long)m * m;
  for (long o = blockIdx.x * (long)blockDim.x + threadIdx.x; o < tot;
       o += (long)gridDim.x * blockDim.x) {
    const int i = (int)(o % m), j = (int)(o / m);
    if (i > j) continue;
    const cplx a = g[(size_t)j * m + i], b = g[(size_t)i * m + j];
    const cplx h = {0.5 * (a.re + b.re), 0.5 * (a.im - b.im)};
    g[(size_t)j * m + i] = h;
    g[(size_t)i * m + j] = cplx{h.re, -h.im};
  }
}

// g += s I
__global__ void add_diag_kernel(cplx* g, int m, double s) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    g[(size_t)i * m + i].re += s;
}

// widest cluster of T's eigenvalues re-orthogonalised by one thread
constexpr int kMaxCluster = 64;
// smallest n that takes the FP32 start
constexpr int kMinStart32 = 1024;

int grid_for(long n, int block) { return (int)std::min<long>((n + block - 1) / block, 4096); }

}  // namespace

int extra_vectors(int n_eig) { return std::max(64, n_eig / 4); }

int block_size(int n, int n_eig) { return std::min(n, n_eig + extra_vectors(n_eig)); }

bool start32(int n, int n_eig) {
  const char* e = getenv("RPA_EIG_START32");
  if (e && e[0] == '0') return false;
  return n >= kMinStart32 && block_size(n, n_eig) < n;
}

bool products_on_tc() {
  const char* e = getenv("RPA_EIG_TC");
  return !(e && e[0] == '0');
}

bool use_library() {
  const char* e = getenv("RPA_EIG");
  return e && strcmp(e, "cusolver") == 0;
}

rpa_status Refine::alloc(int n_max, int mp_max, bool with32, std::string& err) {
  max_n = n_max;
  max_mp = mp_max;
  has32 = with32;
  auto al = [&](void** p, size_t bytes) {
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      (void)cudaGetLastError();
      err = "eigensolver workspace: cudaMalloc of " + std::to_string(bytes) + " bytes";
      return false;
    }
    return true;
  };
  const size_t n = (size_t)n_max, mp = (size_t)mp_max, nblk = (n + 31) / 32;
  bool ok = true;
  if (with32)
    ok = al((void**)&h32, n * n * sizeof(float2)) && al((void**)&d32, n * sizeof(float)) &&
         al((void**)&e32, n * sizeof(float)) && al((void**)&tau32, n * sizeof(float2)) &&
         al((void**)&c32, n * mp * sizeof(float2));
  ok = ok && al((void**)&tau64, n * sizeof(cplx)) && al((void**)&d64, n * sizeof(double)) &&
       al((void**)&e64, n * sizeof(double)) && al((void**)&e2, n * sizeof(double)) &&
       al((void**)&e2f, n * sizeof(float)) && al((void**)&d32b, n * sizeof(float)) &&
       al((void**)&wt, (mp + 1) * sizeof(double)) && al((void**)&first, (mp + 2) * sizeof(int)) &&
       al((void**)&zt, n * mp * sizeof(double)) && al((void**)&lanes, 6 * n * mp * sizeof(double)) &&
       al(&tfac, nblk * 32 * 32 * sizeof(cplx)) && al((void**)&x0, n * mp * sizeof(cplx)) &&
       al((void**)&x1, n * mp * sizeof(cplx)) && al((void**)&x2, n * mp * sizeof(cplx)) &&
       al((void**)&x3, n * mp * sizeof(cplx)) && al((void**)&x4, n * mp * sizeof(cplx)) &&
       al((void**)&bt, n * mp * sizeof(cplx)) && al((void**)&g, mp * mp * sizeof(cplx)) &&
       al((void**)&yv, mp * mp * sizeof(cplx)) && al((void**)&yw, mp * mp * sizeof(cplx)) &&
       al((void**)&rw, mp * mp * sizeof(cplx)) && al((void**)&theta, mp * sizeof(double)) &&
       al((void**)&dinv, mp * sizeof(double)) &&
       al((void**)&chol_inv, cholesky_scratch_count(1) * sizeof(cplx)) &&
       al((void**)&flags, 4 * sizeof(int)) &&
       al((void**)&absmax, sizeof(unsigned long long));
  if (!ok) {
    release();
    return RPA_ENOMEM;
  }
  rpa_status s = RPA_OK;
  if (with32) s = dense::hetrd_alloc(hw32, n_max, sizeof(float2), err);
  if (s == RPA_OK && with32 && products_on_tc()) {
    tc::Slices sl;
    sl.chi0 = 1;
    sl.proj = tc::EIG_SLICES;
    sl.chis = 1;
    // rows up to n (chi~ and the blocks), K up to 2n, columns up to m'
    s = tc::alloc_workspace(tw, n, mp, n, 1, sl, err);
    has_tw = s == RPA_OK;
  }
  if (s == RPA_OK) s = dense::hetrd_alloc(hw64, n_max, sizeof(cplx), err);
  if (s == RPA_OK) s = dense::jacobi_alloc(jw, mp_max, err);
  // host reads of the eigenvalues of T (m' + 1), the Ritz values and a few flags
  if (s == RPA_OK && reader_alloc(reader, (mp + 2) * sizeof(double) + 64) != cudaSuccess) {
    (void)cudaGetLastError();
    err = "eigensolver: mapped host buffer";
    s = RPA_ENOMEM;
  }
  if (s != RPA_OK) {
    release();
    return s;
  }
  return RPA_OK;
}

void Refine::release() {
  void* b[] = {h32, d32,   e32, tau32, c32, tau64, d64, e64, e2, e2f, d32b, wt, first, zt,
               lanes, tfac, x0, x1,   x2,  x3,    x4,  bt,  g,   yv,  yw, rw,  theta, dinv, chol_inv,
               flags, absmax};
  for (void* p : b)
    if (p) cudaFree(p);
  dense::hetrd_free(hw32);
  dense::hetrd_free(hw64);
  dense::jacobi_free(jw);
  if (has_tw) tc::free_workspace(tw);
  reader_free(reader);
  *this = Refine{};
}

#define CU_E(call)                                                       \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) {                                             \
      err = std::string(#call ": ") + cudaGetErrorString(e_);            \
      return RPA_ECUDA;                                                  \
    }                                                                    \
  } while (0)
#define RS_E(call)                 \
  do {                             \
    rpa_status r_ = (call);        \
    if (r_ != RPA_OK) return r_;   \
  } while (0)

rpa_status Refine::subspace(const cplx* hc, int n, int n_eig, double* lam_out, cplx* vec_out,
                            cplx* a64, bool mixed, cudaStream_t st, std::string& err,
                            int* launches) {
  const int mp = block_size(n, n_eig);
  const bool s32 = mixed && has32 && start32(n, n_eig);
  if (n > max_n || mp > max_mp) {
    err = "eigensolver: shape outside its workspace";
    return RPA_EINVAL;
  }
  const long n2 = (long)n * n;
  int nl = 0;
  // 1. tridiagonal start and its FP64 eigenpairs
  CU_E(cudaMemsetAsync(flags, 0, 4 * sizeof(int), st));
  CU_E(cudaMemsetAsync(absmax, 0, sizeof(unsigned long long), st));
  if (s32) {
    absmax_kernel<<<grid_for(n2, 256), 256, 0, st>>>(hc, n2, absmax);
    to_c64_kernel<<<grid_for(n2, 256), 256, 0, st>>>(hc, n2, absmax, h32);
    CU_E(cudaGetLastError());
    RS_E(dense::hetrd<float>(hw32, h32, n, d32, e32, tau32, st, err, &nl));
    promote_tri_kernel<<<grid_for(n, 256), 256, 0, st>>>(d32, e32, n, d64, e64, e2, e2f);
    CU_E(cudaGetLastError());
    nl += 3;
  } else {
    CU_E(cudaMemcpyAsync(a64, hc, sizeof(cplx) * n2, cudaMemcpyDeviceToDevice, st));
    RS_E(dense::hetrd<double>(hw64, a64, n, d64, e64, tau64, st, err, &nl));
    promote64_kernel<<<grid_for(n, 256), 256, 0, st>>>(d64, e64, n, e2, e2f, d32b);
    CU_E(cudaGetLastError());
    nl += 1;
  }
  //    the m' (+ 1 for the filter's bound) most negative eigenvalues of T
  //    (RPA_EIG_BISECT32=0: without the FP32 phase; RPA_EIG_BISECT_BLOCK threads a
  //    block, 32 by default, a multiple of 32 at most 256)
  const int nval = mp < n ? mp + 1 : mp;
  //    The FP32 start takes FP32 bisection only (RPA_EIG_BISECT64=1: finished in FP64);
  //    the FP64 start FP32 bisection finished in FP64 (RPA_EIG_BISECT32=0: FP64 only).
  const char* b32_env = getenv("RPA_EIG_BISECT32");
  const char* b64_env = getenv("RPA_EIG_BISECT64");
  const char* blk_env = getenv("RPA_EIG_BISECT_BLOCK");
  int mode = (b32_env && b32_env[0] == '0') ? 0 : 1;
  if (s32 && !(b64_env && b64_env[0] == '1')) mode = 2;
  const int bb = std::max(1, std::min(256, blk_env ? atoi(blk_env) : 32));
  if (mode == 2)
    bisect32_warp_kernel<<<(nval + 3) / 4, 128, 0, st>>>(d64, e64, d32, e2f, n, nval, wt);
  else
    bisect_kernel<<<(nval + bb - 1) / bb, bb, 0, st>>>(d64, e64, e2, s32 ? d32 : d32b, e2f, n,
                                                       nval, mode, wt);
  CU_E(cudaGetLastError());
  nl += 1;
  std::vector<double> w(nval);
  unsigned long long mx_bits = 0;
  int hst = 0;
  {
    const ReadPiece rp[3] = {{wt, w.data(), nval * sizeof(double)},
                             {absmax, &mx_bits, sizeof mx_bits},
                             {s32 ? hw32.status : hw64.status, &hst, sizeof(int)}};
    CU_E(read_to_host(reader, rp, 3, st));
  }
  if (launches) *launches += nl;
  nl = 0;
  if (hst != 0) {
    CU_E(cudaMemset(s32 ? hw32.status : hw64.status, 0, sizeof(int)));
    err = "eigensolver: a barrier of the tridiagonal reduction gave up waiting";
    return RPA_ETIMEOUT;
  }
  double mx = 1.0;
  if (s32) {
    memcpy(&mx, &mx_bits, sizeof mx);
    if (!(mx > 0.0)) mx = 1.0;
  }
  //    T's eigenvectors for the first m' (inverse iteration, re-orthogonalised within
  //    clusters of eigenvalues closer than 1e-10 of the largest), then Q applied
  const double tnorm = std::max(std::fabs(w[0]), std::fabs(w[nval - 1]));
  if (!(tnorm > 0.0) || !std::isfinite(tnorm)) {
    err = "eigensolver: degenerate tridiagonal spectrum";
    return RPA_ENUMERIC;
  }
  std::vector<int> fh(mp + 1);
  int nc = 0;
  if (mode == 2) {
    // FP32 eigenvalues: a new cluster where the gap exceeds 1e-5 of the eigenvalue,
    // well above the bisection's 4 FP32 ulps (inverse iteration with shifts closer
    // than their errors would return one vector twice)
    for (int j = 0; j < mp; ++j)
      if (j == 0 || w[j] - w[j - 1] > 1e-5 * std::max(std::fabs(w[j]), std::fabs(w[j - 1])))
        fh[nc++] = j;
    fh[nc] = mp;
  } else {
    nc = tri::clusters(w.data(), mp, 1e-10 * tnorm, fh.data());
  }
  int widest = 0;
  for (int c = 0; c < nc; ++c) widest = std::max(widest, fh[c + 1] - fh[c]);
  if (widest > kMaxCluster) {
    err = "eigensolver: a cluster of " + std::to_string(widest) + " eigenvalues";
    return RPA_ENUMERIC;
  }
  for (int o = 0; o <= nc; o += 1000) {
    IntBatch b;
    b.off = o;
    b.cnt = std::min(1000, nc + 1 - o);
    std::copy(fh.begin() + o, fh.begin() + o + b.cnt, b.v);
    put_ints_kernel<<<1, 256, 0, st>>>(b, first);
    nl += 1;
  }
  const char* ib_env = getenv("RPA_EIG_INVIT_BLOCK");
  const int ib = std::max(1, std::min(256, ib_env ? atoi(ib_env) : 32));
  // shared-memory lanes: two clusters a block where 6 n floats each fit twice in 227 KB,
  // one where they fit once (RPA_EIG_INVIT_SMEM=0: lanes in global memory)
  const char* sm_env = getenv("RPA_EIG_INVIT_SMEM");
  const long lane_bytes = 6L * n * (long)sizeof(float);
  const int per = (sm_env && sm_env[0] == '0') ? 0
                  : 2 * lane_bytes <= kInvitSmemMax ? 2 : lane_bytes <= kInvitSmemMax ? 1 : 0;
  if (mode == 2 && per > 0) {
    const size_t smem = (size_t)per * lane_bytes;
    CU_E(cudaFuncSetAttribute(invit32_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem));
    invit32_smem_kernel<<<(nc + per - 1) / per, 32, smem, st>>>(
        d32, e32, n, wt, first, nc, (float)(FLT_EPSILON * tnorm), zt, mp, per);
  } else if (mode == 2)
    invit32_kernel<<<(nc + ib - 1) / ib, ib, 0, st>>>(d32, e32, n, wt, first, nc,
                                                      (float)(FLT_EPSILON * tnorm), zt, mp,
                                                      (float*)lanes);
  else
    invit_kernel<<<(nc + ib - 1) / ib, ib, 0, st>>>(d64, e64, n, wt, first, nc, zt, mp, lanes);
  CU_E(cudaGetLastError());
  if (s32) {
    z_to_c64_kernel<<<grid_for((long)n * mp, 256), 256, 0, st>>>(zt, n, mp, c32);
    CU_E(cudaGetLastError());
    RS_E(dense::apply_q<float>(h32, tau32, n, c32, mp, tfac, st, err, &nl));
    to_c128_kernel<<<grid_for((long)n * mp, 256), 256, 0, st>>>(c32, n, mp, x0);
  } else {
    z_to_c128_kernel<<<grid_for((long)n * mp, 256), 256, 0, st>>>(zt, n, mp, x0);
    CU_E(cudaGetLastError());
    RS_E(dense::apply_q<double>(a64, tau64, n, x0, mp, tfac, st, err, &nl));
  }
  CU_E(cudaGetLastError());
  nl += 3;

  // Block products.  On the tensor cores (FP32 start, unless RPA_EIG_TC=0) they use
  // the projection GEMM, which for a row-major A [rows][K] and a row-major B
  // [K][cols] writes out[c][r] = conj(sum_k A[r][k] B[k][c]), i.e. the column-major
  // rows x cols matrix conj(A B), with the projection's digit slices (6 by
  // default: products exact to ~2^-47 of the row and column scales); a column-major
  // X enters as the row-major conj(X) through a conjugate transpose.  Otherwise
  // they run on the FP64 pipe (dense::gemm_z).
  const bool on_tc = s32 && has_tw && products_on_tc();
  const cplx one = {1.0, 0.0}, zero = {0.0, 0.0};
  auto ctrans = [&](const cplx* x, int rows, int cols, cplx* out) -> rpa_status {
    ctrans_kernel<<<dim3((rows + 31) / 32, (cols + 31) / 32), dim3(32, 8), 0, st>>>(x, rows, cols,
                                                                                   out);
    CU_E(cudaGetLastError());
    ++nl;
    return RPA_OK;
  };
  auto tc_gemm = [&](const cplx* a_rm, int rows, int k, const cplx* b_rm, int cols,
                     cplx* out) -> rpa_status {
    // exact digits with EIG_SLICES planes, in the eigensolver's own workspace
    int l = 0;
    const rpa_status r = tc::project(tw, a_rm, RPA_C128, rows, k, b_rm, cols, out, st, err, &l);
    nl += l;
    return r;
  };
  // Y = H X (n x m')
  auto hx = [&](const cplx* X, cplx* Y) -> rpa_status {
    if (!on_tc) return dense::gemm_z('N', 'N', n, mp, n, one, hc, n, X, n, zero, Y, n, st, err, &nl);
    RS_E(ctrans(X, n, mp, bt));
    return tc_gemm(hc, n, n, bt, mp, Y);
  };
  // G = Q^H Z (m' x m')
  auto qhz = [&](const cplx* Q, const cplx* Z, cplx* G) -> rpa_status {
    if (!on_tc)
      return dense::gemm_z('C', 'N', mp, mp, n, one, Q, n, Z, n, zero, G, mp, st, err, &nl);
    RS_E(ctrans(Q, n, mp, bt));
    return tc_gemm(Z, mp, n, bt, mp, G);
  };
  // U = Q Y[:, 0:cols] (n x cols, Y m' x m')
  auto qy = [&](const cplx* Q, const cplx* Y, int cols, cplx* U) -> rpa_status {
    if (!on_tc)
      return dense::gemm_z('N', 'N', n, cols, mp, one, Q, n, Y, mp, zero, U, n, st, err, &nl);
    RS_E(ctrans(Q, n, mp, bt));
    RS_E(ctrans(Y, mp, cols, rw));
    return tc_gemm(bt, n, mp, rw, cols, U);
  };
  auto axpby = [&](cplx* out, double a, const cplx* x, double b, const cplx* y) -> rpa_status {
    axpby_kernel<<<grid_for((long)n * mp, 256), 256, 0, st>>>((long)n * mp, a, x, b, y, out);
    CU_E(cudaGetLastError());
    ++nl;
    return RPA_OK;
  };

  // One column-scaled Cholesky-QR pass: Y <- Y D^-1 R^-1 with D = diag ||y_j|| and
  // G = (Y D^-1)^H (Y D^-1) = R^H R (tiled FP64 Cholesky; the row-major lower factor
  // of the column-major G buffer is the column-major upper R).  A non-positive pivot
  // repeats the factorisation with G + 1e-12 I (*shifted is set: one more pass is
  // due).  With a companion block P, the same basis change P <- P D^-1 R^-1 is
  // applied to it.  Y and spare (P and pspare) are swapped as the products go.
  auto qr_pass = [&](cplx*& Y, cplx*& spare, cplx** P, cplx** pspare, bool* shifted) -> rpa_status {
    inv_colnorm_kernel<<<mp, 256, 0, st>>>(Y, n, mp, dinv);
    scale_cols_kernel<<<grid_for((long)n * mp, 256), 256, 0, st>>>(Y, n, mp, dinv);
    if (P) scale_cols_kernel<<<grid_for((long)n * mp, 256), 256, 0, st>>>(*P, n, mp, dinv);
    CU_E(cudaGetLastError());
    nl += P ? 3 : 2;
    for (int attempt = 0; attempt < 2; ++attempt) {
      RS_E(qhz(Y, Y, g));
      if (attempt == 1) {
        add_diag_kernel<<<grid_for(mp, 256), 256, 0, st>>>(g, mp, 1e-12);
        CU_E(cudaGetLastError());
        ++nl;
      }
      CU_E(cudaMemsetAsync(flags, 0, sizeof(int), st));
      CU_E(launch_cholesky_tiled(g, mp, 1, nullptr, flags, chol_inv, st, &nl));
      int bad = 0;
      const ReadPiece rp = {flags, &bad, sizeof(int)};
      CU_E(read_to_host(reader, &rp, 1, st));
      if (bad == 0) break;
      if (attempt == 1) {
        err = "eigensolver: Cholesky-QR of the block failed with a shift";
        return RPA_EEIG;
      }
      if (shifted) *shifted = true;
    }
    zero_lower_kernel<<<grid_for((long)mp * mp, 256), 256, 0, st>>>(g, mp);
    CU_E(cudaGetLastError());
    ++nl;
    RS_E(dense::trinv_upper(g, mp, mp, yw, st, err, &nl));
    RS_E(qy(Y, g, mp, spare));  // Y R^-1
    std::swap(Y, spare);
    if (P) {
      RS_E(qy(*P, g, mp, *pspare));
      std::swap(*P, *pspare);
    }
    return RPA_OK;
  };

  // 2.-4. RPA_EIG_STEPS (default 1, at most 8) filtered Rayleigh-Ritz steps (FP32
  //    start; the FP64 start takes one Rayleigh-Ritz step).  A step applies the
  //    degree-3 Chebyshev polynomial that damps [a, 0] -- a = lambda_{m'+1} of T
  //    first, the largest Ritz value of the block after that -- scaled at lambda_1,
  //    by its three-term recurrence.  On these graded spectra one product raises
  //    the weight of lambda_1's direction against that of lambda_{N_eig} by ~1e5,
  //    so after every product the new block is orthonormalised (one Cholesky-QR
  //    pass) and the previous block takes the same basis change: the pair stays a
  //    consistent basis of the recurrence, p(H) X_0 M for an invertible M, and no
  //    block is ever far from orthonormal.  A final pass makes the filtered block
  //    orthonormal to FP64 rounding; then G = Q^H H Q, its eigenpairs (Jacobi) and
  //    the Ritz vectors.
  const char* steps_env = getenv("RPA_EIG_STEPS");
  const int steps = s32 ? std::max(1, std::min(8, steps_env ? atoi(steps_env) : 1)) : 1;
  double a = nval > mp ? w[mp] * mx : 0.0, lo = w[0] * mx;
  const double b = 0.0;
  cplx* bufs[5] = {x0, x1, x2, x3, x4};
  cplx* xs = x0;  // the block the next step starts from
  for (int step = 0; step < steps; ++step) {
    // free buffers other than xs
    cplx* fr[4];
    int nf = 0;
    for (cplx* bp : bufs)
      if (bp != xs) fr[nf++] = bp;
    cplx *xm = xs, *xk = fr[0], *xn = fr[1], *sp = fr[2], *sp2 = fr[3];
    bool shifted = false;
    if (s32) {
      if (!(a < 0.0) || !(lo < a)) {
        err = "eigensolver: degenerate spectrum bounds";
        return RPA_ENUMERIC;
      }
      const double e = 0.5 * (b - a), c = 0.5 * (b + a);
      double sigma = e / (lo - c);
      const double tau2 = 2.0 / sigma;
      // X_1 = (sigma / e) (H - c) X_0
      RS_E(hx(xm, xk));
      RS_E(axpby(xk, sigma / e, xk, -c * sigma / e, xm));
      RS_E(qr_pass(xk, sp, &xm, &sp2, &shifted));
      for (int k = 2; k <= 3; ++k) {
        const double s1 = 1.0 / (tau2 - sigma);
        // X_{k+1} = (2 s1 / e) (H - c) X_k - sigma s1 X_{k-1}
        RS_E(hx(xk, xn));
        RS_E(axpby(xn, 2.0 * s1 / e, xn, -2.0 * s1 * c / e, xk));
        RS_E(axpby(xn, 1.0, xn, -sigma * s1, xm));
        RS_E(qr_pass(xn, sp, k < 3 ? &xk : nullptr, &sp2, &shifted));
        std::swap(xm, xk);  // X_{k-1} <- X_k
        std::swap(xk, xn);  // X_k <- X_{k+1}; xn holds the oldest block (free)
        sigma = s1;
      }
    } else {
      std::swap(xm, xk);  // the start itself (in xk)
      RS_E(qr_pass(xk, sp, nullptr, nullptr, &shifted));
    }
    // the block orthonormal to FP64 rounding (in xk; xm, xn free)
    RS_E(qr_pass(xk, sp, nullptr, nullptr, &shifted));
    if (shifted) RS_E(qr_pass(xk, sp, nullptr, nullptr, nullptr));
    // Rayleigh-Ritz: G = Q^H (H Q), G = Y Theta Y^H
    RS_E(hx(xk, xn));
    RS_E(qhz(xk, xn, g));
    hermitise_kernel<<<grid_for((long)mp * mp, 256), 256, 0, st>>>(g, mp);
    CU_E(cudaGetLastError());
    ++nl;
    RS_E(dense::jacobi(jw, g, mp, theta, yv, yw, st, err, &nl));
    if (step + 1 < steps) {
      RS_E(qy(xk, yv, mp, xn));
      std::vector<double> th(mp);
      const ReadPiece rp = {theta, th.data(), sizeof(double) * mp};
      CU_E(read_to_host(reader, &rp, 1, st));
      a = th[mp - 1];
      lo = th[0];
      xs = xn;
      continue;
    }
    // the N_eig Ritz pairs: U = Q Y[:, 0:N_eig]
    RS_E(qy(xk, yv, n_eig, vec_out));
    CU_E(cudaMemcpyAsync(lam_out, theta, sizeof(double) * n_eig, cudaMemcpyDeviceToDevice, st));
  }
  int jst = 0;
  {
    const ReadPiece rp = {jw.status, &jst, sizeof(int)};
    CU_E(read_to_host(reader, &rp, 1, st));
  }
  if (launches) *launches += nl;
  if (jst != 0) {
    CU_E(cudaMemset(jw.status, 0, sizeof(int)));
    err = "eigensolver: a barrier of the Jacobi sweeps gave up waiting";
    return RPA_ETIMEOUT;
  }
  return RPA_OK;
}

}  // namespace eig
}  // namespace rpa
