// Mixed-precision subspace of chi~(0) (step a3, Method: the N_eig eigenvectors of
// chi~(0) with the most negative eigenvalues).
//
// GB300's FP64 rate makes a dense FP64 eigensolve of chi~ the largest part of a
// q-point.  Its O(n^3) part, the Householder reduction to a real tridiagonal T, is
// done here in FP32; everything after it in FP64:
//   1. chi~ / max|chi~| in complex64, reduced to T = Q^H (chi~/max) Q (cuSOLVER
//      FP32 hetrd).  The reduction keeps the graded structure of chi~ (the cut
//      eigenvalue is ~1e-5 of the largest), so the m' = N_eig + p eigenvectors of T
//      back-transformed by Q span chi~'s leading subspace to ~1e-5 -- provided T's
//      own eigenpairs are FP64: an FP32 solve of T resolves eigenvalues only to
//      ~1e-7 of the largest, which near the cut mixes the subspace to ~0.1;
//   2. the m' + 1 most negative eigenvalues of T by Sturm bisection (an FP32
//      phase, then FP64 from the FP32 bracket once FP64 counts confirm it) and
//      their eigenvectors by inverse iteration in FP64 (rpa_tridiag.h), one thread
//      per eigenvalue or cluster; Q applied to them in FP32 (cuSOLVER unmtr);
//   3. a degree-3 Chebyshev polynomial of chi~ that damps the interval of the
//      unwanted eigenvalues [lambda_{m'+1}, 0] (scaled at lambda_1, after Zhou and
//      Saad 2007), applied to those m' vectors with FP64 products;
//   4. an orthonormal basis (Householder QR) and a Rayleigh-Ritz step in FP64:
//      the eigenpairs of Q^H chi~ Q give the N_eig Ritz vectors and values.
// p = max(64, N_eig/4) extra vectors put the unwanted eigenvalues that the filter
// must damp well below |lambda_{N_eig}| on these spectra (0.55 of it at N_eig =
// 400), so one step gains ~10-200x; with p = 32 one step only just reached 1e-6 Ha
// at N_G = 4000, N_eig = 400.
// The matrix is used as the column-major view of the row-major chi~ buffer, i.e.
// conj(chi~): same eigenvalues, conjugated eigenvectors (undone by the gauge
// kernel, as for the FP64 solver).
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "rpa_internal.h"
#include "rpa_tc.h"
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

// w[j] for j < k: eigenvalue j (ascending) of T by Sturm bisection, a thread each;
// FP32 bisection finished in FP64 (use32) or FP64 throughout
__global__ void bisect_kernel(const double* d, const double* e, const double* e2, const float* d32,
                              const float* e2f, int n, int k, int use32, double* w) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  double lo, hi, pivmin;
  tri::bounds(d, e, n, &lo, &hi, &pivmin);
  const double abstol = 1e-8 * DBL_EPSILON * fmax(fabs(lo), fabs(hi));
  w[j] = use32 ? tri::bisect_mixed(d, e2, d32, e2f, n, j, lo, hi, pivmin, abstol)
               : tri::bisect(d, e2, n, j, lo, hi, pivmin, abstol);
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

// widest cluster of T's eigenvalues re-orthogonalised by one thread
constexpr int kMaxCluster = 64;

int grid_for(long n, int block) { return (int)std::min<long>((n + block - 1) / block, 4096); }

cuDoubleComplex z(double re, double im = 0.0) { return make_cuDoubleComplex(re, im); }

}  // namespace

int extra_vectors(int n_eig) { return std::max(64, n_eig / 4); }

bool applies(int n, int n_eig) {
  // opt-in (RPA_EIG_MIXED=1) until it passes the subspace-size parity cases on the
  // device (its tridiagonal solver is tested on the host against LAPACK)
  const char* e = getenv("RPA_EIG_MIXED");
  if (!e || e[0] != '1') return false;
  return n >= 1024 && n_eig + extra_vectors(n_eig) + 1 < n;
}

bool products_on_tc() {
  const char* e = getenv("RPA_EIG_TC");
  return !(e && e[0] == '0');
}

rpa_status Refine::alloc(void* sol_, void* params_, int n_max, int mp_max, std::string& err) {
  cusolverDnHandle_t sol = (cusolverDnHandle_t)sol_;
  cusolverDnParams_t params = (cusolverDnParams_t)params_;
  max_n = n_max;
  max_mp = mp_max;
  cublasHandle_t bh = nullptr;
  if (cublasCreate(&bh) != CUBLAS_STATUS_SUCCESS) {
    err = "cublasCreate failed";
    return RPA_ECUDA;
  }
  blas = bh;
  cublasSetPointerMode(bh, CUBLAS_POINTER_MODE_HOST);
  auto al = [&](void** p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      (void)cudaGetLastError();
      err = "mixed eigensolver workspace: cudaMalloc of " + std::to_string(bytes) + " bytes";
      return false;
    }
    return true;
  };
  const size_t n = (size_t)n_max, mp = (size_t)mp_max;
  if (!al((void**)&h32, n * n * sizeof(float2)) || !al((void**)&d32, n * sizeof(float)) ||
      !al((void**)&e32, n * sizeof(float)) || !al((void**)&tau32, n * sizeof(float2)) ||
      !al((void**)&d64, n * sizeof(double)) || !al((void**)&e64, n * sizeof(double)) ||
      !al((void**)&e2, n * sizeof(double)) || !al((void**)&e2f, n * sizeof(float)) ||
      !al((void**)&wt, (mp + 1) * sizeof(double)) ||
      !al((void**)&first, (mp + 1) * sizeof(int)) || !al((void**)&zt, n * mp * sizeof(double)) ||
      !al((void**)&lanes, 6 * n * mp * sizeof(double)) ||
      !al((void**)&c32, n * mp * sizeof(float2)) || !al((void**)&bt, n * mp * sizeof(cplx)) ||
      !al((void**)&yb, mp * mp * sizeof(cplx)) || !al((void**)&dinv, mp * sizeof(double)) ||
      !al((void**)&x0, n * mp * sizeof(cplx)) || !al((void**)&x1, n * mp * sizeof(cplx)) ||
      !al((void**)&x2, n * mp * sizeof(cplx)) || !al((void**)&tau, mp * sizeof(cplx)) ||
      !al((void**)&g, mp * mp * sizeof(cplx)) || !al((void**)&theta, mp * sizeof(double)) ||
      !al((void**)&absmax, sizeof(unsigned long long)) || !al((void**)&info, 4 * sizeof(int))) {
    release();
    return RPA_ENOMEM;
  }
  // solver workspace for the largest shapes (the FP32 reduction and back-transform,
  // QR, and Q^H chi~ Q)
  size_t db = 0, hb = 0, d1 = 0, h1 = 0;
  int lw = 0;
  if (cusolverDnChetrd_bufferSize(sol, CUBLAS_FILL_MODE_LOWER, n_max, (const cuComplex*)h32,
                                  n_max, d32, e32, (const cuComplex*)tau32,
                                  &lw) != CUSOLVER_STATUS_SUCCESS) {
    err = "cusolverDnChetrd_bufferSize failed";
    release();
    return RPA_EEIG;
  }
  db = std::max(db, (size_t)lw * sizeof(cuComplex));
  if (cusolverDnCunmtr_bufferSize(sol, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N,
                                  n_max, mp_max, (const cuComplex*)h32, n_max,
                                  (const cuComplex*)tau32, (const cuComplex*)c32, n_max,
                                  &lw) != CUSOLVER_STATUS_SUCCESS) {
    err = "cusolverDnCunmtr_bufferSize failed";
    release();
    return RPA_EEIG;
  }
  db = std::max(db, (size_t)lw * sizeof(cuComplex));
  if (cusolverDnXgeqrf_bufferSize(sol, params, n_max, mp_max, CUDA_C_64F, x1, n_max, CUDA_C_64F,
                                  tau, CUDA_C_64F, &d1, &h1) != CUSOLVER_STATUS_SUCCESS) {
    err = "cusolverDnXgeqrf_bufferSize failed";
    release();
    return RPA_EEIG;
  }
  db = std::max(db, d1);
  hb = std::max(hb, h1);
  if (cusolverDnZungqr_bufferSize(sol, n_max, mp_max, mp_max, (cuDoubleComplex*)x1, n_max,
                                  (cuDoubleComplex*)tau, &lw) != CUSOLVER_STATUS_SUCCESS) {
    err = "cusolverDnZungqr_bufferSize failed";
    release();
    return RPA_EEIG;
  }
  db = std::max(db, (size_t)lw * sizeof(cuDoubleComplex));
  if (cusolverDnXpotrf_bufferSize(sol, params, CUBLAS_FILL_MODE_UPPER, mp_max, CUDA_C_64F, g,
                                  mp_max, CUDA_C_64F, &d1, &h1) != CUSOLVER_STATUS_SUCCESS) {
    err = "cusolverDnXpotrf_bufferSize failed";
    release();
    return RPA_EEIG;
  }
  db = std::max(db, d1);
  hb = std::max(hb, h1);
  if (cusolverDnXtrtri_bufferSize(sol, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, mp_max,
                                  CUDA_C_64F, g, mp_max, &d1, &h1) != CUSOLVER_STATUS_SUCCESS) {
    err = "cusolverDnXtrtri_bufferSize failed";
    release();
    return RPA_EEIG;
  }
  db = std::max(db, d1);
  hb = std::max(hb, h1);
  if (cusolverDnXsyevd_bufferSize(sol, params, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                                  mp_max, CUDA_C_64F, g, mp_max, CUDA_R_64F, theta, CUDA_C_64F,
                                  &d1, &h1) != CUSOLVER_STATUS_SUCCESS) {
    err = "cusolverDnXsyevd_bufferSize (Rayleigh-Ritz) failed";
    release();
    return RPA_EEIG;
  }
  db = std::max(db, d1);
  hb = std::max(hb, h1);
  dbytes = std::max<size_t>(db, 16);
  hbytes = std::max<size_t>(hb, 16);
  if (!al(&dwork, dbytes)) {
    release();
    return RPA_ENOMEM;
  }
  hwork = malloc(hbytes);
  return RPA_OK;
}

void Refine::release() {
  void* b[] = {h32, d32, e32, tau32, d64, e64, e2, e2f, wt, first, zt, lanes, c32,
               bt, yb, dinv, x0, x1, x2, tau, g, theta, absmax, info, dwork};
  for (void* p : b)
    if (p) cudaFree(p);
  if (hwork) free(hwork);
  if (blas) cublasDestroy((cublasHandle_t)blas);
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
#define CS_E(call)                                                       \
  do {                                                                   \
    cusolverStatus_t s_ = (call);                                        \
    if (s_ != CUSOLVER_STATUS_SUCCESS) {                                 \
      err = std::string(#call ": cuSOLVER status ") + std::to_string((int)s_); \
      return RPA_EEIG;                                                   \
    }                                                                    \
  } while (0)
#define CB_E(call)                                                       \
  do {                                                                   \
    cublasStatus_t s_ = (call);                                          \
    if (s_ != CUBLAS_STATUS_SUCCESS) {                                   \
      err = std::string(#call ": cuBLAS status ") + std::to_string((int)s_); \
      return RPA_ECUDA;                                                  \
    }                                                                    \
  } while (0)

rpa_status Refine::subspace(void* sol_, void* params_, const cplx* hc, int n, int n_eig,
                            double* lam_out, cplx* vec_out, tc::Workspace* tcw, cudaStream_t st,
                            std::string& err, int* launches) {
  cusolverDnHandle_t sol = (cusolverDnHandle_t)sol_;
  cusolverDnParams_t params = (cusolverDnParams_t)params_;
  cublasHandle_t bh = (cublasHandle_t)blas;
  const int mp = n_eig + extra_vectors(n_eig);
  if (n > max_n || mp > max_mp || mp + 1 >= n) {
    err = "mixed eigensolver: shape outside its workspace";
    return RPA_EINVAL;
  }
  const long n2 = (long)n * n;
  CB_E(cublasSetStream(bh, st));
  // 1. chi~ / max|chi~| in complex64, reduced to a real tridiagonal T in FP32
  CU_E(cudaMemsetAsync(absmax, 0, sizeof(unsigned long long), st));
  absmax_kernel<<<grid_for(n2, 256), 256, 0, st>>>(hc, n2, absmax);
  CU_E(cudaGetLastError());
  to_c64_kernel<<<grid_for(n2, 256), 256, 0, st>>>(hc, n2, absmax, h32);
  CU_E(cudaGetLastError());
  CU_E(cudaMemsetAsync(info, 0, 4 * sizeof(int), st));
  const int lwc = (int)std::min<size_t>(dbytes / sizeof(cuComplex), (size_t)0x7fffffff);
  CS_E(cusolverDnChetrd(sol, CUBLAS_FILL_MODE_LOWER, n, (cuComplex*)h32, n, d32, e32,
                        (cuComplex*)tau32, (cuComplex*)dwork, lwc, info + 1));
  // 2. the m' + 1 most negative eigenvalues of T in FP64
  //    (RPA_EIG_BISECT32=0: without the FP32 phase; RPA_EIG_BISECT_BLOCK threads a
  //    block, 32 by default, a multiple of 32 at most 256)
  promote_tri_kernel<<<grid_for(n, 256), 256, 0, st>>>(d32, e32, n, d64, e64, e2, e2f);
  CU_E(cudaGetLastError());
  const char* b32_env = getenv("RPA_EIG_BISECT32");
  const char* blk_env = getenv("RPA_EIG_BISECT_BLOCK");
  const int use32 = !(b32_env && b32_env[0] == '0');
  const int bb = std::max(32, std::min(256, (blk_env ? atoi(blk_env) : 32) / 32 * 32));
  bisect_kernel<<<(mp + 1 + bb - 1) / bb, bb, 0, st>>>(d64, e64, e2, d32, e2f, n, mp + 1, use32,
                                                      wt);
  CU_E(cudaGetLastError());
  std::vector<double> w(mp + 1);
  unsigned long long mx_bits = 0;
  int inf = 0;
  CU_E(cudaMemcpyAsync(w.data(), wt, (mp + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
  CU_E(cudaMemcpyAsync(&mx_bits, absmax, sizeof mx_bits, cudaMemcpyDeviceToHost, st));
  CU_E(cudaMemcpyAsync(&inf, info + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU_E(cudaStreamSynchronize(st));
  if (inf != 0) {
    err = "mixed eigensolver: FP32 tridiagonal reduction info " + std::to_string(inf);
    return RPA_EEIG;
  }
  double mx = 0.0;
  memcpy(&mx, &mx_bits, sizeof mx);
  if (!(mx > 0.0)) mx = 1.0;
  // 3. T's eigenvectors for the first m' (inverse iteration, re-orthogonalised within
  //    clusters of eigenvalues closer than 1e-10 of the largest), then Q applied
  const double tnorm = std::max(std::fabs(w[0]), std::fabs(w[mp]));
  if (!(tnorm > 0.0) || !std::isfinite(tnorm)) {
    err = "mixed eigensolver: degenerate tridiagonal spectrum";
    return RPA_ENUMERIC;
  }
  std::vector<int> fh(mp + 1);
  const int nc = tri::clusters(w.data(), mp, 1e-10 * tnorm, fh.data());
  int widest = 0;
  for (int c = 0; c < nc; ++c) widest = std::max(widest, fh[c + 1] - fh[c]);
  if (widest > kMaxCluster) {
    // one thread would re-orthogonalise the whole cluster: the FP64 solver is faster
    err = "mixed eigensolver: a cluster of " + std::to_string(widest) + " eigenvalues";
    return RPA_ENUMERIC;
  }
  CU_E(cudaMemcpyAsync(first, fh.data(), (nc + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
  invit_kernel<<<(nc + 31) / 32, 32, 0, st>>>(d64, e64, n, wt, first, nc, zt, mp, lanes);
  CU_E(cudaGetLastError());
  z_to_c64_kernel<<<grid_for((long)n * mp, 256), 256, 0, st>>>(zt, n, mp, c32);
  CU_E(cudaGetLastError());
  CS_E(cusolverDnCunmtr(sol, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, n, mp,
                        (cuComplex*)h32, n, (cuComplex*)tau32, (cuComplex*)c32, n,
                        (cuComplex*)dwork, lwc, info + 2));
  to_c128_kernel<<<grid_for((long)n * mp, 256), 256, 0, st>>>(c32, n, mp, x0);
  CU_E(cudaGetLastError());
  if (launches) *launches += 7;

  // Products on the tensor cores (unless RPA_EIG_TC=0) use the projection GEMM,
  // which for a row-major A [rows][K] and a row-major B [K][cols] writes
  // out[c][r] = conj(sum_k A[r][k] B[k][c]), i.e. the column-major rows x cols
  // matrix conj(A B).  Its digit slices are the projection's (6 by default:
  // products exact to ~2^-47 of the row and column scales); the stage timers leave
  // these launches in this stage.  Column-major blocks enter through Zgeam's
  // conjugate transpose, which turns a column-major X into the row-major conj(X).
  const bool on_tc = tcw != nullptr && products_on_tc();
  const cuDoubleComplex one = z(1.0), zero = z(0.0);
  auto tc_gemm = [&](const cplx* a_rm, int rows, int k, const cplx* b_rm, int cols,
                     cplx* out) -> rpa_status {
    const tc::Hook saved = tcw->hook;
    tcw->hook = tc::Hook{};
    int nl = 0;
    const rpa_status r = tc::project(*tcw, a_rm, RPA_C128, rows, k, b_rm, cols, out, st, err, &nl);
    tcw->hook = saved;
    if (launches) *launches += nl;
    return r;
  };
  // Y = H X (n x m'): A = the chi~ buffer (chi~[g'][g] = conj(H(g', g))), B = conj(X)
  auto hx = [&](const cplx* X, cplx* Y) -> rpa_status {
    if (!on_tc) {
      CB_E(cublasZgemm(bh, CUBLAS_OP_N, CUBLAS_OP_N, n, mp, n, &one, (const cuDoubleComplex*)hc,
                       n, (const cuDoubleComplex*)X, n, &zero, (cuDoubleComplex*)Y, n));
      return RPA_OK;
    }
    CB_E(cublasZgeam(bh, CUBLAS_OP_C, CUBLAS_OP_N, mp, n, &one, (const cuDoubleComplex*)X, n,
                     &zero, (const cuDoubleComplex*)bt, mp, (cuDoubleComplex*)bt, mp));
    return tc_gemm(hc, n, n, bt, mp, Y);
  };
  // G = Q^H Z (m' x m') for Z = H Q: A = Z read row-major ([m'][n], A[j][g] = Z(g, j)),
  // B = conj(Q); the GEMM gives conj(Z^T conj(Q)) = Z^H Q = Q^H H Q = G (H Hermitian)
  auto qhz = [&](const cplx* Q, const cplx* Z, cplx* G) -> rpa_status {
    if (!on_tc) {
      CB_E(cublasZgemm(bh, CUBLAS_OP_C, CUBLAS_OP_N, mp, mp, n, &one, (const cuDoubleComplex*)Q,
                       n, (const cuDoubleComplex*)Z, n, &zero, (cuDoubleComplex*)G, mp));
      return RPA_OK;
    }
    CB_E(cublasZgeam(bh, CUBLAS_OP_C, CUBLAS_OP_N, mp, n, &one, (const cuDoubleComplex*)Q, n,
                     &zero, (const cuDoubleComplex*)bt, mp, (cuDoubleComplex*)bt, mp));
    return tc_gemm(Z, mp, n, bt, mp, G);
  };
  // U = Q Y[:, 0:cols] (n x cols, Y m' x m'): A = conj(Q), B = conj(Y[:, 0:cols])
  auto qy = [&](const cplx* Q, const cplx* Y, int cols, cplx* U) -> rpa_status {
    if (!on_tc) {
      CB_E(cublasZgemm(bh, CUBLAS_OP_N, CUBLAS_OP_N, n, cols, mp, &one, (const cuDoubleComplex*)Q,
                       n, (const cuDoubleComplex*)Y, mp, &zero, (cuDoubleComplex*)U, n));
      return RPA_OK;
    }
    CB_E(cublasZgeam(bh, CUBLAS_OP_C, CUBLAS_OP_N, mp, n, &one, (const cuDoubleComplex*)Q, n,
                     &zero, (const cuDoubleComplex*)bt, mp, (cuDoubleComplex*)bt, mp));
    CB_E(cublasZgeam(bh, CUBLAS_OP_C, CUBLAS_OP_N, cols, mp, &one, (const cuDoubleComplex*)Y, mp,
                     &zero, (const cuDoubleComplex*)yb, cols, (cuDoubleComplex*)yb, cols));
    return tc_gemm(bt, n, mp, yb, cols, U);
  };

  // Orthonormal basis of a filtered block Y by column-scaled Cholesky-QR2 (with
  // RPA_EIG_QR=chol and the tensor-core products): two passes of Y <- Y D^-1 with
  // D = diag(||y_j||), G = Y^H Y, G = R^H R (FP64 Cholesky), Y <- Y R^-1 (FP64
  // triangular inverse, the product on the tensor cores).  The columns of a filtered
  // block span ~1e14 in norm; scaled they are conditioned ~1e7 on these spectra,
  // within what Cholesky-QR2 takes.  The scaling is applied to the block itself so
  // that the row-scaled digits of the products see columns of one size.  Y and
  // spare are swapped as the passes go; done stays false when a Cholesky factor
  // fails (then Y, rescaled, still spans the filtered block for Householder QR).
  const char* qr_env = getenv("RPA_EIG_QR");
  const bool chol_qr = on_tc && qr_env && strcmp(qr_env, "chol") == 0;
  auto chol_qr2 = [&](cplx*& Y, cplx*& spare, bool& done) -> rpa_status {
    done = false;
    for (int pass = 0; pass < 2; ++pass) {
      inv_colnorm_kernel<<<mp, 256, 0, st>>>(Y, n, mp, dinv);
      CU_E(cudaGetLastError());
      scale_cols_kernel<<<grid_for((long)n * mp, 256), 256, 0, st>>>(Y, n, mp, dinv);
      CU_E(cudaGetLastError());
      rpa_status rq = qhz(Y, Y, g);  // G = Y^H Y
      if (rq != RPA_OK) return rq;
      CU_E(cudaMemsetAsync(info + 3, 0, sizeof(int), st));
      CS_E(cusolverDnXpotrf(sol, params, CUBLAS_FILL_MODE_UPPER, mp, CUDA_C_64F, g, mp,
                            CUDA_C_64F, dwork, dbytes, hwork, hbytes, info + 3));
      int pinf = 0;
      CU_E(cudaMemcpyAsync(&pinf, info + 3, sizeof(int), cudaMemcpyDeviceToHost, st));
      CU_E(cudaStreamSynchronize(st));
      if (pinf != 0) return RPA_OK;
      CS_E(cusolverDnXtrtri(sol, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, mp, CUDA_C_64F, g,
                            mp, dwork, dbytes, hwork, hbytes, info + 3));
      zero_lower_kernel<<<grid_for((long)mp * mp, 256), 256, 0, st>>>(g, mp);
      CU_E(cudaGetLastError());
      if ((rq = qy(Y, g, mp, spare)) != RPA_OK) return rq;  // Y R^-1
      std::swap(Y, spare);
      if (launches) *launches += 3;
    }
    int tinf = 0;
    CU_E(cudaMemcpyAsync(&tinf, info + 3, sizeof(int), cudaMemcpyDeviceToHost, st));
    CU_E(cudaStreamSynchronize(st));
    if (tinf != 0) {
      err = "mixed eigensolver: triangular inverse info " + std::to_string(tinf);
      return RPA_EEIG;
    }
    done = true;
    return RPA_OK;
  };

  // 4.-5. RPA_EIG_STEPS (default 1, at most 8) filtered Rayleigh-Ritz steps.  Each
  //    applies a degree-3 Chebyshev filter damping [a, 0] -- a = lambda_{m'+1} of T
  //    first, the largest Ritz value of the block after that -- scaled at lambda_1,
  //    takes an orthonormal basis Q of the filtered block (Householder QR, FP64)
  //    and the eigenpairs of Q^H H Q (FP64); a further step starts from all m'
  //    Ritz vectors.
  const char* steps_env = getenv("RPA_EIG_STEPS");
  const int steps = std::max(1, std::min(8, steps_env ? atoi(steps_env) : 1));
  double a = w[mp] * mx, lo = w[0] * mx;
  const double b = 0.0;
  cplx* xs = x0;  // the block the next filter starts from
  rpa_status r = RPA_OK;
  for (int step = 0; step < steps; ++step) {
    if (!(a < 0.0) || !(lo < a)) {
      // no unwanted interval to damp (the bound not below zero, or no spread): the
      // caller takes the FP64 solver
      err = "mixed eigensolver: degenerate spectrum bounds";
      return RPA_ENUMERIC;
    }
    const double e = 0.5 * (b - a), c = 0.5 * (b + a);
    double sigma = e / (lo - c);
    const double tau2 = 2.0 / sigma;
    // X_{k-1}, X_k, X_{k+1}: the start block and the two other buffers
    cplx *xm = xs, *xk = xs == x0 ? x1 : x0, *xn = xs == x2 ? x1 : x2;
    // X_1 = (sigma / e) (H - c) X_0
    if ((r = hx(xm, xk)) != RPA_OK) return r;
    {
      const cuDoubleComplex al = z(sigma / e), be = z(-c * sigma / e);
      CB_E(cublasZgeam(bh, CUBLAS_OP_N, CUBLAS_OP_N, n, mp, &al, (const cuDoubleComplex*)xk, n,
                       &be, (const cuDoubleComplex*)xm, n, (cuDoubleComplex*)xk, n));
    }
    for (int k = 2; k <= 3; ++k) {
      const double s1 = 1.0 / (tau2 - sigma);
      // X_{k+1} = (2 s1 / e) (H - c) X_k - sigma s1 X_{k-1}
      if ((r = hx(xk, xn)) != RPA_OK) return r;
      const cuDoubleComplex al = z(2.0 * s1 / e), be = z(-2.0 * s1 * c / e);
      CB_E(cublasZgeam(bh, CUBLAS_OP_N, CUBLAS_OP_N, n, mp, &al, (const cuDoubleComplex*)xn, n,
                       &be, (const cuDoubleComplex*)xk, n, (cuDoubleComplex*)xn, n));
      const cuDoubleComplex be2 = z(-sigma * s1);
      CB_E(cublasZgeam(bh, CUBLAS_OP_N, CUBLAS_OP_N, n, mp, &one, (const cuDoubleComplex*)xn, n,
                       &be2, (const cuDoubleComplex*)xm, n, (cuDoubleComplex*)xn, n));
      std::swap(xm, xk);  // X_{k-1} <- X_k
      std::swap(xk, xn);  // X_k <- X_{k+1}; xn now holds the oldest block (free)
      sigma = s1;
    }
    // orthonormal basis Q of the filtered block (into xk; xm is free)
    bool qr_done = false;
    if (chol_qr && (r = chol_qr2(xk, xm, qr_done)) != RPA_OK) return r;
    if (!qr_done) {
      CS_E(cusolverDnXgeqrf(sol, params, n, mp, CUDA_C_64F, xk, n, CUDA_C_64F, tau, CUDA_C_64F,
                            dwork, dbytes, hwork, hbytes, info));
      CS_E(cusolverDnZungqr(sol, n, mp, mp, (cuDoubleComplex*)xk, n, (const cuDoubleComplex*)tau,
                            (cuDoubleComplex*)dwork, (int)(dbytes / sizeof(cuDoubleComplex)),
                            info));
    }
    // Rayleigh-Ritz: G = Q^H (H Q), G = Y Theta Y^H
    if ((r = hx(xk, xn)) != RPA_OK) return r;
    if ((r = qhz(xk, xn, g)) != RPA_OK) return r;
    CS_E(cusolverDnXsyevd(sol, params, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, mp,
                          CUDA_C_64F, g, mp, CUDA_R_64F, theta, CUDA_C_64F, dwork, dbytes, hwork,
                          hbytes, info));
    int infs[3] = {0, 0, 0};
    if (step + 1 < steps) {
      // U = Q Y (all m' Ritz vectors, into the buffer H Q occupied) starts the next
      // step; its filter damps beyond the largest Ritz value
      if ((r = qy(xk, g, mp, xn)) != RPA_OK) return r;
      std::vector<double> th(mp);
      CU_E(cudaMemcpyAsync(th.data(), theta, sizeof(double) * mp, cudaMemcpyDeviceToHost, st));
      CU_E(cudaMemcpyAsync(infs, info, sizeof infs, cudaMemcpyDeviceToHost, st));
      CU_E(cudaStreamSynchronize(st));
      if (infs[0] != 0) {
        err = "mixed eigensolver: QR or Rayleigh-Ritz info " + std::to_string(infs[0]);
        return RPA_EEIG;
      }
      a = th[mp - 1];
      lo = th[0];
      xs = xn;
      continue;
    }
    // the N_eig Ritz pairs: U = Q Y[:, 0:N_eig]
    if ((r = qy(xk, g, n_eig, vec_out)) != RPA_OK) return r;
    CU_E(cudaMemcpyAsync(lam_out, theta, sizeof(double) * n_eig, cudaMemcpyDeviceToDevice, st));
    CU_E(cudaMemcpyAsync(infs, info, sizeof infs, cudaMemcpyDeviceToHost, st));
    CU_E(cudaStreamSynchronize(st));
    if (infs[0] != 0 || infs[2] != 0) {
      err = "mixed eigensolver: back-transform info " + std::to_string(infs[2]) +
            ", QR or Rayleigh-Ritz info " + std::to_string(infs[0]);
      return RPA_EEIG;
    }
  }
  return RPA_OK;
}

}  // namespace eig
}  // namespace rpa
