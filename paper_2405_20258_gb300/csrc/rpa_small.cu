// Small FP64 kernels of the RPA path: per-q scalars, the imaginary-frequency
// quadrature, eigenvector gauge, the FP64 trace term, the energy reductions,
// and the counter-based input generator.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "rpa_internal.h"

namespace rpa {
namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum (fixed order for a fixed blockDim); result in every thread.
__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < nw ? sh[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

// sv[g] = sqrt(v(q+G)) with the bare or the slab-truncated Coulomb kernel;
// per transition vc = (k n_v + v) n_c + c: delta = e_c - e_v, pair weight
// ow = g_k (f_v - f_c) (Eq. chi0_partial_occs), sf0 = sqrt(ow f(0)) = sqrt(4 ow / delta).
__global__ void prepare_kernel(rpa_qpoint q, double* sv, double* delta, double* ow, double* sf0,
                               int* bad) {
  const int n_k = q.n_k > 1 ? q.n_k : 1;
  const long per_k = (long)q.n_v * q.n_c;
  const long n_vc = n_k * per_k;
  long stride = (long)gridDim.x * blockDim.x;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < q.n_g + n_vc; i += stride) {
    if (i < q.n_g) {
      double k2 = q.qg2[i];
      if (!(k2 > 0.0) || !isfinite(k2)) atomicOr(bad, 1);
      double v = 4.0 * kPi / k2;
      if (q.coulomb == RPA_COULOMB_SLAB) {
        const double* kv = q.qg_vec + 3 * i;
        double kpar = hypot(kv[0], kv[1]);
        v *= 1.0 - exp(-kpar * q.slab_zc) * cos(kv[2] * q.slab_zc);
        if (!(v > 0.0) || !isfinite(v)) atomicOr(bad, 8);
      }
      sv[i] = sqrt(v);
    } else {
      long vc = i - q.n_g;
      int k = (int)(vc / per_k);
      long r = vc % per_k;
      int v = (int)(r / q.n_c), c = (int)(r % q.n_c);
      double d = q.e_c[(long)k * q.n_c + c] - q.e_v[(long)k * q.n_v + v];
      double fv = q.occ_v ? q.occ_v[(long)k * q.n_v + v] : 1.0;
      double fc = q.occ_c ? q.occ_c[(long)k * q.n_c + c] : 0.0;
      double w = (q.k_weight ? q.k_weight[k] : 1.0) * (fv - fc);
      if (!isfinite(d)) atomicOr(bad, 2);
      if (!isfinite(w) || w * d < 0.0 || (d == 0.0 && w != 0.0)) atomicOr(bad, 4);
      delta[vc] = d;
      ow[vc] = w;
      sf0[vc] = w != 0.0 ? sqrt(4.0 * w / d) : 0.0;
    }
  }
}

// Gauss-Legendre nodes and weights on [-1,1] by Newton's method on P_n, then
// the map t = (x+1)/2, w = s t/(1-t), weight = (w_GL/2) s/(1-t)^2.
__global__ void freq_grid_kernel(int n, double s, double* omega, double* weight) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int i = n - k;  // root index, descending in x, so k runs ascending
  double x = cos(kPi * (i - 0.25) / (n + 0.5));
  double p0 = 1.0, p1 = x, dp = 1.0;
  for (int it = 0; it < 100; ++it) {
    p0 = 1.0;
    p1 = x;
    for (int j = 1; j < n; ++j) {
      double p2 = ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0);
      p0 = p1;
      p1 = p2;
    }
    dp = n * (x * p1 - p0) / (x * x - 1.0);
    double dx = p1 / dp;
    x -= dx;
    if (fabs(dx) <= 1e-16) break;
  }
  // derivative at the converged node
  p0 = 1.0;
  p1 = x;
  for (int j = 1; j < n; ++j) {
    double p2 = ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0);
    p0 = p1;
    p1 = p2;
  }
  dp = n * (x * p1 - p0) / (x * x - 1.0);
  double wgl = 2.0 / ((1.0 - x * x) * dp * dp);
  double t = 0.5 * (x + 1.0);
  double omt = 1.0 - t;
  omega[k] = s * t / omt;
  weight[k] = 0.5 * wgl * s / (omt * omt);
}

// One block per eigenvector column: C = conj(U) with its largest-modulus entry
// (lowest row on ties) made real positive; B = sv * C.
__global__ void gauge_kernel(const cplx* U, int ldu, int n_g, int n_eig, const double* sv,
                             cplx* C, cplx* B) {
  __shared__ double bv[32];
  __shared__ int bi[32];
  const int col = blockIdx.x;
  const cplx* u = U + (size_t)col * ldu;
  double best = -1.0;
  int idx = 0x7fffffff;
  for (int g = threadIdx.x; g < n_g; g += blockDim.x) {
    double m = u[g].re * u[g].re + u[g].im * u[g].im;
    if (m > best) {
      best = m;
      idx = g;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double ob = __shfl_xor_sync(0xffffffffu, best, o);
    int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ob > best || (ob == best && oi < idx)) {
      best = ob;
      idx = oi;
    }
  }
  int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    bv[w] = best;
    bi[w] = idx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int nw = blockDim.x >> 5;
    for (int j = 1; j < nw; ++j)
      if (bv[j] > bv[0] || (bv[j] == bv[0] && bi[j] < bi[0])) {
        bv[0] = bv[j];
        bi[0] = bi[j];
      }
  }
  __syncthreads();
  // pivot of C = conj(U[piv]); factor = |p| / p = conj(p)/|p| = U[piv]/|U[piv]|
  cplx up = u[bi[0]];
  double r = hypot(up.re, up.im);
  double fr = r > 0.0 ? up.re / r : 1.0, fi = r > 0.0 ? up.im / r : 0.0;
  for (int g = threadIdx.x; g < n_g; g += blockDim.x) {
    double cr = u[g].re, ci = -u[g].im;  // conj(U)
    double xr = cr * fr - ci * fi, xi = cr * fi + ci * fr;
    if (g == bi[0]) xi = 0.0;
    size_t o = (size_t)g * n_eig + col;
    if (C) C[o] = {xr, xi};
    B[o] = {sv[g] * xr, sv[g] * xi};
  }
}

// w[vc] = sum_i |mt[i][vc]|^2
__global__ void colnorm_kernel(const cplx* mt, int n_eig, int n_vc, double* w) {
  int vc = blockIdx.x * blockDim.x + threadIdx.x;
  if (vc >= n_vc) return;
  double s = 0.0;
  for (int i = 0; i < n_eig; ++i) {
    cplx m = mt[(size_t)i * n_vc + vc];
    s = fma(m.re, m.re, s);
    s = fma(m.im, m.im, s);
  }
  w[vc] = s;
}

// trace[k] = scale sum_vc f_k(vc) w[vc]; one block per frequency, fixed order.
__global__ void trace_kernel(const double* w, const double* delta, const double* ow, int n_vc,
                             const double* omega, double scale, double* trace) {
  __shared__ double sh[33];
  const int k = blockIdx.x;
  const double w2 = omega[k] * omega[k];
  double s = 0.0;
  for (int vc = threadIdx.x; vc < n_vc; vc += blockDim.x) {
    double d = delta[vc], o = ow[vc];
    if (o != 0.0) s += o * (4.0 * d / (d * d + w2)) * w[vc];
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) trace[k] = scale * s;
}

// f[k][vc] = ow[vc] 4 D / (D^2 + w_k^2)
__global__ void all_freq_weights_kernel(const double* delta, const double* ow, int n_vc,
                                        const double* omega, int n_freq, double* f) {
  long n = (long)n_freq * n_vc;
  long stride = (long)gridDim.x * blockDim.x;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += stride) {
    int k = (int)(i / n_vc), vc = (int)(i % n_vc);
    double d = delta[vc], o = ow[vc], w = omega[k];
    f[i] = o != 0.0 ? o * (4.0 * d / (d * d + w * w)) : 0.0;
  }
}

// One block per (row i, group of DIAG_K frequencies): the FP64 diagonal of chi_s.
constexpr int DIAG_K = 16;
__global__ void chis_diagonal_kernel(const cplx* mt, int n_eig, int n_vc, const double* f,
                                     int n_freq, double scale, cplx* chis) {
  __shared__ double red[DIAG_K][33];
  const int i = blockIdx.x, k0 = blockIdx.y * DIAG_K;
  const int nk = min(DIAG_K, n_freq - k0);
  double acc[DIAG_K];
#pragma unroll
  for (int b = 0; b < DIAG_K; ++b) acc[b] = 0.0;
  for (int vc = threadIdx.x; vc < n_vc; vc += blockDim.x) {
    cplx m = mt[(size_t)i * n_vc + vc];
    double a = fma(m.re, m.re, m.im * m.im);
#pragma unroll
    for (int b = 0; b < DIAG_K; ++b)
      if (b < nk) acc[b] = fma(f[(size_t)(k0 + b) * n_vc + vc], a, acc[b]);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int b = 0; b < DIAG_K; ++b) {
    double v = warp_sum(acc[b]);
    if (l == 0) red[b][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < nk) {
    double t = 0.0;
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) t += red[threadIdx.x][j];
    cplx* o = chis + ((size_t)(k0 + threadIdx.x) * n_eig + i) * n_eig + i;
    *o = {scale * t, 0.0};
  }
}

// ec = (1/2pi) sum_k weight_k [sum_i log1p(-lam_ki) + trace_k]
__global__ void logsum_kernel(const double* lam, int n_eig, int ld, int n_freq,
                              const double* trace, const double* weight, double* ec, int* bad) {
  __shared__ double sh[33];
  double tot = 0.0;
  for (int k = 0; k < n_freq; ++k) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n_eig; i += blockDim.x) {
      double l = lam[(size_t)k * ld + i];
      if (!(1.0 - l > 0.0) || !isfinite(l)) atomicOr(bad, 4);
      s += log1p(-l);
    }
    s = block_sum(s, sh);
    tot += weight[k] * (s + trace[k]);
  }
  if (threadIdx.x == 0) {
    if (!isfinite(tot)) atomicOr(bad, 8);
    *ec = tot / (2.0 * kPi);
  }
}

__global__ void logdet_sum_kernel(const double* logdet, int n_freq, const double* trace,
                                  const double* weight, double* ec, int* bad) {
  if (threadIdx.x != 0) return;
  double tot = 0.0;
  for (int k = 0; k < n_freq; ++k) tot += weight[k] * (logdet[k] + trace[k]);
  if (!isfinite(tot)) atomicOr(bad, 8);
  *ec = tot / (2.0 * kPi);
}

// ---- counter-based generator (splitmix64 of Steele, Lea and Flood 2014) ----

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double unit_uniform(uint64_t b) {
  return ((double)(b >> 11) + 0.5) * 0x1.0p-53;
}

template <typename T>
__global__ void generate_m_kernel(int n_g, int iq, unsigned long long seed, const int* miller,
                                  const double* qg2, int v0, int nv, int c0, int nc, T* out) {
  long total = (long)nv * nc * n_g;
  long stride = (long)gridDim.x * blockDim.x;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += stride) {
    int g = (int)(e % n_g);
    long vc = e / n_g;
    uint64_t v = (uint64_t)(v0 + vc / nc), c = (uint64_t)(c0 + vc % nc);
    const uint64_t bias = 1ull << 20;
    uint64_t pk = ((uint64_t)(miller[3 * g] + (long)bias) << 42) |
                  ((uint64_t)(miller[3 * g + 1] + (long)bias) << 21) |
                  (uint64_t)(miller[3 * g + 2] + (long)bias);
    uint64_t key = (((uint64_t)iq << 16) + v) << 32 | c;
    key = splitmix64((uint64_t)seed ^ splitmix64(splitmix64(key) ^ pk));
    double u0 = unit_uniform(splitmix64(key));
    double u1 = unit_uniform(splitmix64(key ^ 2ull));
    double rad = sqrt(-2.0 * log(u0)) / sqrt(2.0);
    double ang = 2.0 * kPi * u1;
    double env = exp(-qg2[g] / 8.0);
    double re = rad * cos(ang) * env, im = rad * sin(ang) * env;
    if constexpr (sizeof(T) == 8) {
      out[e] = make_float2((float)re, (float)im);
    } else {
      out[e] = make_double2(re, im);
    }
  }
}

inline int grid_for(long n, int bs) {
  long b = (n + bs - 1) / bs;
  return (int)(b < 152L * 32 ? (b > 0 ? b : 1) : 152L * 32);
}

// ---- transition order of the tensor-core chi~(0) K-blocks --------------------
// Transitions by decreasing |w_vc / Delta_vc| (w_vc = g_k (f_v - f_c) the pair weight,
// so the key orders like f_vc(0)), equal keys by index (the
// permutation of a stable sort), within segments of consecutive transitions when a
// q-point is drawn in chunks of valence bands.  Items (segment, key bits, index) are
// sorted ascending by a bitonic network: a non-negative double's bit pattern orders
// like its value, so its complement orders by decreasing weight.  Padding items
// carry the largest segment and sort last.
struct OrderItem {
  unsigned long long kb;
  unsigned seg, idx;
};

__device__ __forceinline__ bool item_less(const OrderItem& a, const OrderItem& b) {
  if (a.seg != b.seg) return a.seg < b.seg;
  if (a.kb != b.kb) return a.kb < b.kb;
  return a.idx < b.idx;
}

// Compare-exchange of items i < l of stage k: ascending where bit k of i is clear.
__device__ __forceinline__ void order_cx(OrderItem& a, OrderItem& b, bool asc) {
  if (asc ? item_less(b, a) : item_less(a, b)) {
    const OrderItem t = a;
    a = b;
    b = t;
  }
}

// nvb > 0: segments of nvb valence bands (the chunks of a streamed q-point).
__global__ void order_keys_kernel(const double* delta, const double* ow, long n, int n_v,
                                  int n_c, int nvb, long npad, OrderItem* it) {
  const long stride = (long)gridDim.x * blockDim.x;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < npad; i += stride) {
    OrderItem x;
    x.idx = (unsigned)i;
    if (i < n) {
      const double d = delta[i], w = ow[i];
      const double key = (w != 0.0 && d != 0.0) ? fabs(w / d) : 0.0;
      x.kb = ~(unsigned long long)__double_as_longlong(key);
      x.seg = 0;
      if (nvb > 0) {
        const long per_k = (long)n_v * n_c, k = i / per_k;
        const int vb = (int)((i % per_k) / n_c);
        x.seg = (unsigned)(k * ((n_v + nvb - 1) / nvb) + vb / nvb);
      }
    } else {
      x.kb = ~0ull;
      x.seg = 0xffffffffu;
    }
    it[i] = x;
  }
}

// One tile of kOrderTile items per block in shared memory.  kk == 0: the stages
// k = 2 .. kOrderTile (each tile sorted, in the direction stage kOrderTile gives it);
// kk > kOrderTile: the strides kOrderTile/2 .. 1 of stage kk.
constexpr int kOrderTile = 2048;

__global__ void __launch_bounds__(kOrderTile / 2) order_tile_kernel(OrderItem* it, long kk) {
  __shared__ OrderItem s[kOrderTile];
  const long base = (long)blockIdx.x * kOrderTile;
  const int t = threadIdx.x, h = kOrderTile / 2;
  s[t] = it[base + t];
  s[t + h] = it[base + t + h];
  __syncthreads();
  const long k0 = kk ? kk : 2, k1 = kk ? kk : kOrderTile;
  for (long k = k0; k <= k1; k <<= 1)
    for (int j = (int)(k / 2 < h ? k / 2 : h); j > 0; j >>= 1) {
      const int i = 2 * j * (t / j) + t % j;
      order_cx(s[i], s[i + j], ((base + i) & k) == 0);
      __syncthreads();
    }
  it[base + t] = s[t];
  it[base + t + h] = s[t + h];
}

// Stride j >= kOrderTile of stage k, one compare-exchange per thread.
__global__ void order_merge_kernel(OrderItem* it, long pairs, long k, long j) {
  const long stride = (long)gridDim.x * blockDim.x;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < pairs; t += stride) {
    const long i = 2 * j * (t / j) + t % j;
    OrderItem a = it[i], b = it[i + j];
    const unsigned a0 = a.idx;
    order_cx(a, b, (i & k) == 0);
    if (a.idx != a0) {
      it[i] = a;
      it[i + j] = b;
    }
  }
}

// order[pos] = transition index, local to its segment's first transition.
__global__ void order_out_kernel(const OrderItem* it, long n, int n_v, int n_c, int nvb,
                                 int* order) {
  const long stride = (long)gridDim.x * blockDim.x;
  const unsigned nchk = nvb > 0 ? (unsigned)((n_v + nvb - 1) / nvb) : 1u;
  for (long pos = blockIdx.x * (long)blockDim.x + threadIdx.x; pos < n; pos += stride) {
    const OrderItem x = it[pos];
    long r0 = 0;
    if (nvb > 0) r0 = ((long)(x.seg / nchk) * n_v + (long)(x.seg % nchk) * nvb) * n_c;
    order[pos] = (int)((long)x.idx - r0);
  }
}

// Words of up to four device arrays into one host-mapped buffer (read_to_host).
struct ReadArgs {
  const unsigned* src[4];
  unsigned off[4], words[4];
  int n;
};

__global__ void read_pieces_kernel(ReadArgs a, unsigned* out) {
  for (int k = 0; k < a.n; ++k)
    for (unsigned i = threadIdx.x; i < a.words[k]; i += blockDim.x) out[a.off[k] + i] = a.src[k][i];
  __threadfence_system();
}

}  // namespace

cudaError_t launch_prepare_scalars(const rpa_qpoint& q, double* sv, double* delta, double* ow,
                                   double* sf0, int* bad, cudaStream_t st) {
  long n = q.n_g + n_transitions(q);
  prepare_kernel<<<grid_for(n, 256), 256, 0, st>>>(q, sv, delta, ow, sf0, bad);
  return cudaGetLastError();
}

cudaError_t reader_alloc(HostReader& r, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  void* h = nullptr;
  cudaError_t e = cudaHostAlloc(&h, bytes, cudaHostAllocMapped);
  if (e != cudaSuccess) return e;
  void* d = nullptr;
  e = cudaHostGetDevicePointer(&d, h, 0);
  if (e != cudaSuccess) {
    cudaFreeHost(h);
    return e;
  }
  r.host = (char*)h;
  r.dev = (char*)d;
  r.bytes = bytes;
  return cudaSuccess;
}

void reader_free(HostReader& r) {
  if (r.host) cudaFreeHost(r.host);
  r = HostReader{};
}

cudaError_t read_to_host(HostReader& r, const ReadPiece* p, int n, cudaStream_t st) {
  size_t total = 0;
  bool fits = r.host && n <= 4;
  for (int k = 0; k < n; ++k) {
    fits = fits && p[k].bytes % 4 == 0 && ((uintptr_t)p[k].src & 3) == 0;
    total += p[k].bytes;
  }
  if (!fits || total > r.bytes) {
    for (int k = 0; k < n; ++k) {
      cudaError_t e = cudaMemcpyAsync(p[k].dst, p[k].src, p[k].bytes, cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) return e;
    }
    return cudaStreamSynchronize(st);
  }
  ReadArgs a{};
  a.n = n;
  unsigned off = 0;
  for (int k = 0; k < n; ++k) {
    a.src[k] = (const unsigned*)p[k].src;
    a.off[k] = off;
    a.words[k] = (unsigned)(p[k].bytes / 4);
    off += a.words[k];
  }
  read_pieces_kernel<<<1, 256, 0, st>>>(a, (unsigned*)r.dev);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < n; ++k) memcpy(p[k].dst, r.host + 4 * (size_t)a.off[k], p[k].bytes);
  return cudaSuccess;
}

long order_items(long n) {
  long npad = kOrderTile;
  while (npad < n) npad <<= 1;
  return npad;
}

cudaError_t launch_transition_order(const double* delta, const double* ow, long n, int n_v,
                                    int n_c, int nvb, void* items, int* order, cudaStream_t st,
                                    int* launches) {
  if (n <= 0) return cudaSuccess;
  const long npad = order_items(n);
  OrderItem* it = (OrderItem*)items;
  order_keys_kernel<<<grid_for(npad, 256), 256, 0, st>>>(delta, ow, n, n_v, n_c, nvb, npad, it);
  const unsigned tiles = (unsigned)(npad / kOrderTile);
  order_tile_kernel<<<tiles, kOrderTile / 2, 0, st>>>(it, 0);
  int nl = 2;
  for (long k = 2L * kOrderTile; k <= npad; k <<= 1) {
    for (long j = k / 2; j >= kOrderTile; j >>= 1) {
      order_merge_kernel<<<grid_for(npad / 2, 256), 256, 0, st>>>(it, npad / 2, k, j);
      ++nl;
    }
    order_tile_kernel<<<tiles, kOrderTile / 2, 0, st>>>(it, k);
    ++nl;
  }
  order_out_kernel<<<grid_for(n, 256), 256, 0, st>>>(it, n, n_v, n_c, nvb, order);
  if (launches) *launches += nl + 1;
  return cudaGetLastError();
}

cudaError_t launch_freq_grid(int n_freq, double s, double* omega, double* weight,
                             cudaStream_t st) {
  freq_grid_kernel<<<(n_freq + 63) / 64, 64, 0, st>>>(n_freq, s, omega, weight);
  return cudaGetLastError();
}

cudaError_t launch_gauge(const cplx* U, int ldu, int n_g, int n_eig, const double* sv, cplx* C,
                         cplx* B, cudaStream_t st) {
  gauge_kernel<<<n_eig, 256, 0, st>>>(U, ldu, n_g, n_eig, sv, C, B);
  return cudaGetLastError();
}

cudaError_t launch_trace(const cplx* mt, int n_eig, int n_vc, const double* delta,
                         const double* ow, const double* omega, int n_freq, double scale,
                         double* w, double* trace, cudaStream_t st) {
  colnorm_kernel<<<(n_vc + 255) / 256, 256, 0, st>>>(mt, n_eig, n_vc, w);
  trace_kernel<<<n_freq, 1024, 0, st>>>(w, delta, ow, n_vc, omega, scale, trace);
  return cudaGetLastError();
}

cudaError_t launch_all_freq_weights(const double* delta, const double* ow, int n_vc,
                                    const double* omega, int n_freq, double* f, cudaStream_t st) {
  all_freq_weights_kernel<<<grid_for((long)n_freq * n_vc, 256), 256, 0, st>>>(delta, ow, n_vc,
                                                                              omega, n_freq, f);
  return cudaGetLastError();
}

// FP64 diagonal of chi~(0), which the digit-sliced GEMM gets slightly wrong: it
// multiplies only digit pairs s + t <= S - 1, and on the diagonal the dropped pairs
// include |d_s|^2 terms of one sign, a bias that adds up over every transition.
// part[c][g] = sum over the rows r of chunk c of sf0[r]^2 |A[r][g]|^2 (a thread per
// g, coalesced along G); then chi[g][g] = scale sv[g]^2 sum_c part[c][g] in chunk
// order (deterministic).
__global__ void chi0_diag_partial_kernel(const void* A, int dtype, long n_vc, int n_g,
                                         const double* sf0, long rows_per_chunk, double* part) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_g) return;
  const long r0 = (long)blockIdx.y * rows_per_chunk;
  const long r1 = min(n_vc, r0 + rows_per_chunk);
  double acc = 0.0;
  if (dtype == RPA_C64) {
    const float2* a = (const float2*)A;
    for (long r = r0; r < r1; ++r) {
      const float2 v = a[r * n_g + g];
      const double w = sf0[r], re = v.x, im = v.y;
      acc = fma(w * w, fma(re, re, im * im), acc);
    }
  } else {
    const double2* a = (const double2*)A;
    for (long r = r0; r < r1; ++r) {
      const double2 v = a[r * n_g + g];
      const double w = sf0[r];
      acc = fma(w * w, fma(v.x, v.x, v.y * v.y), acc);
    }
  }
  part[(long)blockIdx.y * n_g + g] = acc;
}

__global__ void chi0_diag_finish_kernel(const double* part, int n_chunks, int n_g,
                                        const double* sv, double scale, cplx* chi, double* acc,
                                        int first, int last) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_g) return;
  double t = (acc && !first) ? acc[g] : 0.0;
  for (int c = 0; c < n_chunks; ++c) t += part[(long)c * n_g + g];
  if (!last) {
    acc[g] = t;
    return;
  }
  const double s = sv[g];
  chi[(long)g * n_g + g] = {scale * s * s * t, 0.0};
}

cudaError_t launch_chi0_diagonal(const void* A, int dtype, long n_vc, int n_g, const double* sf0,
                                 const double* sv, double scale, double* scratch,
                                 size_t scratch_doubles, cplx* chi, cudaStream_t st, int part,
                                 int n_parts) {
  if (n_g < 1 || n_vc < 1) return cudaSuccess;
  // a q-point whose transitions arrive in n_parts pieces: the running sums live at
  // the end of the scratch, the diagonal is written with the last piece
  double* acc = nullptr;
  if (n_parts > 1) {
    if (scratch_doubles < 2 * (size_t)n_g) return cudaErrorInvalidValue;
    scratch_doubles -= (size_t)n_g;
    acc = scratch + scratch_doubles;
  }
  // enough chunks to fill the GPU with a few thousand rows each, within the scratch
  long chunks = std::min<long>(64, (n_vc + 1023) / 1024);
  chunks = std::min<long>(chunks, (long)(scratch_doubles / (size_t)n_g));
  if (chunks < 1) return cudaErrorInvalidValue;
  const long rows = (n_vc + chunks - 1) / chunks;
  const int nc = (int)((n_vc + rows - 1) / rows);
  dim3 grid((n_g + 255) / 256, nc);
  chi0_diag_partial_kernel<<<grid, 256, 0, st>>>(A, dtype, n_vc, n_g, sf0, rows, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  chi0_diag_finish_kernel<<<(n_g + 255) / 256, 256, 0, st>>>(scratch, nc, n_g, sv, scale, chi, acc,
                                                             part == 0, part == n_parts - 1);
  return cudaGetLastError();
}

cudaError_t launch_chis_diagonal(const cplx* mt, int n_eig, int n_vc, const double* f,
                                 int n_freq, double scale, cplx* chis, cudaStream_t st) {
  dim3 grid(n_eig, (n_freq + DIAG_K - 1) / DIAG_K);
  chis_diagonal_kernel<<<grid, 256, 0, st>>>(mt, n_eig, n_vc, f, n_freq, scale, chis);
  return cudaGetLastError();
}

cudaError_t launch_logsum(const double* lam, int n_eig, int ld_lam, int n_freq,
                          const double* trace, const double* weight, double* ec, int* bad,
                          cudaStream_t st) {
  logsum_kernel<<<1, 256, 0, st>>>(lam, n_eig, ld_lam, n_freq, trace, weight, ec, bad);
  return cudaGetLastError();
}

cudaError_t launch_logdet_sum(const double* logdet, int n_freq, const double* trace,
                              const double* weight, double* ec, int* bad, cudaStream_t st) {
  logdet_sum_kernel<<<1, 32, 0, st>>>(logdet, n_freq, trace, weight, ec, bad);
  return cudaGetLastError();
}

cudaError_t launch_generate_m(const rpa_qpoint* q, int v0, int nv, int c0, int nc, void* out,
                              int dtype, cudaStream_t st) {
  long n = (long)nv * nc * q->n_g;
  if (dtype == RPA_C64)
    generate_m_kernel<float2><<<grid_for(n, 256), 256, 0, st>>>(
        q->n_g, q->iq, q->seed, q->miller, q->qg2, v0, nv, c0, nc, (float2*)out);
  else
    generate_m_kernel<double2><<<grid_for(n, 256), 256, 0, st>>>(
        q->n_g, q->iq, q->seed, q->miller, q->qg2, v0, nv, c0, nc, (double2*)out);
  return cudaGetLastError();
}

}  // namespace rpa
