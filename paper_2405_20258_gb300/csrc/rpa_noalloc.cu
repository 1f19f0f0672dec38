// Allocation-free trace term.
//
// rpa_trace_term_static computes the same FP64 trace term as rpa_chi_freq,
//   T_k = -(1/Omega) sum_vc f_vc(w_k) |M~[:, vc]|^2,
// but without a plan and without allocating: its only scratch (the column
// norms |M~[:, vc]|^2) lives in the fixed device array below.  It exists for
// callers that cannot allocate device memory at the point of the call, for
// example applications whose memory is entirely reserved by their own pool
// allocator, or code that must not trigger the device-wide synchronisation
// that cudaMalloc and cudaFree can cause.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "rpa_internal.h"

namespace {

constexpr int kMaxVc = RPA_STATIC_TRACE_MAX_VC;

// Scratch of every call: the first n_vc entries hold |M~[:, vc]|^2 of the
// latest call.  Each call writes these entries before reading them, so
// nothing has to start at zero; calls that overlap on the GPU race on it.
__device__ __align__(256) double g_trace_scratch[kMaxVc];

// Device address of g_trace_scratch per device ordinal, looked up once per
// device (with that device current) on the first call made on it.
std::mutex g_mu;
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// w[vc] = sum_i |mt[i][vc]|^2
__global__ void colnorm_static_kernel(const double2* mt, int n_eig, int n_vc, double* w) {
  int vc = blockIdx.x * blockDim.x + threadIdx.x;
  if (vc >= n_vc) return;
  double s = 0.0;
  for (int i = 0; i < n_eig; ++i) {
    double2 m = mt[(size_t)i * n_vc + vc];
    s = fma(m.x, m.x, s);
    s = fma(m.y, m.y, s);
  }
  w[vc] = s;
}

// trace[k] = scale sum_vc f_k(vc) w[vc], f_k = 4 D/(D^2 + w_k^2), D = e_c[c] - e_v[v];
// one block of 1024 threads per frequency, fixed summation order.
__global__ void trace_static_kernel(const double* w, const double* e_v, const double* e_c,
                                    int n_c, int n_vc, const double* omega, double scale,
                                    double* trace) {
  __shared__ double sh[33];
  const int k = blockIdx.x;
  const double w2 = omega[k] * omega[k];
  double s = 0.0;
  for (int vc = threadIdx.x; vc < n_vc; vc += blockDim.x) {
    double d = e_c[vc % n_c] - e_v[vc / n_c];
    s += 4.0 * d / (d * d + w2) * w[vc];
  }
  s = warp_sum(s);
  const int wp = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[wp] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (int)(blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) trace[k] = scale * t;
  }
}

}  // namespace

extern "C" rpa_status rpa_trace_term_static(const void* mtilde, int n_eig, int n_v, int n_c,
                                            const double* e_v, const double* e_c,
                                            const double* omega, int n_freq, double omega_cell,
                                            double* trace_out, void* stream) {
  char msg[200];
  if (!mtilde || !e_v || !e_c || !omega || !trace_out) {
    rpa::set_call_error("rpa_trace_term_static: NULL pointer argument");
    return RPA_EINVAL;
  }
  if (n_eig < 1 || n_v < 1 || n_c < 1 || n_freq < 1 || !(omega_cell > 0.0)) {
    rpa::set_call_error("rpa_trace_term_static: n_eig, n_v, n_c, n_freq must be >= 1 and "
                        "omega_cell > 0");
    return RPA_EINVAL;
  }
  const long n_vc = (long)n_v * n_c;
  if (n_vc > kMaxVc) {
    snprintf(msg, sizeof msg,
             "rpa_trace_term_static: n_v*n_c = %ld exceeds the fixed scratch of %d transitions",
             n_vc, kMaxVc);
    rpa::set_call_error(msg);
    return RPA_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    rpa::set_call_error("rpa_trace_term_static: no usable current CUDA device");
    return RPA_ECUDA;
  }
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      // host code may not use g_trace_scratch's name as an address: ask the runtime
      e = cudaGetSymbolAddress(&g_scratch_addr[dev], g_trace_scratch);
      if (e != cudaSuccess) {
        g_scratch_addr[dev] = nullptr;
        snprintf(msg, sizeof msg, "rpa_trace_term_static: cudaGetSymbolAddress failed: %s",
                 cudaGetErrorString(e));
        rpa::set_call_error(msg);
        return RPA_ECUDA;
      }
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  colnorm_static_kernel<<<(unsigned)((n_vc + 255) / 256), 256, 0, st>>>(
      (const double2*)mtilde, n_eig, (int)n_vc, (double*)scratch);
  trace_static_kernel<<<n_freq, 1024, 0, st>>>((const double*)scratch, e_v, e_c, n_c, (int)n_vc,
                                               omega, -1.0 / omega_cell, trace_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(msg, sizeof msg, "rpa_trace_term_static: launch failed: %s", cudaGetErrorString(e));
    rpa::set_call_error(msg);
    return RPA_ECUDA;
  }
  return RPA_OK;
}
