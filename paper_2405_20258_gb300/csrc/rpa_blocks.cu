// Building blocks exposed through the C ABI, so that each can be checked on its own:
// the Householder tridiagonalisation that starts the subspace eigensolver (a3, Method:
// the N_eig eigenvectors of chi~(0)), the Jacobi eigensolver of its Rayleigh-Ritz
// step, and the transition order of the mixed path's chi~(0) K-blocks.  Each
// allocates its scratch per call and synchronises.
#include <cuda_runtime.h>

#include <string>

#include "rpa_dense.h"
#include "rpa_internal.h"

namespace {

rpa_status fail(rpa_status s, const std::string& msg) {
  rpa::set_call_error(msg.c_str());
  return s;
}

// Reads the kernel's barrier status after the stream has drained.
rpa_status finish_call(rpa_status s, const int* status_dev, cudaStream_t st, const char* what,
                       std::string& err) {
  if (s != RPA_OK) return s;
  int status = 0;
  if (cudaMemcpyAsync(&status, status_dev, sizeof(int), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    err = std::string(what) + ": " + cudaGetErrorString(cudaGetLastError());
    return RPA_ECUDA;
  }
  if (status != 0) {
    err = std::string(what) + ": a grid barrier gave up waiting";
    return RPA_ETIMEOUT;
  }
  return RPA_OK;
}

}  // namespace

extern "C" rpa_status rpa_tridiagonalize(int n, int bits, void* a, void* d, void* e,
                                         void* stream) {
  using namespace rpa::dense;
  if (n < 1 || (bits != 32 && bits != 64) || !a || !d || (n > 1 && !e))
    return fail(RPA_EINVAL, "rpa_tridiagonalize: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t elem = bits == 64 ? 16 : 8;
  std::string err;
  HetrdWork w;
  rpa_status s = hetrd_alloc(w, n, elem, err);
  if (s != RPA_OK) return fail(s, err);
  void* tau = nullptr;
  if (cudaMalloc(&tau, (size_t)n * elem) != cudaSuccess) {
    (void)cudaGetLastError();
    hetrd_free(w);
    return fail(RPA_ENOMEM, "rpa_tridiagonalize: cudaMalloc failed");
  }
  s = bits == 64 ? hetrd<double>(w, a, n, (double*)d, (double*)e, tau, st, err, nullptr)
                 : hetrd<float>(w, a, n, (float*)d, (float*)e, tau, st, err, nullptr);
  s = finish_call(s, w.status, st, "rpa_tridiagonalize", err);
  cudaFree(tau);
  hetrd_free(w);
  return s == RPA_OK ? RPA_OK : fail(s, err);
}

extern "C" rpa_status rpa_hermitian_eig_jacobi(int m, void* g, double* theta, void* y,
                                               void* stream) {
  using namespace rpa::dense;
  if (m < 1 || !g || !theta || !y)
    return fail(RPA_EINVAL, "rpa_hermitian_eig_jacobi: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  std::string err;
  JacobiWork w;
  rpa_status s = jacobi_alloc(w, m, err);
  if (s != RPA_OK) return fail(s, err);
  rpa::cplx* ywork = nullptr;
  if (cudaMalloc(&ywork, sizeof(rpa::cplx) * (size_t)m * m) != cudaSuccess) {
    (void)cudaGetLastError();
    jacobi_free(w);
    return fail(RPA_ENOMEM, "rpa_hermitian_eig_jacobi: cudaMalloc failed");
  }
  s = jacobi(w, (rpa::cplx*)g, m, theta, (rpa::cplx*)y, ywork, st, err, nullptr);
  s = finish_call(s, w.status, st, "rpa_hermitian_eig_jacobi", err);
  cudaFree(ywork);
  jacobi_free(w);
  return s == RPA_OK ? RPA_OK : fail(s, err);
}

extern "C" rpa_status rpa_transition_order(int n, int n_v, int n_c, int seg_bands,
                                           const double* delta, const double* ow, int* order,
                                           void* stream) {
  if (n < 1 || n_v < 1 || n_c < 1 || seg_bands < 0 || seg_bands > n_v || !delta || !ow ||
      !order || (seg_bands > 0 && n % ((long)n_v * n_c) != 0))
    return fail(RPA_EINVAL, "rpa_transition_order: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  void* items = nullptr;
  if (cudaMalloc(&items, 16 * (size_t)rpa::order_items(n)) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(RPA_ENOMEM, "rpa_transition_order: cudaMalloc failed");
  }
  cudaError_t e =
      rpa::launch_transition_order(delta, ow, n, n_v, n_c, seg_bands, items, order, st, nullptr);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(items);
  if (e != cudaSuccess)
    return fail(RPA_ECUDA, std::string("rpa_transition_order: ") + cudaGetErrorString(e));
  return RPA_OK;
}
