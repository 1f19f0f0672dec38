// Building blocks of the subspace step (a3, Method: the N_eig eigenvectors of chi~(0))
// exposed through the C ABI, so that each can be checked on its own: the Householder
// tridiagonalisation that starts the eigensolver, and the Jacobi eigensolver of its
// Rayleigh-Ritz step.  Both allocate their scratch per call and synchronise.
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
