// Tensor-core (tcgen05, BF16) contractions of the mixed-precision path.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "rpa_internal.h"

namespace rpa {
namespace tc {

struct Workspace {
  void* slices = nullptr;     // sliced BF16 operand planes
  size_t slice_bytes = 0;
  void* exps = nullptr;       // per-row power-of-two scales of the sliced operands
  size_t exp_bytes = 0;
  void* acc = nullptr;        // FP64 accumulation target
  size_t acc_bytes = 0;
  int* status = nullptr;      // device error word of the bounded waits
};

rpa_status alloc_workspace(Workspace& w, size_t max_g, size_t max_eig, size_t max_vc,
                           size_t max_freq);
void free_workspace(Workspace& w);

rpa_status chi0(Workspace& w, const void* A, int dtype, int n_vc, int n_g, const double* sf,
                const double* sv, double scale, cplx* chi, cudaStream_t st, std::string& err, int* launches);
rpa_status project(Workspace& w, const void* A, int dtype, int n_vc, int n_g, const cplx* B,
                   int n_eig, cplx* mt, cudaStream_t st, std::string& err, int* launches);
rpa_status chis(Workspace& w, const cplx* mt, int n_eig, int n_vc, const double* delta,
                const double* omega, int n_freq, double scale, cplx* out, cudaStream_t st,
                std::string& err, int* launches);

}  // namespace tc
}  // namespace rpa
