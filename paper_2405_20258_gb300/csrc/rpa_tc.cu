// Tensor-core (tcgen05) contractions of the mixed-precision path.
#include "rpa_tc.h"

namespace rpa {
namespace tc {

rpa_status alloc_workspace(Workspace& w, size_t, size_t, size_t, size_t) {
  w = Workspace{};
  return RPA_EINVAL;
}

void free_workspace(Workspace& w) {
  if (w.slices) cudaFree(w.slices);
  if (w.exps) cudaFree(w.exps);
  if (w.acc) cudaFree(w.acc);
  if (w.status) cudaFree(w.status);
  w = Workspace{};
}

rpa_status chi0(Workspace&, const void*, int, int, int, const double*, const double*, double,
                cplx*, cudaStream_t, std::string& err, int*) {
  err = "mixed-precision path not available";
  return RPA_EINVAL;
}
rpa_status project(Workspace&, const void*, int, int, int, const cplx*, int, cplx*, cudaStream_t,
                   std::string& err, int*) {
  err = "mixed-precision path not available";
  return RPA_EINVAL;
}
rpa_status chis(Workspace&, const cplx*, int, int, const double*, const double*, int, double,
                cplx*, cudaStream_t, std::string& err, int*) {
  err = "mixed-precision path not available";
  return RPA_EINVAL;
}

}  // namespace tc
}  // namespace rpa
