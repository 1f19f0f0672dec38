// Tensor-core (tcgen05, BF16) contractions of the mixed-precision path.
//
// Every contraction D = A B^T (real, K-major operands) is evaluated on exact
// digit slices: each operand row r is scaled by 2^-e_r (e_r from the row's
// largest magnitude) and cut into S signed 8-bit integer digits, so
//   x = 2^(e_r - 7) * sum_s d_s 2^(-8 s),   |d_s| <= 128  (exact in BF16).
// Digit products are exact; the FP32 sums of the leading levels s + t < Le over
// a drain interval of K are exact (integers below 2^24 times the level weight),
// the lower levels share one FP32 accumulator, and the epilogue folds each
// interval into a double-float accumulator.  The approximations are the
// truncation of the digit expansion and of the product triangle
// (s + t <= S - 1), about 2^-(7 + 8(S-1)) relative to the row scales, and the
// rounding of the low-level accumulator below it.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "rpa_internal.h"

namespace rpa {
namespace tc {

constexpr int MAX_SLICES = 8;
// Digit planes of the eigensolver's block products on the projection GEMM: products
// exact to ~2^-55 of the row and column scales (its Rayleigh quotient resolves
// eigenvalues 1e-4 of the largest to FP64-class accuracy).
constexpr int EIG_SLICES = 7;

struct Slices {
  int chi0 = 4, proj = 6, chis = 3;
};

// Optional stage-timing hook: mark(ctx, timer id, 1) before and (.., 0) after
// a group of launches.
struct Hook {
  void* ctx = nullptr;
  void (*mark)(void* ctx, int id, int begin) = nullptr;
  void operator()(int id, int begin) const {
    if (mark) mark(ctx, id, begin);
  }
};

struct Workspace {
  void* planes = nullptr;     // BF16 digit planes (largest stage)
  size_t plane_bytes = 0;
  void* planes2 = nullptr;    // second operand planes (projection B, chi_s A)
  size_t plane2_bytes = 0;
  int* exps = nullptr;        // per-row exponents
  size_t exp_count = 0;
  unsigned long long* rowmax = nullptr;  // per-row max |x| (double bits)
  size_t rowmax_count = 0;
  int4* work = nullptr;       // tile work lists (each distinct list uploaded once)
  size_t work_count = 0, work_used = 0;
  std::vector<std::pair<std::vector<int4>, size_t>> work_cache;  // list, offset in `work`
  int* status = nullptr;      // device error word of the bounded waits
  float* fweights = nullptr;  // transition weights f(omega_k) rounded up to FP32, [n_freq][n_vc]
  size_t fweight_count = 0;
  Slices slices;
  int freq_group = 8;         // frequencies per chi_s GEMM launch
  long proj_chunk = 0;        // rows of A whose projection planes are cut at a time
  bool chis_overlap = true;   // cut the chi_s B planes on the side stream
  int chi0_blocks = 32;       // K-blocks of chi~(0) (transitions sorted by sqrt f(0))
  int split = 0;              // 1: round-to-nearest BF16 hi/lo split planes, FP32 sums over K
  int proj_slices_override = 0;  // > 0: slice count of project() (the eigensolver's products)
  int tf32 = 0;               // 1: planes of TF32 values (FP32 storage), kind::tf32 MMAs
  int debug_stall = 0;
  Hook hook;
  // Side stream for digit slicing that overlaps the GEMMs and the eigensolve
  // on the caller's stream.  ev_side_last marks the end of the latest batch of
  // side-stream work; the caller's stream waits on it before it writes the
  // shared planes, exponents or row maxima itself.
  cudaStream_t side = nullptr;
  cudaEvent_t ev_in = nullptr, ev_side_last = nullptr;
  cudaEvent_t ev_sliced[2] = {nullptr, nullptr}, ev_gemm[2] = {nullptr, nullptr};
  // Projection A planes cut ahead of time (valid while nothing else wrote the planes).
  struct {
    bool valid = false;
    const void* a = nullptr;
    int dtype = 0, n_vc = 0, n_g = 0, S = 0;
  } proj_a;
};

rpa_status alloc_workspace(Workspace& w, size_t max_g, size_t max_eig, size_t max_vc,
                           size_t max_freq, const Slices& s, std::string& err);
void free_workspace(Workspace& w);

// chi~(0) from the transitions in `order` (a permutation of 0..n_vc-1, device),
// processed in K-blocks with their own digit exponents (w.chi0_blocks, or `blocks`
// when > 0).  zero: chi is set to zero first; else the contributions are added
// (a q-point whose transitions arrive in chunks).
rpa_status chi0(Workspace& w, const void* A, int dtype, int n_vc, int n_g, const double* sf,
                const int* order, const double* sv, double scale, cplx* chi, cudaStream_t st,
                std::string& err, int* launches, bool zero = true, int blocks = 0);
// The caller's stream `st` waits for all side-stream work queued so far.
rpa_status join_side(Workspace& w, cudaStream_t st, std::string& err);

// Cut the projection's A operand (the rows of A) into the digit planes on the
// side stream, after the work queued so far on `st`, so that it overlaps the
// eigensolve that follows on `st`; the caller joins the side stream before it
// returns control to its user.  project() uses these planes when its A is
// the same and no other stage wrote the planes in between; otherwise it cuts
// them again.
rpa_status project_prepare(Workspace& w, const void* A, int dtype, int n_vc, int n_g,
                           cudaStream_t st, std::string& err, int* launches);
// mt[i][r] (row stride ld_out, n_vc when <= 0) = conj(sum_g A[r][g] B[g][i]) for the
// n_vc rows r of A.
rpa_status project(Workspace& w, const void* A, int dtype, int n_vc, int n_g, const cplx* B,
                   int n_eig, cplx* mt, cudaStream_t st, std::string& err, int* launches,
                   long ld_out = 0);
// chi_s(i omega_k) for all k from M~ and the transition weights f[k][vc] of every
// frequency (FP64, device).
rpa_status chis(Workspace& w, const cplx* mt, int n_eig, int n_vc, const double* f,
                int n_freq, double scale, cplx* out, cudaStream_t st, std::string& err,
                int* launches);

}  // namespace tc
}  // namespace rpa
