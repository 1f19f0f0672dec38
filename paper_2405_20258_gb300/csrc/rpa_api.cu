// C ABI of the static-subspace RPA path: plan life cycle, argument checks,
// stage ordering, workspace, and the FP64 eigensolves (cuSOLVER).
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "rpa_eig.h"
#include "rpa_internal.h"
#include "rpa_tc.h"

using rpa::cplx;

namespace {


thread_local std::string g_create_error;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

namespace rpa {
void set_call_error(const char* msg) { g_create_error = msg; }
}  // namespace rpa

struct rpa_plan_s {
  int n_q = 0;
  std::vector<rpa_qpoint> q;
  rpa_options opt{};
  cudaStream_t st = nullptr;
  cusolverDnHandle_t sol = nullptr;
  cusolverDnParams_t params = nullptr;
  // The plan holds one q-point's intermediates per stage: the q-point whose
  // scalars (v^1/2, Delta, pair weights), chi~(0), basis (C, B) and chi_s stage
  // outputs (M~, chi_s, traces) are resident (-1: none).  A stage checks that the
  // previous stage's outputs are those of its own q-point.
  int scalars_iq = -1, chi_iq = -1, basis_iq = -1, freq_iq = -1;
  std::string err;
  int max_g = 0, max_eig = 0, max_freq = 0;
  long max_vc = 0;
  // device workspace
  double *sv = nullptr, *delta = nullptr, *sf0 = nullptr, *w = nullptr, *ow = nullptr;
  double* fall = nullptr;  // [max_freq][max_vc] transition weights (mixed path's FP64 diagonal)
  int* order = nullptr;    // [max_vc] transitions sorted by sqrt f(0) (mixed path's chi~ blocks)
  void* order_scratch = nullptr;  // the device sort's items (order_items(max_vc) x 16 bytes)
  double *omega = nullptr, *weight = nullptr;  // [n_q][max_freq]
  double *lam_all = nullptr, *lam = nullptr, *trace = nullptr, *ec = nullptr, *logdet = nullptr;
  int* flags = nullptr;  // [0] bad-input bits, [1] numeric bits, [2] solver info
  cplx *chi = nullptr, *chi_work = nullptr, *C = nullptr, *B = nullptr, *mt = nullptr;
  cplx *chis = nullptr, *chis_work = nullptr;
  cplx* chol_inv = nullptr;   // inverses of the diagonal tiles of the tiled Cholesky
  void* gen_a = nullptr;      // device-drawn A for q-points with m == NULL
  int gen_iq = -1;            // which q-point gen_a currently holds
  void* sol_dev = nullptr;
  size_t sol_dev_bytes = 0;
  void* sol_host = nullptr;
  size_t sol_host_bytes = 0;
  bool batched_eig = false;   // cusolverDnXsyevBatched usable for the chi_s eigenvalues
  int* infos = nullptr;       // [max_freq] solver info of the batched solve
  rpa::tc::Workspace tcw;     // tensor-core path workspace
  rpa::HostReader reader;     // small host reads outside the copy engines
  rpa::eig::Refine refine;    // the library's own eigensolver of chi~ (rpa_eig.cu)
  bool refine_ready = false;
  // stage timers (CUDA events on the plan stream) and the library's launch count
  struct Pending {
    int id;
    cudaEvent_t a, b;
  };
  std::vector<cudaEvent_t> ev_pool;
  std::vector<Pending> pending;
  cudaEvent_t open_ev[RPA_N_TIMERS] = {};
  long long launches = 0;
};

namespace {

rpa_status fail(rpa_plan_t p, rpa_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (p)
    p->err = buf;
  else
    g_create_error = buf;
  return s;
}

#define CU(p, call)                                                                     \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(p, RPA_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                                  \
  } while (0)

#define CS(p, call)                                                                     \
  do {                                                                                  \
    cusolverStatus_t s_ = (call);                                                       \
    if (s_ != CUSOLVER_STATUS_SUCCESS)                                                  \
      return fail(p, RPA_EEIG, "%s failed: cusolver status %d", #call, (int)s_);        \
  } while (0)

template <typename T>
rpa_status dalloc(rpa_plan_t p, T** ptr, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)ptr, count * sizeof(T));
  if (e != cudaSuccess) {
    *ptr = nullptr;
    (void)cudaGetLastError();
    return fail(p, RPA_ENOMEM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                cudaGetErrorString(e));
  }
  return RPA_OK;
}

void free_plan(rpa_plan_t p) {
  if (!p) return;
  for (auto& e : p->pending) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  for (auto e : p->open_ev)
    if (e) cudaEventDestroy(e);
  for (auto e : p->ev_pool) cudaEventDestroy(e);
  void* bufs[] = {p->sv,   p->delta, p->sf0,       p->w,     p->ow,    p->omega, p->weight,
                  p->lam_all,
                  p->lam,  p->trace, p->ec,        p->logdet, p->flags, p->chi,   p->chi_work,
                  p->C,    p->B,     p->mt,        p->chis,  p->chis_work, p->gen_a, p->sol_dev,
                  p->infos, p->fall, p->order, p->order_scratch, p->chol_inv};
  for (void* b : bufs)
    if (b) cudaFree(b);
  rpa::tc::free_workspace(p->tcw);
  p->refine.release();
  rpa::reader_free(p->reader);
  if (p->sol_host) free(p->sol_host);
  if (p->params) cusolverDnDestroyParams(p->params);
  if (p->sol) cusolverDnDestroy(p->sol);
  delete p;
}

cudaEvent_t get_event(rpa_plan_t p) {
  if (!p->ev_pool.empty()) {
    cudaEvent_t e = p->ev_pool.back();
    p->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Records a pair of events around one stage when the plan times its stages.
struct StageTimer {
  rpa_plan_t p;
  int id;
  cudaEvent_t a = nullptr;
  StageTimer(rpa_plan_t p_, int id_) : p(p_), id(id_) {
    if (p->opt.timing && (a = get_event(p))) cudaEventRecord(a, p->st);
  }
  ~StageTimer() {
    if (!a) return;
    cudaEvent_t b = get_event(p);
    if (!b) {
      p->ev_pool.push_back(a);
      return;
    }
    cudaEventRecord(b, p->st);
    p->pending.push_back({id, a, b});
  }
};

// Timing hook used by the tensor-core path: begin/end marks of one timer id.
void mark_event(void* ctx, int id, int begin) {
  rpa_plan_t p = (rpa_plan_t)ctx;
  if (!p->opt.timing || id < 0 || id >= RPA_N_TIMERS) return;
  if (begin) {
    if (!p->open_ev[id] && (p->open_ev[id] = get_event(p))) cudaEventRecord(p->open_ev[id], p->st);
  } else if (p->open_ev[id]) {
    cudaEvent_t b = get_event(p);
    if (b) {
      cudaEventRecord(b, p->st);
      p->pending.push_back({id, p->open_ev[id], b});
    } else {
      p->ev_pool.push_back(p->open_ev[id]);
    }
    p->open_ev[id] = nullptr;
  }
}

rpa_status check_qpoint(const rpa_qpoint& q, int i) {
  auto bad = [&](const char* what) {
    return fail(nullptr, RPA_EINVAL, "q-point %d: %s", i, what);
  };
  if (q.n_g < 1) return bad("n_g must be >= 1");
  if (q.n_v < 1 || q.n_c < 1) return bad("n_v and n_c must be >= 1");
  if (q.n_k < 0) return bad("n_k must be >= 0");
  if (rpa::n_transitions(q) > (1L << 31) - 1) return bad("n_k*n_v*n_c too large");
  if (q.coulomb != RPA_COULOMB_BARE && q.coulomb != RPA_COULOMB_SLAB)
    return bad("unknown coulomb kernel");
  if (q.coulomb == RPA_COULOMB_SLAB && (!q.qg_vec || !(q.slab_zc > 0.0)))
    return bad("the slab Coulomb kernel needs qg_vec and slab_zc > 0");
  if (q.n_eig < 1 || q.n_eig > q.n_g) return bad("n_eig must be in [1, n_g]");
  if (q.n_freq < 1 || q.n_freq > 256) return bad("n_freq must be in [1, 256]");
  if (!(q.omega_cell > 0.0) || !std::isfinite(q.omega_cell)) return bad("omega_cell must be > 0");
  if (!q.qg2 || !q.e_v || !q.e_c) return bad("qg2, e_v and e_c must be device pointers");
  if (q.m_dtype != RPA_C128 && q.m_dtype != RPA_C64) return bad("unknown m_dtype");
  if (!q.m && !q.miller) return bad("m == NULL needs miller indices for the generator");
  return RPA_OK;
}

const rpa_qpoint* qp(rpa_plan_t p, int iq) { return &p->q[iq]; }

rpa_status check_iq(rpa_plan_t p, int iq) {
  if (!p) return RPA_EINVAL;
  if (iq < 0 || iq >= p->n_q) return fail(p, RPA_EINVAL, "iq %d out of range [0, %d)", iq, p->n_q);
  return RPA_OK;
}

// A of q-point iq, drawing it on the device when the caller passed none.
rpa_status matrix_a(rpa_plan_t p, int iq, const void** a, int* dtype) {
  const rpa_qpoint& q = p->q[iq];
  if (!q.m && p->opt.vc_chunk > 0)
    return fail(p, RPA_EINVAL, "q-point %d is drawn in chunks: A is never whole", iq);
  if (q.m) {
    *a = q.m;
    *dtype = q.m_dtype;
    return RPA_OK;
  }
  if (p->gen_iq != iq) {
    StageTimer t(p, RPA_T_OTHER);
    const int n_k = q.n_k > 1 ? q.n_k : 1;
    const size_t blk = (size_t)q.n_v * q.n_c * q.n_g * (q.m_dtype == RPA_C64 ? 8 : 16);
    for (int k = 0; k < n_k; ++k) {
      // k-point k draws the generator's band indices k*n_v + v and k*n_c + c
      CU(p, rpa::launch_generate_m(&q, k * q.n_v, q.n_v, k * q.n_c, q.n_c,
                                   (char*)p->gen_a + k * blk, q.m_dtype, p->st));
      p->launches += 1;
    }
    p->gen_iq = iq;
  }
  *a = p->gen_a;
  *dtype = q.m_dtype;
  return RPA_OK;
}

// Streaming (options.vc_chunk > 0, m == NULL): A is drawn again per chunk of whole
// valence bands of one k-point, rows [r0, r0 + rows) of A.
struct Chunk {
  long r0;
  int rows, k, v0, nv;
};

bool streamed(rpa_plan_t p, int iq) { return !p->q[iq].m && p->opt.vc_chunk > 0; }

int chunk_bands(const rpa_qpoint& q, int vc_chunk) {
  return std::max(1, std::min(q.n_v, vc_chunk / q.n_c));
}

std::vector<Chunk> chunks_of(const rpa_qpoint& q, int vc_chunk) {
  std::vector<Chunk> out;
  const int n_k = q.n_k > 1 ? q.n_k : 1, nvb = chunk_bands(q, vc_chunk);
  for (int k = 0; k < n_k; ++k)
    for (int v0 = 0; v0 < q.n_v; v0 += nvb) {
      const int nv = std::min(nvb, q.n_v - v0);
      out.push_back(Chunk{((long)k * q.n_v + v0) * q.n_c, nv * q.n_c, k, v0, nv});
    }
  return out;
}

// Draw chunk c of q-point iq into the generator buffer.
rpa_status draw_chunk(rpa_plan_t p, int iq, const Chunk& c, const void** a, int* dtype) {
  const rpa_qpoint& q = p->q[iq];
  {
    StageTimer t(p, RPA_T_OTHER);
    CU(p, rpa::launch_generate_m(&q, c.k * q.n_v + c.v0, c.nv, c.k * q.n_c, q.n_c, p->gen_a,
                                 q.m_dtype, p->st));
  }
  p->launches += 1;
  p->gen_iq = -1;  // the buffer holds a chunk, not the whole A
  *a = p->gen_a;
  *dtype = q.m_dtype;
  return RPA_OK;
}

// A tensor-core kernel that gave up on a bounded wait leaves a code in the
// status word; report it (and clear it) at the next host synchronisation.
rpa_status tc_status(rpa_plan_t p) {
  if (!p->tcw.status) return RPA_OK;
  int code = 0;
  const rpa::ReadPiece rp = {p->tcw.status, &code, sizeof(int)};
  CU(p, rpa::read_to_host(p->reader, &rp, 1, p->st));
  if (code == 0) return RPA_OK;
  CU(p, cudaMemsetAsync(p->tcw.status, 0, sizeof(int), p->st));
  return fail(p, RPA_ETIMEOUT, "a tensor-core kernel gave up waiting (code %d)", code);
}

// Transitions of q-point iq ordered by decreasing f_vc(0) = 4 w/Delta (the
// permutation of a stable sort, sorted on the device from the scalars prepare()
// left for iq): the K-blocks of the tensor-core chi~(0) then group transitions of
// similar weight.  Recomputed on every call, since the caller may have copied a
// new q-point's inputs into the same entry; nothing crosses the host link.
rpa_status transition_order(rpa_plan_t p, int iq) {
  const rpa_qpoint& q = p->q[iq];
  if (p->scalars_iq != iq) return fail(p, RPA_ESTATE, "q-point %d: scalars not prepared", iq);
  const int nvb = streamed(p, iq) ? chunk_bands(q, p->opt.vc_chunk) : 0;
  int nl = 0;
  CU(p, rpa::launch_transition_order(p->delta, p->ow, rpa::n_transitions(q), q.n_v, q.n_c, nvb,
                                     p->order_scratch, p->order, p->st, &nl));
  p->launches += nl;
  return RPA_OK;
}

rpa_status prepare(rpa_plan_t p, int iq) {
  const rpa_qpoint& q = p->q[iq];
  p->scalars_iq = -1;
  CU(p, cudaMemsetAsync(p->flags, 0, 4 * sizeof(int), p->st));
  {
    StageTimer t(p, RPA_T_OTHER);
    CU(p, rpa::launch_prepare_scalars(q, p->sv, p->delta, p->ow, p->sf0, p->flags, p->st));
    p->launches += 1;
  }
  int h = 0;
  const rpa::ReadPiece rp = {p->flags, &h, sizeof(int)};
  CU(p, rpa::read_to_host(p->reader, &rp, 1, p->st));
  if (h & 1) return fail(p, RPA_EINVAL, "q-point %d: |q+G|^2 must be finite and > 0", iq);
  if (h & 2) return fail(p, RPA_EINVAL, "q-point %d: e_c[c] - e_v[v] must be finite", iq);
  if (h & 4)
    return fail(p, RPA_EINVAL,
                "q-point %d: pair weights g_k (f_v - f_c) must be finite, of the sign of "
                "e_c - e_v, and zero where e_c = e_v",
                iq);
  if (h & 8) return fail(p, RPA_EINVAL, "q-point %d: slab Coulomb kernel not positive", iq);
  p->scalars_iq = iq;
  return RPA_OK;
}

// The per-q-point scalars of iq, recomputed if another q-point's replaced them.
rpa_status ensure_scalars(rpa_plan_t p, int iq) {
  return p->scalars_iq == iq ? RPA_OK : prepare(p, iq);
}

// chi~(0) of a q-point drawn in chunks: every chunk's contribution added into chi
// (tensor-core K-blocks of the chunk's sorted transitions, or FP64 atomics), and
// the mixed path's FP64 diagonal summed over the chunks.
rpa_status chi0_streamed(rpa_plan_t p, int iq, double scale) {
  const rpa_qpoint& q = p->q[iq];
  const long n_vc = rpa::n_transitions(q);
  const std::vector<Chunk> ch = chunks_of(q, p->opt.vc_chunk);
  const bool mixed = p->opt.precision != RPA_FP64;
  const char* dg = getenv("RPA_TC_CHI0_DIAG");
  const bool diag = mixed && !(dg && dg[0] == '0');
  rpa_status s;
  if (mixed && (s = transition_order(p, iq)) != RPA_OK) return s;
  if (!mixed) CU(p, cudaMemsetAsync(p->chi, 0, sizeof(cplx) * (size_t)q.n_g * q.n_g, p->st));
  for (size_t ci = 0; ci < ch.size(); ++ci) {
    const Chunk& c = ch[ci];
    const void* A = nullptr;
    int dt = 0;
    if ((s = draw_chunk(p, iq, c, &A, &dt)) != RPA_OK) return s;
    if (mixed) {
      int nl = 0;
      const int blocks =
          std::max(1, (int)std::lround((double)p->tcw.chi0_blocks * c.rows / (double)n_vc));
      s = rpa::tc::chi0(p->tcw, A, dt, c.rows, q.n_g, p->sf0 + c.r0, p->order + c.r0, p->sv,
                        scale, p->chi, p->st, p->err, &nl, ci == 0, blocks);
      p->launches += nl;
      if (s != RPA_OK) return s;
      if (diag) {
        StageTimer t(p, RPA_T_CHI0);
        CU(p, rpa::launch_chi0_diagonal(A, dt, c.rows, q.n_g, p->sf0 + c.r0, p->sv, scale,
                                        (double*)p->chi_work, 2 * (size_t)q.n_g * q.n_g, p->chi,
                                        p->st, (int)ci, (int)ch.size()));
        p->launches += 2;
      }
    } else {
      StageTimer t(p, RPA_T_CHI0);
      CU(p, rpa::launch_herk_fp64(A, dt, c.rows, q.n_g, p->sf0 + c.r0, p->sv, scale, p->chi,
                                  p->st, true));
      p->launches += 1;
    }
  }
  return RPA_OK;
}

// M~ of a q-point drawn in chunks: the columns of every chunk's transitions.
rpa_status project_streamed(rpa_plan_t p, int iq) {
  const rpa_qpoint& q = p->q[iq];
  const long n_vc = rpa::n_transitions(q);
  rpa_status s;
  for (const Chunk& c : chunks_of(q, p->opt.vc_chunk)) {
    const void* A = nullptr;
    int dt = 0;
    if ((s = draw_chunk(p, iq, c, &A, &dt)) != RPA_OK) return s;
    if (p->opt.precision != RPA_FP64) {
      int nl = 0;
      s = rpa::tc::project(p->tcw, A, dt, c.rows, q.n_g, p->B, q.n_eig, p->mt + c.r0, p->st,
                           p->err, &nl, n_vc);
      p->launches += nl;
      if (s != RPA_OK) return s;
    } else {
      StageTimer t(p, RPA_T_PROJ);
      CU(p, rpa::launch_project_fp64(A, dt, c.rows, q.n_g, p->B, q.n_eig, p->mt + c.r0, p->st,
                                     n_vc));
      p->launches += 1;
    }
  }
  return RPA_OK;
}

}  // namespace

extern "C" {

const char* rpa_version(void) { return "gb300-rpa 0.1 (sm_103a)"; }

const char* rpa_status_string(int s) {
  switch (s) {
    case RPA_OK: return "ok";
    case RPA_EINVAL: return "invalid argument";
    case RPA_ENOMEM: return "out of memory";
    case RPA_ECUDA: return "CUDA error";
    case RPA_EEIG: return "eigensolver failure";
    case RPA_ENUMERIC: return "numerical failure";
    case RPA_ETIMEOUT: return "device wait timed out";
    case RPA_ESTATE: return "stage called out of order";
    default: return "unknown status";
  }
}

const char* rpa_last_error(rpa_plan_t p) { return p ? p->err.c_str() : g_create_error.c_str(); }

rpa_status rpa_plan_create(rpa_plan_t* out, const rpa_qpoint* q, int n_q, const rpa_options* opt,
                           void* stream) {
  if (!out) return fail(nullptr, RPA_EINVAL, "out is NULL");
  *out = nullptr;
  if (!q || n_q < 1) return fail(nullptr, RPA_EINVAL, "need n_q >= 1 q-point descriptors");
  rpa_options o{};
  o.precision = RPA_FP64;
  o.energy_route = RPA_ROUTE_CHOLESKY;
  o.omega_scale = 0.5;
  if (opt) o = *opt;
  if (!(o.omega_scale > 0.0)) o.omega_scale = 0.5;
  if (o.precision < RPA_FP64 || o.precision > RPA_MIXED_TF32X3)
    return fail(nullptr, RPA_EINVAL, "unknown precision %d", o.precision);
  if (o.energy_route != RPA_ROUTE_EIG && o.energy_route != RPA_ROUTE_CHOLESKY)
    return fail(nullptr, RPA_EINVAL, "unknown energy route %d", o.energy_route);
  if (o.vc_chunk < 0) return fail(nullptr, RPA_EINVAL, "vc_chunk must be >= 0");
  for (int sl : {o.slices_chi0, o.slices_proj, o.slices_chis})
    if (sl < 0 || sl > rpa::tc::MAX_SLICES)
      return fail(nullptr, RPA_EINVAL, "digit slices must be in [0, %d]", rpa::tc::MAX_SLICES);
  for (int i = 0; i < n_q; ++i) {
    rpa_status s = check_qpoint(q[i], i);
    if (s != RPA_OK) return s;
  }
  rpa_plan_t p = new rpa_plan_s();
  p->n_q = n_q;
  p->q.assign(q, q + n_q);
  p->opt = o;
  p->st = (cudaStream_t)stream;
  bool need_gen = false;
  size_t gen_bytes = 0;
  for (int i = 0; i < n_q; ++i) {
    p->max_g = std::max(p->max_g, q[i].n_g);
    p->max_eig = std::max(p->max_eig, q[i].n_eig);
    p->max_freq = std::max(p->max_freq, q[i].n_freq);
    long nvc = rpa::n_transitions(q[i]);
    p->max_vc = std::max(p->max_vc, nvc);
    if (!q[i].m) {
      need_gen = true;
      const size_t rows = o.vc_chunk > 0 ? (size_t)chunk_bands(q[i], o.vc_chunk) * q[i].n_c
                                         : (size_t)nvc;
      gen_bytes = std::max(gen_bytes, rows * q[i].n_g * (q[i].m_dtype == RPA_C64 ? 8 : 16));
    }
  }
  rpa_status s;
#define ALLOC(ptr, n)                                                  \
  do {                                                                 \
    s = dalloc(nullptr, &p->ptr, (size_t)(n));                         \
    if (s != RPA_OK) {                                                 \
      free_plan(p);                                                    \
      return s;                                                        \
    }                                                                  \
  } while (0)
  const size_t G = p->max_g, E = p->max_eig, F = p->max_freq, V = p->max_vc;
  ALLOC(sv, G);
  ALLOC(delta, V);
  ALLOC(sf0, V);
  ALLOC(w, V);
  ALLOC(ow, V);
  ALLOC(omega, (size_t)n_q * F);
  ALLOC(weight, (size_t)n_q * F);
  ALLOC(lam_all, G);
  ALLOC(lam, F * E);
  ALLOC(trace, F);
  ALLOC(ec, 1);
  ALLOC(logdet, F);
  ALLOC(flags, 4);
  ALLOC(chi, G * G);
  ALLOC(chi_work, G * G);
  ALLOC(C, G * E);
  ALLOC(B, G * E);
  ALLOC(mt, E * V);
  ALLOC(chis, F * E * E);
  ALLOC(chis_work, F * E * E);
  ALLOC(chol_inv, rpa::cholesky_scratch_count((int)F));
#undef ALLOC
  if (need_gen) {
    cudaError_t e = cudaMalloc(&p->gen_a, gen_bytes);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      free_plan(p);
      return fail(nullptr, RPA_ENOMEM, "generator buffer of %zu bytes: %s", gen_bytes,
                  cudaGetErrorString(e));
    }
  }
  if (o.precision != RPA_FP64) {
    rpa::tc::Slices sl;
    // the split precisions: every contraction on round-to-nearest BF16 hi/lo planes
    // (2 planes, 3 products; or 3 planes, 6 products) summed in FP32
    const bool tf32 = o.precision == RPA_MIXED_TF32X3;
    const bool split = o.precision == RPA_MIXED_BF16X3 || o.precision == RPA_MIXED_BF16X6 || tf32;
    // TF32 planes take 4 bytes an element: the workspace is sized for twice the planes
    if (split) sl.chi0 = sl.proj = sl.chis = o.precision == RPA_MIXED_BF16X6 ? 3 : (tf32 ? 4 : 2);
    if (o.slices_chi0 > 0) sl.chi0 = o.slices_chi0;
    if (o.slices_proj > 0) sl.proj = o.slices_proj;
    if (o.slices_chis > 0) sl.chis = o.slices_chis;
    std::string e;
    s = rpa::tc::alloc_workspace(p->tcw, G, E, V, F, sl, e);
    if (s != RPA_OK) {
      free_plan(p);
      return fail(nullptr, s, "tensor-core workspace: %s", e.c_str());
    }
    p->tcw.debug_stall = o.debug_stall;
    p->tcw.split = split ? 1 : 0;
    p->tcw.tf32 = tf32 ? 1 : 0;
    if (tf32) p->tcw.slices.chi0 = p->tcw.slices.proj = p->tcw.slices.chis = 2;
    if (dalloc(nullptr, &p->fall, F * V) != RPA_OK || dalloc(nullptr, &p->order, V) != RPA_OK ||
        dalloc(nullptr, (char**)&p->order_scratch, 16 * (size_t)rpa::order_items(V)) != RPA_OK) {
      free_plan(p);
      return RPA_ENOMEM;
    }
    p->tcw.hook.ctx = p;
    p->tcw.hook.mark = mark_event;
  }
  if (rpa::reader_alloc(p->reader, 4096) != cudaSuccess) {
    (void)cudaGetLastError();
    free_plan(p);
    return fail(nullptr, RPA_ENOMEM, "mapped host buffer of 4 KB");
  }
  if (cusolverDnCreate(&p->sol) != CUSOLVER_STATUS_SUCCESS ||
      cusolverDnCreateParams(&p->params) != CUSOLVER_STATUS_SUCCESS) {
    free_plan(p);
    return fail(nullptr, RPA_ECUDA, "cusolverDnCreate failed");
  }
  cusolverDnSetStream(p->sol, p->st);
  // solver workspace: range eigensolve of chi~ and eigenvalue-only solves of chi_s
  size_t dmax = 0, hmax = 0;
  for (int i = 0; i < n_q; ++i) {
    size_t db = 0, hb = 0;
    double vl = 0, vu = 0;
    int64_t meig = 0;
    if (cusolverDnXsyevdx_bufferSize(p->sol, p->params, CUSOLVER_EIG_MODE_VECTOR,
                                     CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_LOWER, q[i].n_g,
                                     CUDA_C_64F, p->chi_work, q[i].n_g, &vl, &vu, 1, q[i].n_eig,
                                     &meig, CUDA_R_64F, p->lam_all, CUDA_C_64F, &db,
                                     &hb) != CUSOLVER_STATUS_SUCCESS) {
      free_plan(p);
      return fail(nullptr, RPA_EEIG, "cusolverDnXsyevdx_bufferSize failed");
    }
    dmax = std::max(dmax, db);
    hmax = std::max(hmax, hb);
    if (cusolverDnXsyevd_bufferSize(p->sol, p->params, CUSOLVER_EIG_MODE_NOVECTOR,
                                    CUBLAS_FILL_MODE_LOWER, q[i].n_eig, CUDA_C_64F, p->chis_work,
                                    q[i].n_eig, CUDA_R_64F, p->lam, CUDA_C_64F, &db,
                                    &hb) != CUSOLVER_STATUS_SUCCESS) {
      free_plan(p);
      return fail(nullptr, RPA_EEIG, "cusolverDnXsyevd_bufferSize failed");
    }
    dmax = std::max(dmax, db);
    hmax = std::max(hmax, hb);
  }
  // batched eigenvalue solve of all chi_s(w_k) of a q-point, when the library offers it
  p->batched_eig = true;
  for (int i = 0; i < n_q && p->batched_eig; ++i) {
    size_t db = 0, hb = 0;
    if (cusolverDnXsyevBatched_bufferSize(p->sol, p->params, CUSOLVER_EIG_MODE_NOVECTOR,
                                          CUBLAS_FILL_MODE_LOWER, q[i].n_eig, CUDA_C_64F,
                                          p->chis_work, q[i].n_eig, CUDA_R_64F, p->lam,
                                          CUDA_C_64F, &db, &hb,
                                          q[i].n_freq) != CUSOLVER_STATUS_SUCCESS) {
      p->batched_eig = false;
      break;
    }
    dmax = std::max(dmax, db);
    hmax = std::max(hmax, hb);
  }
  if (dalloc(nullptr, &p->infos, (size_t)F) != RPA_OK) {
    free_plan(p);
    return RPA_ENOMEM;
  }
  p->sol_dev_bytes = std::max<size_t>(dmax, 16);
  p->sol_host_bytes = std::max<size_t>(hmax, 16);
  if (cudaMalloc(&p->sol_dev, p->sol_dev_bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    free_plan(p);
    return fail(nullptr, RPA_ENOMEM, "solver workspace of %zu bytes", dmax);
  }
  p->sol_host = malloc(p->sol_host_bytes);
  if (!rpa::eig::use_library()) {
    int n_max = 0, mp_max = 0;
    bool with32 = false;
    for (int i = 0; i < n_q; ++i) {
      n_max = std::max(n_max, q[i].n_g);
      mp_max = std::max(mp_max, rpa::eig::block_size(q[i].n_g, q[i].n_eig));
      with32 = with32 || (o.precision != RPA_FP64 && rpa::eig::start32(q[i].n_g, q[i].n_eig));
    }
    std::string e;
    rpa_status rs = p->refine.alloc(n_max, mp_max, with32, e);
    if (rs != RPA_OK) {
      free_plan(p);
      return fail(nullptr, rs, "%s", e.c_str());
    }
    p->refine_ready = true;
  }
  // quadrature of every q-point
  for (int i = 0; i < n_q; ++i) {
    if (rpa::launch_freq_grid(q[i].n_freq, o.omega_scale, p->omega + (size_t)i * F,
                              p->weight + (size_t)i * F, p->st) != cudaSuccess) {
      free_plan(p);
      return fail(nullptr, RPA_ECUDA, "frequency grid launch failed");
    }
  }
  if (cudaStreamSynchronize(p->st) != cudaSuccess) {
    free_plan(p);
    return fail(nullptr, RPA_ECUDA, "stream synchronize failed during plan creation");
  }
  *out = p;
  return RPA_OK;
}

rpa_status rpa_plan_destroy(rpa_plan_t p) {
  if (!p) return RPA_EINVAL;
  if (p->st) cudaStreamSynchronize(p->st);
  free_plan(p);
  return RPA_OK;
}

rpa_status rpa_plan_frequencies(rpa_plan_t p, int iq, double* omega_host, double* weight_host) {
  rpa_status s = check_iq(p, iq);
  if (s != RPA_OK) return s;
  if (!omega_host || !weight_host) return fail(p, RPA_EINVAL, "NULL output");
  size_t F = p->max_freq, n = p->q[iq].n_freq;
  CU(p, cudaMemcpyAsync(omega_host, p->omega + iq * F, n * sizeof(double), cudaMemcpyDeviceToHost,
                        p->st));
  CU(p, cudaMemcpyAsync(weight_host, p->weight + iq * F, n * sizeof(double),
                        cudaMemcpyDeviceToHost, p->st));
  CU(p, cudaStreamSynchronize(p->st));
  return RPA_OK;
}

rpa_status rpa_chi0_static(rpa_plan_t p, int iq, void* chi_out) {
  rpa_status s = check_iq(p, iq);
  if (s != RPA_OK) return s;
  const rpa_qpoint& q = *qp(p, iq);
  p->chi_iq = -1;
  s = prepare(p, iq);
  if (s != RPA_OK) return s;
  const long n_vc = rpa::n_transitions(q);
  const double scale = -1.0 / q.omega_cell;
  if (streamed(p, iq)) {
    if ((s = chi0_streamed(p, iq, scale)) != RPA_OK) return s;
  } else {
  const void* A;
  int dt;
  s = matrix_a(p, iq, &A, &dt);
  if (s != RPA_OK) return s;
  if (p->opt.precision != RPA_FP64) {
    int nl = 0;
    if ((s = transition_order(p, iq)) != RPA_OK) return s;
    s = rpa::tc::chi0(p->tcw, A, dt, (int)n_vc, q.n_g, p->sf0, p->order, p->sv, scale, p->chi,
                      p->st, p->err, &nl);
    p->launches += nl;
    if (s != RPA_OK) return s;
    const char* dg = getenv("RPA_TC_CHI0_DIAG");
    if (!(dg && dg[0] == '0')) {
      // the diagonal in FP64 (RPA_TC_CHI0_DIAG=0 leaves the sliced GEMM's): the
      // digit pairs the GEMM drops bias it; chi_work is free until the eigensolve
      StageTimer t(p, RPA_T_CHI0);
      CU(p, rpa::launch_chi0_diagonal(A, dt, n_vc, q.n_g, p->sf0, p->sv, scale,
                                      (double*)p->chi_work, 2 * (size_t)q.n_g * q.n_g, p->chi,
                                      p->st));
      p->launches += 2;
    }
  } else {
    StageTimer t(p, RPA_T_CHI0);
    CU(p, rpa::launch_herk_fp64(A, dt, (int)n_vc, q.n_g, p->sf0, p->sv, scale, p->chi, p->st));
    p->launches += 1;
  }
  }
  {
    StageTimer t(p, RPA_T_OTHER);
    CU(p, rpa::launch_mirror_hermitian(p->chi, q.n_g, 1, p->st));
    p->launches += 1;
  }
  if (chi_out)
    CU(p, cudaMemcpyAsync(chi_out, p->chi, sizeof(cplx) * (size_t)q.n_g * q.n_g,
                          cudaMemcpyDeviceToDevice, p->st));
  p->chi_iq = iq;
  return RPA_OK;
}

rpa_status rpa_subspace_basis(rpa_plan_t p, int iq, double* lambda_out, void* c_out) {
  rpa_status s = check_iq(p, iq);
  if (s != RPA_OK) return s;
  if (p->chi_iq != iq)
    return fail(p, RPA_ESTATE, "rpa_chi0_static(%d) must come first (chi~ held: q-point %d)", iq,
                p->chi_iq);
  if ((s = ensure_scalars(p, iq)) != RPA_OK) return s;
  p->basis_iq = -1;
  const rpa_qpoint& q = *qp(p, iq);
  const int n = q.n_g;
  const bool mixed = p->opt.precision != RPA_FP64;
  const bool refine_here = p->refine_ready && !rpa::eig::use_library();
  // the projection's A planes are cut on the side stream during the eigensolve (whose
  // own tensor-core products use a workspace of their own)
  if (mixed && !streamed(p, iq)) {
    const void* A;
    int dt, nl = 0;
    if ((s = matrix_a(p, iq, &A, &dt)) != RPA_OK) return s;
    s = rpa::tc::project_prepare(p->tcw, A, dt, (int)rpa::n_transitions(q), n, p->st, p->err,
                                 &nl);
    p->launches += nl;
    if (s != RPA_OK) return s;
  }
  StageTimer timer(p, RPA_T_EIG0);
  bool refined = false;
  if (refine_here) {
    // own eigensolver (rpa_eig.cu): FP32 (mixed plans, n >= 1024) or FP64 tridiagonal
    // start, FP64 tridiagonal eigenpairs, Cholesky-QR2 and Rayleigh-Ritz; the
    // eigenvectors land where the library solver would leave them, for the gauge kernel
    int nl = 0;
    s = p->refine.subspace(p->chi, n, q.n_eig, p->lam_all, p->chi_work, p->chi_work, mixed,
                           p->st, p->err, &nl);
    p->launches += nl;
    if (s != RPA_OK && s != RPA_ENUMERIC) return s;
    refined = s == RPA_OK;  // RPA_ENUMERIC: a degenerate spectrum, the library solver takes it
  }
  if (refined) {
    if (mixed && (s = rpa::tc::join_side(p->tcw, p->st, p->err)) != RPA_OK) return s;
    CU(p, cudaStreamSynchronize(p->st));
    if ((s = tc_status(p)) != RPA_OK) return s;
  } else {
    CU(p, cudaMemcpyAsync(p->chi_work, p->chi, sizeof(cplx) * (size_t)n * n,
                          cudaMemcpyDeviceToDevice, p->st));
    double vl = 0.0, vu = 0.0;
    int64_t meig = 0;
    CU(p, cudaMemsetAsync(p->flags + 2, 0, sizeof(int), p->st));
    // The row-major Hermitian chi~ read column-major is conj(chi~): same eigenvalues,
    // conjugated eigenvectors, undone by the gauge kernel.
    CS(p, cusolverDnXsyevdx(p->sol, p->params, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I,
                            CUBLAS_FILL_MODE_LOWER, n, CUDA_C_64F, p->chi_work, n, &vl, &vu, 1,
                            q.n_eig, &meig, CUDA_R_64F, p->lam_all, CUDA_C_64F, p->sol_dev,
                            p->sol_dev_bytes, p->sol_host, p->sol_host_bytes, p->flags + 2));
    int info = 0;
    CU(p, cudaMemcpyAsync(&info, p->flags + 2, sizeof(int), cudaMemcpyDeviceToHost, p->st));
    if (p->opt.precision != RPA_FP64 &&
        (s = rpa::tc::join_side(p->tcw, p->st, p->err)) != RPA_OK)
      return s;
    CU(p, cudaStreamSynchronize(p->st));
    if ((s = tc_status(p)) != RPA_OK) return s;
    if (info != 0) return fail(p, RPA_EEIG, "Xsyevdx info = %d", info);
    if (meig != q.n_eig) return fail(p, RPA_EEIG, "Xsyevdx returned %lld of %d eigenpairs",
                                     (long long)meig, q.n_eig);
  }
  CU(p, rpa::launch_gauge(p->chi_work, n, n, q.n_eig, p->sv, p->C, p->B, p->st));
  p->launches += 1;
  if (lambda_out)
    CU(p, cudaMemcpyAsync(lambda_out, p->lam_all, sizeof(double) * q.n_eig,
                          cudaMemcpyDeviceToDevice, p->st));
  if (c_out)
    CU(p, cudaMemcpyAsync(c_out, p->C, sizeof(cplx) * (size_t)n * q.n_eig,
                          cudaMemcpyDeviceToDevice, p->st));
  p->basis_iq = iq;
  return RPA_OK;
}

rpa_status rpa_chi_freq(rpa_plan_t p, int iq, void* mt_out, void* chis_out, double* trace_out) {
  rpa_status s = check_iq(p, iq);
  if (s != RPA_OK) return s;
  if (p->basis_iq != iq)
    return fail(p, RPA_ESTATE, "rpa_subspace_basis(%d) must come first (basis held: q-point %d)",
                iq, p->basis_iq);
  if ((s = ensure_scalars(p, iq)) != RPA_OK) return s;
  p->freq_iq = -1;
  const rpa_qpoint& q = *qp(p, iq);
  const void* A = nullptr;
  int dt = 0;
  const bool strm = streamed(p, iq);
  if (strm) {
    if ((s = project_streamed(p, iq)) != RPA_OK) return s;
  } else if ((s = matrix_a(p, iq, &A, &dt)) != RPA_OK) {
    return s;
  }
  const int n_vc = (int)rpa::n_transitions(q), E = q.n_eig, F = q.n_freq;
  const double scale = -1.0 / q.omega_cell;
  const double* om = p->omega + (size_t)iq * p->max_freq;
  if (p->opt.precision != RPA_FP64) {
    int nl = 0;
    if (!strm) {
      s = rpa::tc::project(p->tcw, A, dt, n_vc, q.n_g, p->B, E, p->mt, p->st, p->err, &nl);
      if (s != RPA_OK) return s;
    }
    {
      StageTimer t(p, RPA_T_TRACE);
      CU(p, rpa::launch_all_freq_weights(p->delta, p->ow, n_vc, om, F, p->fall, p->st));
      p->launches += 1;
    }
    s = rpa::tc::chis(p->tcw, p->mt, E, n_vc, p->fall, F, scale, p->chis, p->st, p->err, &nl);
    if (s != RPA_OK) return s;
    p->launches += nl;
    {
      // the diagonal of every chi_s in FP64: the rounding of the digit-sliced
      // products then leaves Tr chi_s exact and moves E_c only at second order
      StageTimer t(p, RPA_T_TRACE);
      CU(p, rpa::launch_chis_diagonal(p->mt, E, n_vc, p->fall, F, scale, p->chis, p->st));
      p->launches += 1;
    }
  } else {
    if (!strm) {
      StageTimer t(p, RPA_T_PROJ);
      CU(p, rpa::launch_project_fp64(A, dt, n_vc, q.n_g, p->B, E, p->mt, p->st));
    }
    {
      StageTimer t(p, RPA_T_CHIS);
      CU(p, rpa::launch_chis_fp64(p->mt, E, n_vc, p->delta, p->ow, om, F, scale, p->chis,
                                  p->st));
    }
    p->launches += 2;
  }
  {
    StageTimer t(p, RPA_T_OTHER);
    CU(p, rpa::launch_mirror_hermitian(p->chis, E, F, p->st));
  }
  {
    StageTimer t(p, RPA_T_TRACE);
    CU(p, rpa::launch_trace(p->mt, E, n_vc, p->delta, p->ow, om, F, scale, p->w, p->trace,
                            p->st));
  }
  p->launches += 3;
  if (mt_out)
    CU(p, cudaMemcpyAsync(mt_out, p->mt, sizeof(cplx) * (size_t)E * n_vc, cudaMemcpyDeviceToDevice,
                          p->st));
  if (chis_out)
    CU(p, cudaMemcpyAsync(chis_out, p->chis, sizeof(cplx) * (size_t)F * E * E,
                          cudaMemcpyDeviceToDevice, p->st));
  if (trace_out)
    CU(p, cudaMemcpyAsync(trace_out, p->trace, sizeof(double) * F, cudaMemcpyDeviceToDevice,
                          p->st));
  p->freq_iq = iq;
  return RPA_OK;
}

static rpa_status energy_one(rpa_plan_t p, int iq, double* ec_host, double* lam_out) {
  const rpa_qpoint& q = *qp(p, iq);
  const int E = q.n_eig, F = q.n_freq;
  const double* wt = p->weight + (size_t)iq * p->max_freq;
  CU(p, cudaMemsetAsync(p->flags, 0, 4 * sizeof(int), p->st));
  if (p->opt.energy_route == RPA_ROUTE_CHOLESKY) {
    {
      StageTimer t(p, RPA_T_EIGS);
      int nl = 0;
      CU(p, rpa::launch_cholesky_logdet(p->chis_work, p->chis, E, F, p->logdet, p->flags + 1,
                                        p->chol_inv, p->st, &nl));
      p->launches += nl;
    }
    StageTimer t(p, RPA_T_ENERGY);
    CU(p, rpa::launch_logdet_sum(p->logdet, F, p->trace, wt, p->ec, p->flags + 1, p->st));
    p->launches += 1;
  } else {
    {
      StageTimer t(p, RPA_T_EIGS);
      CU(p, cudaMemcpyAsync(p->chis_work, p->chis, sizeof(cplx) * (size_t)F * E * E,
                            cudaMemcpyDeviceToDevice, p->st));
      bool done = false;
      if (p->batched_eig) {
        CU(p, cudaMemsetAsync(p->infos, 0, sizeof(int) * F, p->st));
        cusolverStatus_t cs = cusolverDnXsyevBatched(
            p->sol, p->params, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, E, CUDA_C_64F,
            p->chis_work, E, CUDA_R_64F, p->lam, CUDA_C_64F, p->sol_dev, p->sol_dev_bytes,
            p->sol_host, p->sol_host_bytes, p->infos, F);
        if (cs == CUSOLVER_STATUS_SUCCESS) {
          done = true;
        } else {
          p->batched_eig = false;  // fall back to one solve per frequency from now on
          CU(p, cudaMemcpyAsync(p->chis_work, p->chis, sizeof(cplx) * (size_t)F * E * E,
                                cudaMemcpyDeviceToDevice, p->st));
        }
      }
      if (!done) {
        CU(p, cudaMemsetAsync(p->infos, 0, sizeof(int) * F, p->st));
        for (int k = 0; k < F; ++k) {
          CS(p, cusolverDnXsyevd(p->sol, p->params, CUSOLVER_EIG_MODE_NOVECTOR,
                                 CUBLAS_FILL_MODE_LOWER, E, CUDA_C_64F,
                                 p->chis_work + (size_t)k * E * E, E, CUDA_R_64F,
                                 p->lam + (size_t)k * E, CUDA_C_64F, p->sol_dev, p->sol_dev_bytes,
                                 p->sol_host, p->sol_host_bytes, p->infos + k));
        }
      }
    }
    {
      StageTimer t(p, RPA_T_ENERGY);
      CU(p, rpa::launch_logsum(p->lam, E, E, F, p->trace, wt, p->ec, p->flags + 1, p->st));
    }
    p->launches += 1;
    if (lam_out)
      CU(p, cudaMemcpyAsync(lam_out, p->lam, sizeof(double) * (size_t)F * E,
                            cudaMemcpyDeviceToDevice, p->st));
  }
  int fl[4];
  {
    const rpa::ReadPiece rp[2] = {{p->flags, fl, sizeof fl}, {p->ec, ec_host, sizeof(double)}};
    CU(p, rpa::read_to_host(p->reader, rp, 2, p->st));
  }
  rpa_status ts = tc_status(p);
  if (ts != RPA_OK) return ts;
  if (p->opt.energy_route == RPA_ROUTE_EIG) {
    std::vector<int> info(F);
    CU(p, cudaMemcpy(info.data(), p->infos, sizeof(int) * F, cudaMemcpyDeviceToHost));
    for (int k = 0; k < F; ++k)
      if (info[k] != 0) return fail(p, RPA_EEIG, "eigenvalues of chi_s(%d): info = %d", k, info[k]);
  }
  if (fl[1] != 0)
    return fail(p, RPA_ENUMERIC, "energy of q-point %d: 1 - lambda <= 0 or non-finite (bits %d)",
                iq, fl[1]);
  return RPA_OK;
}

rpa_status rpa_ecorr(rpa_plan_t p, int iq, double* ec_host, double* lam_out) {
  if (!p) return RPA_EINVAL;
  if (!ec_host) return fail(p, RPA_EINVAL, "ec_host is NULL");
  if (iq == -1) {
    for (int i = 0; i < p->n_q; ++i) {
      rpa_status s;
      if ((s = rpa_chi0_static(p, i, nullptr)) != RPA_OK) return s;
      if ((s = rpa_subspace_basis(p, i, nullptr, nullptr)) != RPA_OK) return s;
      if ((s = rpa_chi_freq(p, i, nullptr, nullptr, nullptr)) != RPA_OK) return s;
      if ((s = energy_one(p, i, ec_host + i, nullptr)) != RPA_OK) return s;
    }
    return RPA_OK;
  }
  rpa_status s = check_iq(p, iq);
  if (s != RPA_OK) return s;
  if (p->freq_iq != iq)
    return fail(p, RPA_ESTATE, "rpa_chi_freq(%d) must come first (chi_s held: q-point %d)", iq,
                p->freq_iq);
  return energy_one(p, iq, ec_host, lam_out);
}

rpa_status rpa_plan_timings(rpa_plan_t p, double* times_ms, long long* launches) {
  if (!p) return RPA_EINVAL;
  CU(p, cudaStreamSynchronize(p->st));
  double acc[RPA_N_TIMERS] = {0};
  for (auto& e : p->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess && e.id >= 0 && e.id < RPA_N_TIMERS)
      acc[e.id] += ms;
    p->ev_pool.push_back(e.a);
    p->ev_pool.push_back(e.b);
  }
  p->pending.clear();
  if (times_ms)
    for (int i = 0; i < RPA_N_TIMERS; ++i) times_ms[i] = acc[i];
  if (launches) *launches = p->launches;
  p->launches = 0;
  return RPA_OK;
}

rpa_status rpa_generate_m(const rpa_qpoint* q, int v0, int nv, int c0, int nc, void* out,
                          int dtype, void* stream) {
  if (!q || !out || !q->miller || !q->qg2) return fail(nullptr, RPA_EINVAL, "NULL argument");
  if (q->n_g < 1 || nv < 0 || nc < 0 || v0 < 0 || c0 < 0)
    return fail(nullptr, RPA_EINVAL, "bad generator range");
  if (dtype != RPA_C128 && dtype != RPA_C64) return fail(nullptr, RPA_EINVAL, "unknown dtype");
  if ((long)nv * nc == 0) return RPA_OK;
  cudaError_t e = rpa::launch_generate_m(q, v0, nv, c0, nc, out, dtype, (cudaStream_t)stream);
  if (e != cudaSuccess)
    return fail(nullptr, RPA_ECUDA, "generator launch failed: %s", cudaGetErrorString(e));
  return RPA_OK;
}

}  // extern "C"
