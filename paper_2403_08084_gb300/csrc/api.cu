// C-ABI entry points and the host-side orchestration of one RK step:
// right-hand side, FP64 flexible GMRES with the block stage preconditioners of
// Sec. 3.1 (each diagonal block approximated by one geometric-multigrid V-cycle),
// and the RK update of Sec. 2.  See include/irk.h for the contract.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/irk.h"
#include "common.cuh"
#include "hierarchy.h"
#include "kernels.h"

using namespace irk;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(call)                                                                               \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return fail(IRK_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define CK_LAUNCH()                                                                                  \
  do {                                                                                               \
    cudaError_t e_ = cudaGetLastError();                                                             \
    if (e_ != cudaSuccess) return fail(IRK_ECUDA, "kernel launch failed: %s", cudaGetErrorString(e_)); \
  } while (0)

#define TRY(x)          \
  do {                  \
    int r_ = (x);       \
    if (r_ != IRK_OK) return r_; \
  } while (0)

// An NVTX range over a host scope: the entry points, the FGMRES solve and each Arnoldi step (host time
// of enqueueing; a profiler maps the kernels launched inside to it, e.g. ncu --nvtx --nvtx-include
// "irk_step/").  A no-op unless a tool is attached.
struct Nvtx {
  explicit Nvtx(const char* name) { nvtxRangePushA(name); }
  ~Nvtx() { nvtxRangePop(); }
  Nvtx(const Nvtx&) = delete;
  Nvtx& operator=(const Nvtx&) = delete;
};

size_t prec_bytes(int prec) { return prec == IRK_PREC_FP64 ? 8 : (prec == IRK_PREC_FP32 ? 4 : 2); }

struct Level {
  int N = 0, nx = 0, dim = 2;
  size_t nn = 0;
  double hm = 0.0;  // h^2 / 36 (2D mass stencil scale)
  double mcls[4] = {0, 0, 0, 0}, kcls[4] = {0, 0, 0, 0};  // 3D: Q1 mass / stiffness class values
  std::vector<double> cf_host;  // stencil records {D, E, N, NE, NW} per node (node-major)
  // device copies are planar (one plane of nn values per coefficient, see planar())
  double* cf_d = nullptr;     // stencil records, double
  float* cf_f = nullptr;      // stencil records, float
  double* brec_d = nullptr;   // FP64 V-cycles: records of M + dt a_ii K, stage-major
  float* brec_f = nullptr;    // FP32 / BF16 V-cycles: the same records in FP32
  double* mblk_d = nullptr;   // monolithic multigrid: omega (M_pp I + dt K_pp A)^{-1} per node (s x s planes)
  float* mblk_f = nullptr;
  // FP64 V-cycles, coarse levels with the large-tile legs: the scaled Jacobi stencils of the one-block
  // V-cycles (nine planes per stage, scaled_jacobi_records_2d)
  double* srec_d = nullptr;
  double* dinv_d = nullptr;   // omega / diag(B_i): node-major (s per node), then stage-major (nn per stage)
  float* dinv_f = nullptr;
  void* xa = nullptr;         // V-cycle vectors (s per node, V-cycle precision)
  void* xb = nullptr;
  void* b = nullptr;
  void* r = nullptr;
};

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct irk_handle {
  int dim = 2, N = 0, s = 0, L = 0;  // dim: 2 (quads, per-cell kappa) or 3 (hexahedra, kappa = 1)
  double dt = 0.0;
  irk_options opt{};
  cudaStream_t st = nullptr;
  std::vector<double> A, b, c, kappa;
  std::vector<double> Ap;  // the preconditioner's approximation of A: tril(A), or L D from A = L D U
  // IA form: A^{-1}, the preconditioner matrix T (D, L + D, U + D or L D), T^{-1}, and A^{-T} b
  std::vector<double> Ainv, Tm, Tinv, bIA;
  bool ainv_ok = false;  // A is invertible and Ainv holds A^{-1}
  std::vector<Level> lev;
  // coarsest-level exact solve
  int nint = 0;
  int* cmap = nullptr;
  double* binv_d = nullptr;
  float* binv_f = nullptr;
  double* kappa_d = nullptr;
  double* minv_d = nullptr;  // monolithic multigrid: dense inverse of the coupled coarsest system
  float* minv_f = nullptr;
  // Krylov space
  size_t ne = 0;  // entries of a stage vector
  int m = 0;
  double* V = nullptr;
  double* Z = nullptr;
  double *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr;
  double *h1 = nullptr, *h2 = nullptr, *partial = nullptr, *scal = nullptr;
  int* iflag = nullptr;  // device flags (re-orthogonalisation decision)
  double* pinned = nullptr;  // host-visible copies of the residual estimate
  double *rhs = nullptr, *k = nullptr, *tmp = nullptr;
  void* zt = nullptr;  // FP32 / BF16 triangular sweeps: the blocks' V-cycle outputs, stage-major, precision T
  double* bnd = nullptr;  // boundary unknowns of irk_step_dirichlet (allocated on first use)
  // FP64 triangular sweeps (2D, V(2, .) or V(., 2)): the finest level's scaled Jacobi stencils, nine planes per
  // stage block (scaled_jacobi_records_2d), and the current block's first sweep x1 = d b
  double* srec_d = nullptr;
  double* x1_d = nullptr;
  // IA form, 2D: per stage the planar records of A^{-1}_ii M + dt K (the stage operator's diagonal terms;
  // A^{-T} has the same diagonal, so the transposed operator uses them too)
  double* iarec_d = nullptr;
  DevBuf stage_bufs[8];
  int vcycles = 0;
  // one CUDA graph per FGMRES iteration index j and direction (captured on first use)
  struct IterGraph {
    cudaGraphExec_t exec = nullptr;
    irk_perf delta{};
    int vcycles = 0;
  };
  std::vector<IterGraph> graphs[2];
  std::vector<IterGraph> cg_graphs[2];  // one per stage and direction (DIRK solver)
  double *cg_x = nullptr, *cg_r = nullptr, *cg_z = nullptr, *cg_p = nullptr, *cg_q = nullptr, *cg_b = nullptr;
  cudaStream_t cap_stream = nullptr;
  bool use_graphs = true;
  // small-level V-cycle tails as one cooperative launch (mg2d_tail.cuh): barrier words and error flag
  unsigned* tail_state = nullptr;  // [0] arrivals, [1] generation, [2] error flag
  bool tail_on = false;
  bool tail_used = false;
  bool k_from_step = false;  // h->k holds the stage solution of the last forward irk_step (warm start)
  long long tail_spin = 2000000000LL;  // barrier wait limit, SM clock cycles (about one second)
  // instrumentation
  irk_perf perf{};
  unsigned perf_mask = 0;
  std::vector<cudaEvent_t> ev;  // start/stop pairs
  std::vector<int> ev_cls;
  size_t ev_used = 0;
};

namespace {

// ----------------------------------------------------------------------------
// memory helpers
// ----------------------------------------------------------------------------
// Allocation-failure injection (environment IRK_FAIL_DEVICE_ALLOC=n, read once per process): every n-th
// device allocation of the process fails with IRK_ENOMEM before cudaMalloc is called, so that the error
// paths (and their clean-up) can be exercised without exhausting the device.
long injected_failure_period() {
  static const long n = [] {
    const char* e = getenv("IRK_FAIL_DEVICE_ALLOC");
    return e ? atol(e) : 0L;
  }();
  return n;
}
std::atomic<long> g_device_allocs{0};

template <typename P>
int dalloc(P** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (const long n = injected_failure_period(); n > 0 && ++g_device_allocs % n == 0)
    return fail(IRK_ENOMEM, "device allocation of %zu bytes failed (injected by IRK_FAIL_DEVICE_ALLOC)", bytes);
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(IRK_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
  }
  return IRK_OK;
}

template <typename P>
void dfree(P*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

bool is_device_ptr(const void* p) {
  if (p == nullptr) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device view of a caller input: the pointer itself if it is device memory,
// else a copy in staging slot `slot` (enqueued on the handle's stream).
int dev_in(irk_handle* h, const void* p, size_t bytes, int slot, const void** out) {
  if (p == nullptr || is_device_ptr(p)) {
    *out = p;
    return IRK_OK;
  }
  DevBuf& b = h->stage_bufs[slot];
  if (b.bytes < bytes) {
    dfree(b.p);
    b.bytes = 0;
    TRY(dalloc(&b.p, bytes));
    b.bytes = bytes;
  }
  CK(cudaMemcpyAsync(b.p, p, bytes, cudaMemcpyHostToDevice, h->st));
  *out = b.p;
  return IRK_OK;
}

// Device destination for a caller output; *host is set when the result must be
// copied back to the caller's host memory with dev_out_finish.
int dev_out(irk_handle* h, void* p, size_t bytes, int slot, void** out, bool* host) {
  *host = false;
  if (p == nullptr || is_device_ptr(p)) {
    *out = p;
    return IRK_OK;
  }
  DevBuf& b = h->stage_bufs[slot];
  if (b.bytes < bytes) {
    dfree(b.p);
    b.bytes = 0;
    TRY(dalloc(&b.p, bytes));
    b.bytes = bytes;
  }
  *out = b.p;
  *host = true;
  return IRK_OK;
}

int dev_out_finish(irk_handle* h, void* host_ptr, const void* dev, size_t bytes) {
  CK(cudaMemcpyAsync(host_ptr, dev, bytes, cudaMemcpyDeviceToHost, h->st));
  return IRK_OK;
}

// ----------------------------------------------------------------------------
// instrumentation: launch counts, algorithmic bytes / flops, optional event timing
// ----------------------------------------------------------------------------
void perf_drain(irk_handle* h, bool accumulate) {
  if (h->ev_used == 0) return;
  cudaStreamSynchronize(h->st);
  for (size_t i = 0; i < h->ev_used; ++i) {
    float ms = 0.f;
    if (accumulate && cudaEventElapsedTime(&ms, h->ev[2 * i], h->ev[2 * i + 1]) == cudaSuccess)
      h->perf.timed_ms[h->ev_cls[i]] += ms;
  }
  cudaGetLastError();
  h->ev_used = 0;
}

int perf_slot(irk_handle* h, int cls) {
  constexpr size_t kMaxPairs = 8192;
  if (h->ev_used == h->ev.size() / 2) {
    if (h->ev.size() / 2 >= kMaxPairs) {
      perf_drain(h, true);
    } else {
      cudaEvent_t a, b;
      if (cudaEventCreate(&a) != cudaSuccess) return -1;
      if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return -1;
      }
      h->ev.push_back(a);
      h->ev.push_back(b);
      h->ev_cls.push_back(0);
    }
  }
  const size_t i = h->ev_used++;
  h->ev_cls[i] = cls;
  return (int)i;
}

// Counts one kernel launch of class `cls`; brackets it with events when selected.
struct KScope {
  irk_handle* h;
  int slot = -1;
  KScope(irk_handle* hh, int cls, double bytes, double flops) : h(hh) {
    h->perf.launches++;
    h->perf.class_launches[cls]++;
    h->perf.class_bytes[cls] += bytes;
    h->perf.class_flops[cls] += flops;
    if (h->perf_mask & (1u << cls)) {
      slot = perf_slot(h, cls);
      if (slot >= 0) {
        h->perf.timed_launches[cls]++;
        h->perf.timed_bytes[cls] += bytes;
        h->perf.timed_flops[cls] += flops;
        cudaEventRecord(h->ev[2 * slot], h->st);
      }
    }
  }
  ~KScope() {
    if (slot >= 0) cudaEventRecord(h->ev[2 * slot + 1], h->st);
  }
};

inline double n_int(int nx) { return (double)(nx - 2) * (double)(nx - 2); }

// ----------------------------------------------------------------------------
// setup
// ----------------------------------------------------------------------------
// Inverse of a small dense s x s matrix (Gauss-Jordan, partial pivoting); false if singular.
bool small_inverse(const std::vector<double>& A, int s, std::vector<double>& inv) {
  std::vector<double> B = A;
  inv.assign(s * s, 0.0);
  for (int i = 0; i < s; ++i) inv[i * s + i] = 1.0;
  double scale = 0.0;
  for (double v : A) scale = std::max(scale, std::fabs(v));
  for (int k = 0; k < s; ++k) {
    int piv = k;
    for (int r = k + 1; r < s; ++r)
      if (std::fabs(B[r * s + k]) > std::fabs(B[piv * s + k])) piv = r;
    if (!(std::fabs(B[piv * s + k]) > 1e-13 * scale)) return false;
    for (int c = 0; c < s; ++c) std::swap(B[k * s + c], B[piv * s + c]), std::swap(inv[k * s + c], inv[piv * s + c]);
    const double d = 1.0 / B[k * s + k];
    for (int c = 0; c < s; ++c) B[k * s + c] *= d, inv[k * s + c] *= d;
    for (int r = 0; r < s; ++r) {
      if (r == k) continue;
      const double f = B[r * s + k];
      for (int c = 0; c < s; ++c) B[r * s + c] -= f * B[k * s + c], inv[r * s + c] -= f * inv[k * s + c];
    }
  }
  return true;
}

int validate(const irk_mesh* mesh, const irk_tableau* tab, double dt, const irk_options* opt) {
  if (!mesh || !tab || !opt) return fail(IRK_EINVAL, "null mesh, tableau or options");
  if (mesh->dim != 2 && mesh->dim != 3) return fail(IRK_EINVAL, "dim = %d: must be 2 or 3", mesh->dim);
  if (mesh->dim == 3 && mesh->kappa) return fail(IRK_EINVAL, "dim = 3 supports kappa = 1 only (pass NULL)");
  const int N = mesh->n_cells, L = mesh->levels;
  if (N < 2 || N > 16384) return fail(IRK_EINVAL, "n_cells = %d out of range [2, 16384]", N);
  if (L < 1 || L > 14) return fail(IRK_EINVAL, "levels = %d out of range [1, 14]", L);
  const int div = 1 << (L - 1);
  if (N % div != 0) return fail(IRK_EINVAL, "n_cells = %d not divisible by 2^(levels-1) = %d", N, div);
  const int Nc = N / div;
  if (Nc < 2) return fail(IRK_EINVAL, "coarsest level has %d cells per axis (< 2)", Nc);
  if (mesh->dim == 2 && Nc > 64) return fail(IRK_EINVAL, "coarsest level has %d cells per axis (> 64): add levels", Nc);
  if (mesh->dim == 3 && Nc > 16) return fail(IRK_EINVAL, "coarsest level has %d cells per axis (> 16): add levels", Nc);
  if (mesh->dim == 3 && N > 1024) return fail(IRK_EINVAL, "n_cells = %d too large for dim = 3", N);
  if (mesh->kappa) {
    const size_t nc = (size_t)N * N;
    for (size_t i = 0; i < nc; ++i)
      if (!(mesh->kappa[i] > 0.0) || !std::isfinite(mesh->kappa[i]))
        return fail(IRK_EINVAL, "kappa[%zu] = %g is not positive and finite", i, mesh->kappa[i]);
  }
  const int s = tab->s;
  if (s < 1 || s > IRK_MAX_STAGES) return fail(IRK_EINVAL, "s = %d out of range [1, %d]", s, IRK_MAX_STAGES);
  if (!tab->A || !tab->b || !tab->c) return fail(IRK_EINVAL, "null tableau array");
  double bsum = 0.0;
  for (int i = 0; i < s; ++i) {
    double row = 0.0;
    for (int j = 0; j < s; ++j) {
      const double a = tab->A[i * s + j];
      if (!std::isfinite(a)) return fail(IRK_EINVAL, "A[%d][%d] is not finite", i, j);
      row += a;
    }
    if (!std::isfinite(tab->b[i]) || !std::isfinite(tab->c[i])) return fail(IRK_EINVAL, "b or c not finite");
    if (std::fabs(row - tab->c[i]) > 1e-6)
      return fail(IRK_EINVAL, "row %d of A sums to %.17g but c[%d] = %.17g (transposed A?)", i, row, i, tab->c[i]);
    bsum += tab->b[i];
  }
  if (std::fabs(bsum - 1.0) > 1e-6) return fail(IRK_EINVAL, "sum(b) = %.17g != 1", bsum);
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(IRK_EINVAL, "dt = %g must be positive", dt);
  if (opt->precond < IRK_PC_DIAG || opt->precond > IRK_PC_MONOLITHIC) return fail(IRK_EINVAL, "bad precond %d", opt->precond);
  if (opt->precond == IRK_PC_MONOLITHIC &&
      (mesh->dim != 2 || opt->splitting != IRK_SPLIT_AI || opt->solver != IRK_SOLVER_FGMRES))
    return fail(IRK_EINVAL, "monolithic multigrid is implemented for dim = 2, the AI splitting and FGMRES");
  if (opt->precond == IRK_PC_MONOLITHIC) {  // the coupled coarsest system is inverted densely
    const int m = mesh->n_cells / (1 << (mesh->levels - 1)) - 1;
    if ((long long)tab->s * m * m > 4096)
      return fail(IRK_EINVAL, "monolithic multigrid: the coupled coarsest system has %lld > 4096 unknowns; add levels",
                  (long long)tab->s * m * m);
  }
  if (opt->vcycle_prec < IRK_PREC_FP64 || opt->vcycle_prec > IRK_PREC_BF16)
    return fail(IRK_EINVAL, "bad vcycle_prec %d", opt->vcycle_prec);
  if (opt->nu_pre < 1 || opt->nu_post < 1 || opt->nu_pre > 16 || opt->nu_post > 16)
    return fail(IRK_EINVAL, "nu_pre / nu_post must be in [1, 16]");
  if (!(opt->omega > 0.0 && opt->omega < 2.0)) return fail(IRK_EINVAL, "omega = %g not in (0, 2)", opt->omega);
  if (!(opt->rtol > 0.0 && opt->rtol < 1.0)) return fail(IRK_EINVAL, "rtol = %g not in (0, 1)", opt->rtol);
  if (opt->restart < 1 || opt->restart > 100) return fail(IRK_EINVAL, "restart = %d not in [1, 100]", opt->restart);
  if (opt->maxit < 1) return fail(IRK_EINVAL, "maxit = %d < 1", opt->maxit);
  if (opt->orth != IRK_ORTH_CGS2 && opt->orth != IRK_ORTH_DGKS && opt->orth != IRK_ORTH_CGS)
    return fail(IRK_EINVAL, "bad orth %d", opt->orth);
  if (opt->solver != IRK_SOLVER_FGMRES && opt->solver != IRK_SOLVER_DIRK_CG)
    return fail(IRK_EINVAL, "bad solver %d", opt->solver);
  if (opt->splitting != IRK_SPLIT_AI && opt->splitting != IRK_SPLIT_IA)
    return fail(IRK_EINVAL, "bad splitting %d", opt->splitting);
  if (opt->warm_start != 0 && opt->warm_start != 1) return fail(IRK_EINVAL, "bad warm_start %d", opt->warm_start);
  if (opt->splitting == IRK_SPLIT_IA && opt->solver != IRK_SOLVER_FGMRES)
    return fail(IRK_EINVAL, "the IA splitting is implemented for the FGMRES solver");
  if (opt->solver == IRK_SOLVER_DIRK_CG) {
    for (int i = 0; i < s; ++i) {
      if (!(tab->A[i * s + i] > 0.0)) return fail(IRK_EINVAL, "DIRK solver needs a_ii > 0 (a_%d%d = %g)", i, i, tab->A[i * s + i]);
      for (int j = i + 1; j < s; ++j)
        if (tab->A[i * s + j] != 0.0) return fail(IRK_EINVAL, "DIRK solver needs a lower-triangular A (a_%d%d != 0)", i, j);
    }
  }
  return IRK_OK;
}

// Device copy of per-node host data: `aos` holds blocks of nn nodes x k values (node-major); the
// device layout is planar, value c of node q of block b at [(b k + c) nn + q] (coalesced warp loads).
template <typename D>
std::vector<D> planar(const std::vector<double>& aos, size_t nn, int k) {
  std::vector<D> out(aos.size());
  const size_t blocks = aos.size() / (nn * k);
  for (size_t b = 0; b < blocks; ++b)
    for (size_t q = 0; q < nn; ++q)
      for (int c = 0; c < k; ++c) out[(b * k + c) * nn + q] = (D)aos[(b * nn + q) * k + c];
  return out;
}

// Build the hierarchy's host data and upload it (also used by irk_set_kappa).
int build_operators_3d(irk_handle* h, const std::vector<double>& sigma) {
  const int s = h->s;
  for (Level& Lv : h->lev) q1_classes_3d(1.0 / Lv.N, Lv.mcls, Lv.kcls);
  Level& Lc = h->lev[h->L - 1];
  std::vector<int> map;
  interior_nodes_3d(Lc.N, map);
  const int nint = (int)map.size();
  std::vector<double> all((size_t)s * nint * nint), inv;
  for (int i = 0; i < s; ++i) {
    if (!dense_block_inverse_3d(Lc.N, Lc.mcls, Lc.kcls, sigma[i], map, inv))
      return fail(IRK_EINVAL, "coarsest block %d (sigma = %g) is singular", i, sigma[i]);
    std::copy(inv.begin(), inv.end(), all.begin() + (size_t)i * nint * nint);
  }
  std::vector<float> allf(all.begin(), all.end());
  CK(cudaMemcpyAsync(h->cmap, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice, h->st));
  CK(cudaMemcpyAsync(h->binv_d, all.data(), all.size() * 8, cudaMemcpyHostToDevice, h->st));
  CK(cudaMemcpyAsync(h->binv_f, allf.data(), allf.size() * 4, cudaMemcpyHostToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  return IRK_OK;
}

int build_operators(irk_handle* h) {
  const int s = h->s;
  std::vector<double> sigma(s);
  for (int i = 0; i < s; ++i) sigma[i] = h->dt * h->Ap[i * s + i];
  if (h->dim == 3) return build_operators_3d(h, sigma);
  for (int l = 0; l < h->L; ++l) {
    Level& Lv = h->lev[l];
    if (l == 0)
      stiffness_records_2d(Lv.N, h->kappa.empty() ? nullptr : h->kappa.data(), Lv.cf_host);
    else
      galerkin_coarsen_2d(h->lev[l - 1].N, h->lev[l - 1].cf_host, Lv.cf_host);
    std::vector<double> dinv;
    jacobi_inverse_diag_2d(Lv.N, Lv.cf_host, Lv.hm, sigma.data(), s, h->opt.omega, dinv);
    // the same values stage-major, for the one-block-at-a-time V-cycles of the triangular sweeps
    dinv.resize(2 * Lv.nn * s);
    for (size_t q = 0; q < Lv.nn; ++q)
      for (int i = 0; i < s; ++i) dinv[Lv.nn * s + (size_t)i * Lv.nn + q] = dinv[q * s + i];
    const std::vector<double> cfd = planar<double>(Lv.cf_host, Lv.nn, kCoef2);
    const std::vector<float> cff = planar<float>(Lv.cf_host, Lv.nn, kCoef2);
    std::vector<float> dinvf(dinv.begin(), dinv.end());
    CK(cudaMemcpyAsync(Lv.cf_d, cfd.data(), cfd.size() * 8, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(Lv.dinv_d, dinv.data(), dinv.size() * 8, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(Lv.cf_f, cff.data(), cff.size() * 4, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(Lv.dinv_f, dinvf.data(), dinvf.size() * 4, cudaMemcpyHostToDevice, h->st));
    if (Lv.mblk_d) {  // monolithic multigrid: stage-coupled point blocks of this level
      std::vector<double> blk;
      if (!mmg_block_inverses_2d(Lv.N, Lv.cf_host, Lv.hm, h->A.data(), s, h->dt, h->opt.omega, blk))
        return fail(IRK_EINVAL, "a point block M_pp I + dt K_pp A of level %d is singular", l);
      const std::vector<float> blkf = planar<float>(blk, Lv.nn, s * s);
      blk = planar<double>(blk, Lv.nn, s * s);
      CK(cudaMemcpyAsync(Lv.mblk_d, blk.data(), blk.size() * 8, cudaMemcpyHostToDevice, h->st));
      CK(cudaMemcpyAsync(Lv.mblk_f, blkf.data(), blkf.size() * 4, cudaMemcpyHostToDevice, h->st));
      CK(cudaStreamSynchronize(h->st));
    }
    std::vector<double> brec, srec;
    std::vector<float> brecf;
    if (Lv.brec_d || Lv.brec_f) block_records_2d(Lv.N, Lv.cf_host, Lv.hm, sigma.data(), s, brec);
    std::vector<double> iarec;
    if (l == 0 && h->iarec_d) {  // A^{-1}_ii M + dt K per stage; M's record is hm {16, 4, 4, 1, 1}
      const double mrec[kCoef2] = {16.0, 4.0, 4.0, 1.0, 1.0};
      iarec.resize(Lv.nn * kCoef2 * s);
      for (int i = 0; i < s; ++i) {
        const double am = h->Ainv[i * s + i] * Lv.hm;
        for (size_t q = 0; q < Lv.nn; ++q)
          for (int k = 0; k < kCoef2; ++k)
            iarec[((size_t)i * Lv.nn + q) * kCoef2 + k] = am * mrec[k] + h->dt * Lv.cf_host[q * kCoef2 + k];
      }
      iarec = planar<double>(iarec, Lv.nn, kCoef2);
      CK(cudaMemcpyAsync(h->iarec_d, iarec.data(), iarec.size() * 8, cudaMemcpyHostToDevice, h->st));
    }
    if (l >= 1 && Lv.srec_d) {  // coarse level with large-tile legs: its own scaled stencils
      std::vector<double> sl(9 * Lv.nn * s);
      for (int i = 0; i < s; ++i)
        scaled_jacobi_records_2d(Lv.N, brec.data() + (size_t)i * Lv.nn * kCoef2, dinv.data() + Lv.nn * s + (size_t)i * Lv.nn,
                                 sl.data() + (size_t)i * 9 * Lv.nn);
      srec.swap(sl);
      CK(cudaMemcpyAsync(Lv.srec_d, srec.data(), srec.size() * 8, cudaMemcpyHostToDevice, h->st));
    }
    if (l == 0 && h->srec_d) {
      srec.resize(9 * Lv.nn * s);
      for (int i = 0; i < s; ++i)
        scaled_jacobi_records_2d(Lv.N, brec.data() + (size_t)i * Lv.nn * kCoef2, dinv.data() + Lv.nn * s + (size_t)i * Lv.nn,
                                 srec.data() + (size_t)i * 9 * Lv.nn);
      CK(cudaMemcpyAsync(h->srec_d, srec.data(), srec.size() * 8, cudaMemcpyHostToDevice, h->st));
    }
    if (Lv.brec_f) brecf = planar<float>(brec, Lv.nn, kCoef2);
    if (Lv.brec_d) brec = planar<double>(brec, Lv.nn, kCoef2);
    if (Lv.brec_d) CK(cudaMemcpyAsync(Lv.brec_d, brec.data(), brec.size() * 8, cudaMemcpyHostToDevice, h->st));
    if (Lv.brec_f) {
      CK(cudaMemcpyAsync(Lv.brec_f, brecf.data(), brecf.size() * 4, cudaMemcpyHostToDevice, h->st));
    }
    CK(cudaStreamSynchronize(h->st));  // host vectors above go out of scope
  }
  // exact coarsest solve: dense inverse of each diagonal block
  Level& Lc = h->lev[h->L - 1];
  std::vector<int> map;
  interior_nodes_2d(Lc.N, map);
  const int nint = (int)map.size();
  std::vector<double> all((size_t)s * nint * nint), inv;
  for (int i = 0; i < s; ++i) {
    if (!dense_block_inverse_2d(Lc.N, Lc.cf_host, Lc.hm, sigma[i], map, inv))
      return fail(IRK_EINVAL, "coarsest block %d (sigma = %g) is singular", i, sigma[i]);
    std::copy(inv.begin(), inv.end(), all.begin() + (size_t)i * nint * nint);
  }
  std::vector<float> allf(all.begin(), all.end());
  if (h->minv_d) {  // monolithic multigrid: the coupled coarsest system
    std::vector<double> minv;
    if (!mmg_coarse_inverse_2d(Lc.N, Lc.cf_host, Lc.hm, h->A.data(), s, h->dt, minv))
      return fail(IRK_EINVAL, "the coupled coarsest system is singular");
    std::vector<float> minvf(minv.begin(), minv.end());
    CK(cudaMemcpyAsync(h->minv_d, minv.data(), minv.size() * 8, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(h->minv_f, minvf.data(), minvf.size() * 4, cudaMemcpyHostToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
  }
  CK(cudaMemcpyAsync(h->cmap, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice, h->st));
  CK(cudaMemcpyAsync(h->binv_d, all.data(), all.size() * 8, cudaMemcpyHostToDevice, h->st));
  CK(cudaMemcpyAsync(h->binv_f, allf.data(), allf.size() * 4, cudaMemcpyHostToDevice, h->st));
  if (!h->kappa.empty())
    CK(cudaMemcpyAsync(h->kappa_d, h->kappa.data(), h->kappa.size() * 8, cudaMemcpyHostToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  return IRK_OK;
}

void destroy(irk_handle* h) {
  if (!h) return;
  for (Level& Lv : h->lev) {
    dfree(Lv.cf_d), dfree(Lv.cf_f), dfree(Lv.brec_d), dfree(Lv.brec_f), dfree(Lv.dinv_d), dfree(Lv.dinv_f);
    dfree(Lv.mblk_d), dfree(Lv.mblk_f), dfree(Lv.srec_d);
    dfree(Lv.xa), dfree(Lv.xb), dfree(Lv.b), dfree(Lv.r);
  }
  dfree(h->cmap), dfree(h->binv_d), dfree(h->binv_f), dfree(h->kappa_d), dfree(h->minv_d), dfree(h->minv_f);
  dfree(h->V), dfree(h->Z), dfree(h->H), dfree(h->cs), dfree(h->sn), dfree(h->g), dfree(h->y);
  dfree(h->h1), dfree(h->h2), dfree(h->partial), dfree(h->scal), dfree(h->iflag);
  dfree(h->rhs), dfree(h->k), dfree(h->tmp), dfree(h->bnd), dfree(h->zt), dfree(h->srec_d), dfree(h->x1_d), dfree(h->iarec_d);
  for (DevBuf& b : h->stage_bufs) dfree(b.p);
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  for (auto& gv : h->graphs)
    for (auto& G : gv)
      if (G.exec) cudaGraphExecDestroy(G.exec);
  for (auto& gv : h->cg_graphs)
    for (auto& G : gv)
      if (G.exec) cudaGraphExecDestroy(G.exec);
  dfree(h->cg_x), dfree(h->cg_r), dfree(h->cg_z), dfree(h->cg_p), dfree(h->cg_q), dfree(h->cg_b);
  dfree(h->tail_state);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->pinned) cudaFreeHost(h->pinned);
  delete h;
}

int create(irk_handle** out, const irk_mesh* mesh, const irk_tableau* tab, double dt, const irk_options* opt,
           void* stream) {
  if (!out) return fail(IRK_EINVAL, "null output handle pointer");
  *out = nullptr;
  TRY(validate(mesh, tab, dt, opt));
  irk_handle* h = new irk_handle();
  h->N = mesh->n_cells;
  h->dim = mesh->dim;
  h->L = mesh->levels;
  h->s = tab->s;
  h->dt = dt;
  h->opt = *opt;
  h->st = (cudaStream_t)stream;
  const int s = h->s;
  h->A.assign(tab->A, tab->A + s * s);
  h->Ap = h->A;
  if (opt->precond == IRK_PC_RANA_LD) {
    // A = L D U (L unit lower, U unit upper, no pivoting); the preconditioner uses L D (Sec. 3.1, eq. pcranald)
    std::vector<double> Lm(s * s, 0.0), Um(s * s, 0.0);  // Doolittle: A = Lm Um, Um upper with diagonal D
    for (int i = 0; i < s; ++i) {
      for (int j = i; j < s; ++j) {
        double v = h->A[i * s + j];
        for (int k = 0; k < i; ++k) v -= Lm[i * s + k] * Um[k * s + j];
        Um[i * s + j] = v;
      }
      Lm[i * s + i] = 1.0;
      for (int r = i + 1; r < s; ++r) {
        double v = h->A[r * s + i];
        for (int k = 0; k < i; ++k) v -= Lm[r * s + k] * Um[k * s + i];
        if (Um[i * s + i] == 0.0) {
          destroy(h);
          return fail(IRK_EINVAL, "A has a zero leading principal minor: no L D U factorisation");
        }
        Lm[r * s + i] = v / Um[i * s + i];
      }
    }
    for (int i = 0; i < s; ++i)
      for (int j = 0; j < s; ++j) h->Ap[i * s + j] = (j <= i) ? Lm[i * s + j] * Um[j * s + j] : 0.0;
  }
  h->ainv_ok = small_inverse(h->A, s, h->Ainv);
  if (opt->splitting == IRK_SPLIT_IA) {
    if (!h->ainv_ok) {
      destroy(h);
      return fail(IRK_EINVAL, "the IA splitting needs an invertible Butcher matrix");
    }
    // T: the part of Ap the preconditioner keeps (D, L + D, U + D; Rana: L D is already lower triangular)
    h->Tm.assign(s * s, 0.0);
    for (int i = 0; i < s; ++i)
      for (int j = 0; j < s; ++j) {
        const bool keep = (i == j) || (opt->precond == IRK_PC_LOWER && j < i) ||
                          (opt->precond == IRK_PC_UPPER && j > i) || (opt->precond == IRK_PC_RANA_LD && j < i);
        if (keep && s > 1) h->Tm[i * s + j] = h->Ap[i * s + j];
        if (s == 1) h->Tm[0] = h->Ap[0];
      }
    if (!small_inverse(h->Tm, s, h->Tinv)) {
      destroy(h);
      return fail(IRK_EINVAL, "the IA preconditioner matrix is singular (a zero diagonal entry?)");
    }
    h->bIA.assign(s, 0.0);
    for (int j = 0; j < s; ++j)
      for (int i = 0; i < s; ++i) h->bIA[j] += tab->b[i] * h->Ainv[i * s + j];
  }
  h->b.assign(tab->b, tab->b + s);
  h->c.assign(tab->c, tab->c + s);
  if (mesh->kappa) h->kappa.assign(mesh->kappa, mesh->kappa + (size_t)h->N * h->N);
  const int dim = h->dim;
  auto bail = [&](int code) {
    destroy(h);
    return code;
  };
  const size_t vb = prec_bytes(opt->vcycle_prec);
  h->lev.resize(h->L);
  for (int l = 0; l < h->L; ++l) {
    Level& Lv = h->lev[l];
    Lv.N = h->N >> l;
    Lv.nx = Lv.N + 1;
    Lv.dim = dim;
    Lv.nn = (size_t)Lv.nx * Lv.nx * (dim == 3 ? Lv.nx : 1);
    const double hh = 1.0 / Lv.N;
    Lv.hm = hh * hh / 36.0;
    int r = IRK_OK;
    if (dim == 2) {  // stencil records (3D uses constant class values instead)
      // records of each diagonal block B_i = M + dt a_ii K, in the V-cycle's arithmetic precision
      if (opt->vcycle_prec == IRK_PREC_FP64 && (r = dalloc(&Lv.brec_d, Lv.nn * kCoef2 * s * 8))) return bail(r);
      if (opt->vcycle_prec != IRK_PREC_FP64 && (r = dalloc(&Lv.brec_f, Lv.nn * kCoef2 * s * 4))) return bail(r);
      if (opt->precond == IRK_PC_MONOLITHIC &&
          ((r = dalloc(&Lv.mblk_d, Lv.nn * s * s * 8)) || (r = dalloc(&Lv.mblk_f, Lv.nn * s * s * 4))))
        return bail(r);
      if (l >= 1 && Lv.nx >= kMgLargeNx && opt->vcycle_prec == IRK_PREC_FP64 && opt->precond != IRK_PC_MONOLITHIC &&
          (r = dalloc(&Lv.srec_d, Lv.nn * 9 * s * 8)))
        return bail(r);
      if ((r = dalloc(&Lv.cf_d, Lv.nn * kCoef2 * 8)) || (r = dalloc(&Lv.cf_f, Lv.nn * kCoef2 * 4)) ||
          (r = dalloc(&Lv.dinv_d, Lv.nn * s * 2 * 8)) || (r = dalloc(&Lv.dinv_f, Lv.nn * s * 2 * 4)))
        return bail(r);
    }
    if ((r = dalloc(&Lv.xa, Lv.nn * s * vb)) || (r = dalloc(&Lv.xb, Lv.nn * s * vb)) ||
        (r = dalloc(&Lv.b, Lv.nn * s * vb)) || (r = dalloc(&Lv.r, Lv.nn * s * vb)))
      return bail(r);
    // boundary entries of every level vector stay zero for the handle's lifetime
    if (cudaMemsetAsync(Lv.xa, 0, Lv.nn * s * vb, h->st) || cudaMemsetAsync(Lv.xb, 0, Lv.nn * s * vb, h->st) ||
        cudaMemsetAsync(Lv.b, 0, Lv.nn * s * vb, h->st) || cudaMemsetAsync(Lv.r, 0, Lv.nn * s * vb, h->st))
      return bail(fail(IRK_ECUDA, "cudaMemsetAsync failed"));
  }
  const int Nc = h->lev[h->L - 1].N;
  h->nint = (Nc - 1) * (Nc - 1) * (dim == 3 ? Nc - 1 : 1);
  int r = IRK_OK;
  if ((r = dalloc(&h->cmap, (size_t)h->nint * sizeof(int))) ||
      (r = dalloc(&h->binv_d, (size_t)s * h->nint * h->nint * 8)) ||
      (r = dalloc(&h->binv_f, (size_t)s * h->nint * h->nint * 4)) ||
      (r = dalloc(&h->kappa_d, dim == 2 ? (size_t)h->N * h->N * 8 : 16)))
    return bail(r);
  if (opt->precond == IRK_PC_MONOLITHIC) {
    const size_t nm = (size_t)s * h->nint;
    if ((r = dalloc(&h->minv_d, nm * nm * 8)) || (r = dalloc(&h->minv_f, nm * nm * 4))) return bail(r);
  }
  h->ne = h->lev[0].nn * s;
  h->m = opt->restart;
  const bool sweeps = opt->precond == IRK_PC_LOWER || opt->precond == IRK_PC_UPPER || opt->precond == IRK_PC_RANA_LD;
  if (dim == 2 && opt->splitting == IRK_SPLIT_IA && (r = dalloc(&h->iarec_d, h->lev[0].nn * kCoef2 * s * 8)))
    return bail(r);
  if (sweeps && s > 1 && dim == 2 && opt->vcycle_prec == IRK_PREC_FP64 && (opt->nu_pre == 2 || opt->nu_post == 2)) {
    const size_t nn0 = h->lev[0].nn;
    if ((r = dalloc(&h->srec_d, nn0 * 9 * s * 8)) || (r = dalloc(&h->x1_d, nn0 * 8))) return bail(r);
    if (cudaMemsetAsync(h->x1_d, 0, nn0 * 8, h->st)) return bail(fail(IRK_ECUDA, "cudaMemsetAsync failed"));
  }
  if (sweeps && s > 1 && opt->vcycle_prec != IRK_PREC_FP64) {
    if ((r = dalloc(&h->zt, h->lev[0].nn * s * vb))) return bail(r);
    // boundary entries are read by the stencils next to the boundary and must stay zero
    if (cudaMemsetAsync(h->zt, 0, h->lev[0].nn * s * vb, h->st)) return bail(fail(IRK_ECUDA, "cudaMemsetAsync failed"));
  }
  const size_t ne = h->ne, m = h->m;
  if ((r = dalloc(&h->V, (m + 1) * ne * 8)) || (r = dalloc(&h->Z, m * ne * 8)) ||
      (r = dalloc(&h->H, (m + 1) * m * 8)) || (r = dalloc(&h->cs, m * 8)) || (r = dalloc(&h->sn, m * 8)) ||
      (r = dalloc(&h->g, (m + 1) * 8)) || (r = dalloc(&h->y, m * 8)) || (r = dalloc(&h->h1, (m + 1) * 8)) ||
      (r = dalloc(&h->h2, (m + 1) * 8)) ||
      (r = dalloc(&h->partial, (m + 1) * (size_t)krylov_partial_blocks() * 8)) || (r = dalloc(&h->scal, 16 * 8)) ||
      (r = dalloc(&h->iflag, 16 * sizeof(int))) ||
      (r = dalloc(&h->rhs, ne * 8)) || (r = dalloc(&h->k, ne * 8)) || (r = dalloc(&h->tmp, ne * 8)))
    return bail(r);
  if (cudaMemsetAsync(h->V, 0, (m + 1) * ne * 8, h->st) || cudaMemsetAsync(h->Z, 0, m * ne * 8, h->st) ||
      cudaMemsetAsync(h->H, 0, (m + 1) * m * 8, h->st) || cudaMemsetAsync(h->h2, 0, (m + 1) * 8, h->st))
    return bail(fail(IRK_ECUDA, "cudaMemsetAsync failed"));
  if (cudaMallocHost((void**)&h->pinned, 8 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(IRK_ENOMEM, "cudaMallocHost failed"));
  }
  if ((r = build_operators(h)) != IRK_OK) return bail(r);
  if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(IRK_ECUDA, "cudaStreamCreateWithFlags failed"));
  }
  h->graphs[0].resize(h->m);
  h->graphs[1].resize(h->m);
  h->cg_graphs[0].resize(s);
  h->cg_graphs[1].resize(s);
  if (opt->solver == IRK_SOLVER_DIRK_CG) {
    const size_t nb = h->lev[0].nn * 8;
    if ((r = dalloc(&h->cg_x, nb)) || (r = dalloc(&h->cg_r, nb)) || (r = dalloc(&h->cg_z, nb)) ||
        (r = dalloc(&h->cg_p, nb)) || (r = dalloc(&h->cg_q, nb)) || (r = dalloc(&h->cg_b, nb)))
      return bail(r);
    if (cudaMemsetAsync(h->cg_x, 0, nb, h->st) || cudaMemsetAsync(h->cg_r, 0, nb, h->st) ||
        cudaMemsetAsync(h->cg_z, 0, nb, h->st) || cudaMemsetAsync(h->cg_p, 0, nb, h->st) ||
        cudaMemsetAsync(h->cg_q, 0, nb, h->st) || cudaMemsetAsync(h->cg_b, 0, nb, h->st))
      return bail(fail(IRK_ECUDA, "cudaMemsetAsync failed"));
  }
  if (const char* e = getenv("IRK_NO_GRAPHS")) h->use_graphs = (e[0] == '\0' || e[0] == '0');
  // IRK_TAIL=1: run the small-level legs and the coarsest solve as one cooperative launch instead of
  // separate ones (off by default: on GB300 inside CUDA graphs the separate launches measured faster, the
  // kernel's six grid barriers costing more than the graph's launch latency);
  // IRK_TAIL_SPIN_CYCLES: the tail kernel's barrier wait limit
  if (const char* e = getenv("IRK_TAIL")) h->tail_on = (e[0] == '1');
  if (const char* e = getenv("IRK_TAIL_SPIN_CYCLES")) h->tail_spin = atoll(e);
  if ((r = dalloc(&h->tail_state, 4 * sizeof(unsigned))) != IRK_OK) return bail(r);
  if (cudaMemsetAsync(h->tail_state, 0, 4 * sizeof(unsigned), h->st)) return bail(fail(IRK_ECUDA, "cudaMemsetAsync failed"));
  *out = h;
  return IRK_OK;
}

// ----------------------------------------------------------------------------
// V-cycle (one per block, or S blocks batched over interleaved stages)
// ----------------------------------------------------------------------------
template <typename T, typename C>
struct Prec;
template <>
struct Prec<double, double> {
  static const double* rec(const Level& L) { return L.brec_d; }
  static const double* cf(const Level& L) { return L.cf_d; }
  static const double* dinv(const Level& L) { return L.dinv_d; }
  static const double* binv(const irk_handle* h) { return h->binv_d; }
};
template <>
struct Prec<float, float> {
  static const float* rec(const Level& L) { return L.brec_f; }
  static const float* cf(const Level& L) { return L.cf_f; }
  static const float* dinv(const Level& L) { return L.dinv_f; }
  static const float* binv(const irk_handle* h) { return h->binv_f; }
};
template <>
struct Prec<__nv_bfloat16, float> {
  static const float* rec(const Level& L) { return L.brec_f; }
  static const float* cf(const Level& L) { return L.cf_f; }
  static const float* dinv(const Level& L) { return L.dinv_f; }
  static const float* binv(const irk_handle* h) { return h->binv_f; }
};

// x0 = V(b0) for blocks st0 .. st0+S-1 (S == s: all blocks batched; S == 1: block st0).
// b0 and x0 are S-interleaved level-0 vectors of precision T; x0 may be nullptr, in
// which case the result is left in an internal buffer that is returned.
// first_done: the finest level's first sweep from a zero guess has already been written, by the
// kernel that formed b0, to the buffer that sweep would write (level 0's xa if nu1 + nu2 is odd,
// else xb; see precond_apply).
// A request to put a one-block cycle's result, times scale, straight into stage i of the interleaved FP64
// stage vector z (the triangular sweeps' scatter); done is set when the last finest-level sweep did so.
struct ZOut {
  double* z;
  int i;         // < 0: all stages of a batched or monolithic cycle, stage k scaled by sc[k]
  double scale;
  bool done;
  void* zt = nullptr;  // FP32 / BF16 one-block cycles: stage i's copy in the V-cycle precision (stage-major)
  double sc[4] = {1.0, 1.0, 1.0, 1.0};
};

// The up-leg sink for a ZOut request (FP32 / BF16 cycles; see ZSink).
template <typename T>
ZSink<T> zsink_of(const ZOut& zo, int s) {
  ZSink<T> zs{};
  zs.z = zo.z;
  zs.sf = s;
  zs.i = zo.i;
  zs.scale = zo.scale;
  zs.zt = reinterpret_cast<T*>(zo.zt);
  for (int k = 0; k < 4; ++k) zs.sc[k] = zo.sc[k];
  return zs;
}

template <typename T, typename C>
T* vcycle(irk_handle* h, int S, int st0, const T* b0, T* x0, int nu1, int nu2, bool first_done = false,
          ZOut* zo = nullptr) {
  using MG = MG2<T, C>;
  using MG3T = MG3<T, C>;
  using P = Prec<T, C>;
  const int s = h->s, L = h->L;
  const bool d3 = (h->dim == 3);
  const double p = sizeof(T), c = sizeof(C);
  Vec8 sig{};
  for (int i = 0; i < S; ++i) sig.v[i] = h->dt * h->Ap[(st0 + i) * s + (st0 + i)];
  cudaStream_t st = h->st;
  const T* bl = b0;
  std::vector<T*> cur(L, nullptr);
  auto interior = [&](const Level& Lv) {
    const double m = Lv.nx - 2;
    return d3 ? m * m * m : m * m;
  };
  // 3D: class values of B_i = M + sigma_i K and omega / B_i(centre), per level
  auto classes = [&](const Level& Lv, Cls4& bc, Vec8& dv) {
    for (int i = 0; i < S; ++i) {
      for (int k = 0; k < 4; ++k) bc.v[i][k] = Lv.mcls[k] + sig.v[i] * Lv.kcls[k];
      dv.v[i] = h->opt.omega / bc.v[i][0];
    }
  };
  // finest-level launches keep their class; launches on a coarser level are IRK_K_MG_COARSE (large
  // levels) or IRK_K_MG_TAIL
  auto coarse_cls = [&](const Level& Lv) { return Lv.nx >= kMgLargeNx ? IRK_K_MG_COARSE : IRK_K_MG_TAIL; };
  auto cls = [&](const Level& Lv, int fine_class) { return (&Lv == &h->lev[0]) ? fine_class : coarse_cls(Lv); };
  // Jacobi diagonal: one block (S == 1) reads the stage-major copy, batched blocks the node-major one
  const int s_d = (S == 1) ? 1 : s;
  auto dinv_of = [&](const Level& Lv) {
    return S == 1 ? P::dinv(Lv) + (size_t)Lv.nn * s + (size_t)st0 * Lv.nn : P::dinv(Lv) + st0;
  };
  // a block of the FP64 triangular sweeps whose first finest-level sweep x1 = d b is in h->x1_d: the
  // later finest-level sweeps use the scaled stencil, x1 + sum_k c'_k x_k (jacobi_scaled)
  constexpr bool f64 = std::is_same<T, double>::value && std::is_same<C, double>::value;
  const bool scaled = f64 && !d3 && first_done && S == 1 && nu1 == 2 && h->srec_d != nullptr;
  auto sweep = [&](Level& Lv, const C* cf, const C* dinv, const T* xin, const T* b, T* xout) {
    const double n = interior(Lv);
    const int kj = cls(Lv, IRK_K_JACOBI);
    if constexpr (f64) {
      if (scaled && &Lv == &h->lev[0] && xin != nullptr) {  // x1, nine planes, x; out
        KScope k(h, kj, n * (3 * p + 9 * c), 18.0 * n);
        MG::jacobi_scaled(st, Lv.nx, h->srec_d + (size_t)st0 * 9 * Lv.nn, h->x1_d, xin, xout);
        return;
      }
    }
    if (d3) {
      Cls4 bc{};
      Vec8 dv{};
      classes(Lv, bc, dv);
      KScope k(h, kj, n * S * (xin ? 3 : 2) * p, (xin ? 34.0 : 1.0) * n * S);
      MG3T::jacobi(S, st, Lv.nx, bc, dv, xin, b, xout);
      return;
    }
    const C* rec = P::rec(Lv);
    if (xin == nullptr) {
      KScope k(h, kj, n * S * (2 * p + c), n * S);
      MG::jacobi(S, st, Lv.nx, cf, Lv.hm, sig, dinv, s_d, xin, b, xout);
    } else if (rec != nullptr) {  // B_i records: 9 products + 2 per node and stage
      KScope k(h, kj, n * S * (3 * p + c + kCoef2 * c), 20.0 * n * S);
      MG::jacobi_rec(S, st, Lv.nx, rec + (size_t)st0 * Lv.nn * kCoef2, Lv.nn * kCoef2, dinv, s_d, xin, b, xout);
    } else {
      KScope k(h, kj, n * (S * (3 * p + c) + kCoef2 * c), 33.0 * n * S);
      MG::jacobi(S, st, Lv.nx, cf, Lv.hm, sig, dinv, s_d, xin, b, xout);
    }
  };
  // 2D levels under V(2, 2): one fused kernel per leg (mg2d_legs.cuh) instead of six launches; on the
  // coarse levels, and for FP32 / BF16 cycles also on the finest one (memory-bound there: the legs read
  // b, the records and the diagonal once instead of three times)
  constexpr bool lowp = !std::is_same<C, double>::value;
  auto fused_leg = [&](int l) {
    return !d3 && nu1 == 2 && nu2 == 2 && (l >= 1 || (lowp && x0 == nullptr && !first_done));
  };
  auto rec_of = [&](const Level& Lv) {
    const C* rec = P::rec(Lv);
    return rec ? rec + (size_t)st0 * Lv.nn * kCoef2 : nullptr;
  };
  // FP64 one-block V-cycles: the large-tile legs sweep with the level's scaled stencil
  auto srec_of = [&](const Level& Lv) -> const C* {
    if (!f64 || S != 1 || Lv.srec_d == nullptr) return nullptr;
    return reinterpret_cast<const C*>(Lv.srec_d + (size_t)st0 * 9 * Lv.nn);
  };
  // the small-level tail (levels tl0 .. L - 1: fused legs below kMgLargeNx nodes per axis, never the
  // finest level, and the coarsest solve) as one cooperative launch (mg2d_tail.cuh); tl0 = L: none
  int tl0 = L;
  if (h->tail_on && !d3 && nu1 == 2 && nu2 == 2 && L >= 3) {
    int l0 = L - 1;
    while (l0 - 1 >= 1 && h->lev[l0 - 1].nx < kMgLargeNx && fused_leg(l0 - 1) && rec_of(h->lev[l0 - 1]) != nullptr)
      --l0;
    if (l0 <= L - 2 && L - 1 - l0 <= kTailMaxLevels) tl0 = l0;
  }
  const int l_down_end = (tl0 < L) ? tl0 : L - 1;
  for (int l = 0; l < l_down_end; ++l) {
    Level& Lv = h->lev[l];
    Level& Lc = h->lev[l + 1];
    const C* cf = d3 ? nullptr : P::cf(Lv);
    const C* dinv = d3 ? nullptr : dinv_of(Lv);
    if (fused_leg(l)) {
      const double n = interior(Lv), nc = interior(Lc);
      const bool rec = P::rec(Lv) != nullptr;
      KScope k(h, cls(Lv, IRK_K_JACOBI), n * S * (2 * p + c) + n * kCoef2 * c * (rec ? S : 1) + nc * S * p,
               n * S * (rec ? 42.0 : 66.0));
      MG::down_leg(S, st, Lv.nx, cf, Lv.hm, sig, rec_of(Lv), Lv.nn * kCoef2, dinv, s_d, bl, (T*)Lv.xa, Lc.nx,
                   (T*)Lc.b, srec_of(Lv));
      cur[l] = (T*)Lv.xa;
      bl = (const T*)Lc.b;
      continue;
    }
    // choose the two buffers so that the last of the nu1 + nu2 sweeps lands in `last`
    T* last = (l == 0 && x0) ? x0 : (T*)Lv.xa;
    T* other = (l == 0 && x0) ? (T*)Lv.xa : (T*)Lv.xb;
    T* bufs[2];
    if ((nu1 + nu2) % 2 == 1) {
      bufs[0] = last, bufs[1] = other;
    } else {
      bufs[0] = other, bufs[1] = last;
    }
    int w = 0;
    // the first sweep's result is already in bufs[0] (written together with b0); with the scaled
    // finest-level sweeps it is in h->x1_d instead, which they read on every sweep (nu1 == 2: never written)
    const bool skip_first = first_done && l == 0 && nu1 >= 1;
    if (scaled && l == 0) bufs[0] = reinterpret_cast<T*>(h->x1_d);
    // two sweeps from zero fused into one pass: always for FP32 / BF16; for FP64 only on the
    // coarse levels (on the finest level it would add FP64 work to an FP64-pipe-bound sweep)
    const bool fuse2 = !skip_first && nu1 >= 2 && (!std::is_same<C, double>::value || l > 0);
    int k0 = 1;
    if (fuse2) {
      const double n = interior(Lv);
      if (d3) {
        Cls4 bc{};
        Vec8 dv{};
        classes(Lv, bc, dv);
        KScope kk(h, cls(Lv, IRK_K_JACOBI), n * S * 2 * p, 36.0 * n * S);
        MG3T::jacobi2z(S, st, Lv.nx, bc, dv, bl, bufs[1]);
      } else {
        const C* rec = P::rec(Lv);
        KScope kk(h, cls(Lv, IRK_K_JACOBI), n * S * (2 * p + c + kCoef2 * c) + (rec ? 0.0 : n * kCoef2 * c),
                  (rec ? 30.0 : 42.0) * n * S);
        MG::jacobi2z(S, st, Lv.nx, cf, Lv.hm, sig, rec ? rec + (size_t)st0 * Lv.nn * kCoef2 : nullptr,
                     Lv.nn * kCoef2, dinv, s_d, bl, bufs[1]);
      }
      w = 1;
      k0 = 2;
    } else if (!skip_first) {
      sweep(Lv, cf, dinv, nullptr, bl, bufs[w]);
    }
    for (int k = k0; k < nu1; ++k, w ^= 1) sweep(Lv, cf, dinv, bufs[w], bl, bufs[w ^ 1]);
    cur[l] = bufs[w];
    const double nf = interior(Lv), nc = interior(Lc);
    if (d3) {
      Cls4 bc{};
      Vec8 dv{};
      classes(Lv, bc, dv);
      {
        KScope k(h, cls(Lv, IRK_K_RESIDUAL), nf * S * 3 * p, 33.0 * nf * S);
        MG3T::residual(S, st, Lv.nx, bc, cur[l], bl, (T*)Lv.r);
      }
      KScope k(h, cls(Lv, IRK_K_RESTRICT), (nf + nc) * S * p, 30.0 * nc * S);
      MG3T::restrict_(S, st, Lv.nx, (const T*)Lv.r, Lc.nx, (T*)Lc.b);
    } else {
      if (const C* rec = P::rec(Lv)) {
        KScope k(h, cls(Lv, IRK_K_RESIDUAL), nf * S * (3 * p + kCoef2 * c), 18.0 * nf * S);
        MG::residual_rec(S, st, Lv.nx, rec + (size_t)st0 * Lv.nn * kCoef2, Lv.nn * kCoef2, cur[l], bl, (T*)Lv.r);
      } else {
        KScope k(h, cls(Lv, IRK_K_RESIDUAL), nf * (3 * S * p + kCoef2 * c), 31.0 * nf * S);
        MG::residual(S, st, Lv.nx, cf, Lv.hm, sig, cur[l], bl, (T*)Lv.r);
      }
      KScope k(h, cls(Lv, IRK_K_RESTRICT), (nf + nc) * S * p, 12.0 * nc * S);
      MG::restrict_(S, st, Lv.nx, (const T*)Lv.r, Lc.nx, (T*)Lc.b);
    }
    bl = (const T*)Lc.b;
  }
  if (tl0 < L) {
    TailSpec<C> sp{};
    sp.levels = L - 1 - tl0;
    double bytes = 0.0, flops = 0.0;
    for (int k = 0; k < sp.levels; ++k) {
      Level& Lv = h->lev[tl0 + k];
      const double n = interior(Lv), nc = interior(h->lev[tl0 + k + 1]);
      sp.nx[k] = Lv.nx;
      sp.rec[k] = rec_of(Lv);
      sp.rstride[k] = Lv.nn * kCoef2;
      sp.dinv[k] = dinv_of(Lv);
      sp.b[k] = Lv.b;
      sp.xa[k] = Lv.xa;
      sp.xb[k] = Lv.xb;
      // the down and up legs' algorithmic bytes and flops (as counted for the separate legs)
      bytes += n * S * (2 * p + c) + n * kCoef2 * c * S + nc * S * p + n * S * (4 * p + c) + n * kCoef2 * c * S +
               nc * S * p;
      flops += n * S * (42.0 + 45.0);
    }
    Level& Lc = h->lev[L - 1];
    const double ni = h->nint;
    sp.nxc = Lc.nx;
    sp.binv = P::binv(h) + (size_t)st0 * h->nint * h->nint;
    sp.bc = Lc.b;
    sp.xc = Lc.xa;
    sp.bar = h->tail_state;
    sp.err = reinterpret_cast<int*>(h->tail_state + 2);
    sp.spin_cycles = h->tail_spin;
    {
      KScope k(h, IRK_K_MG_TAIL, bytes + S * ni * ni * c + 2 * S * ni * p, flops + 2.0 * S * ni * ni);
      MG::tail_cycle(S, st, sp, s_d);  // a failed launch is reported by the caller's launch check
    }
    h->tail_used = true;
    for (int l = tl0; l <= L - 2; ++l) cur[l] = (T*)h->lev[l].xb;
    cur[L - 1] = (T*)Lc.xa;
  } else {  // coarsest level: exact solve
    Level& Lc = h->lev[L - 1];
    T* xc = (L == 1 && x0) ? x0 : (T*)Lc.xa;
    const C* binv = P::binv(h) + (size_t)st0 * h->nint * h->nint;
    const double ni = h->nint;
    KScope k(h, IRK_K_COARSE, S * ni * ni * c + 2 * S * ni * p, 2.0 * S * ni * ni);
    if (d3)
      MG3T::coarse_solve(S, st, h->nint, binv, h->cmap, bl, xc);
    else
      MG::coarse_solve(S, st, Lc.nx, binv, bl, xc);
    cur[L - 1] = xc;
  }
  for (int l = (tl0 < L ? tl0 - 1 : L - 2); l >= 0; --l) {
    Level& Lv = h->lev[l];
    Level& Lc = h->lev[l + 1];
    const C* cf = d3 ? nullptr : P::cf(Lv);
    const C* dinv = d3 ? nullptr : dinv_of(Lv);
    const T* bfine = (l == 0) ? b0 : (const T*)Lv.b;
    const double nf = interior(Lv), nc = interior(Lc);
    if (fused_leg(l)) {
      T* xo = (cur[l] == (T*)Lv.xa) ? (T*)Lv.xb : (T*)Lv.xa;
      const bool rec = P::rec(Lv) != nullptr;
      // FP32 / BF16 cycle: the finest up leg writes the caller's stage vector directly (one block, or all
      // stages of the batched cycle)
      ZSink<T> zs{};
      if (lowp && zo && l == 0 && x0 == nullptr &&
          ((S == 1 && zo->i >= 0 && zo->zt != nullptr) || (S == s && S > 1 && zo->i < 0))) {
        zs = zsink_of<T>(*zo, s);
        zo->done = true;
      }
      KScope k(h, cls(Lv, IRK_K_JACOBI),
               nf * S * (4 * p + c) + nf * kCoef2 * c * (rec ? S : 1) + nc * S * p + (zs.z ? nf * 8.0 : 0.0),
               nf * S * (rec ? 45.0 : 69.0) + (zs.z ? nf : 0.0));
      MG::up_leg(S, st, Lv.nx, cf, Lv.hm, sig, rec_of(Lv), Lv.nn * kCoef2, dinv, s_d, cur[l], bfine, Lc.nx,
                 cur[l + 1], xo, srec_of(Lv), zs);
      cur[l] = xo;
      continue;
    }
    {
      KScope k(h, cls(Lv, IRK_K_PROLONG), (nc + 2 * nf) * S * p, (d3 ? 9.0 : 5.0) * nf * S);
      if (d3)
        MG3T::prolong_add(S, st, Lc.nx, cur[l + 1], Lv.nx, cur[l]);
      else
        MG::prolong_add(S, st, Lc.nx, cur[l + 1], Lv.nx, cur[l]);
    }
    T* last = (l == 0 && x0) ? x0 : (T*)Lv.xa;
    T* other = (l == 0 && x0) ? (T*)Lv.xa : (T*)Lv.xb;
    T* a = cur[l];
    T* bnext = (a == last) ? other : last;
    for (int k = 0; k < nu2; ++k) {
      if constexpr (f64) {
        // the last finest-level sweep of a scaled one-block cycle may write the caller's stage vector
        if (zo && l == 0 && k == nu2 - 1 && scaled && x0 == nullptr) {
          const double n = interior(Lv);
          KScope kk(h, IRK_K_JACOBI, n * (3 * p + 9 * c), 19.0 * n);
          if (MG::jacobi_scaled_z(s, st, Lv.nx, h->srec_d + (size_t)st0 * 9 * Lv.nn, h->x1_d, a, zo->i, zo->z,
                                  zo->scale)) {
            zo->done = true;
            break;
          }
        }
      }
      sweep(Lv, cf, dinv, a, bfine, bnext);
      std::swap(a, bnext);
    }
    cur[l] = a;
  }
  h->vcycles += S;
  return cur[0];
}

// One monolithic multigrid V-cycle (Sec. 3, monolithic multigrid) on the s-interleaved stage
// vectors: x0 = V(b0) for the whole system I (x) M + dt A (x) K, with stage-coupled point-block
// Jacobi relaxation on every level and the exact coupled coarsest solve.  x0 may be nullptr (the
// result stays in a level buffer, which is returned).
// transpose: the transposed cycle (the adjoint's preconditioner): S^T = I (x) M + dt A^T (x) K, D^{-T},
// inv^T; the caller swaps nu1 and nu2, and R = P^T keeps the transfer pair.
template <typename T, typename C>
T* mmg_vcycle(irk_handle* h, const T* b0, T* x0, int nu1, int nu2, bool transpose = false, ZOut* zo = nullptr) {
  using MG = MG2<T, C>;
  using P = Prec<T, C>;
  constexpr bool f64 = std::is_same<C, double>::value;
  const int s = h->s, L = h->L;
  const double p = sizeof(T), c = sizeof(C);
  cudaStream_t st = h->st;
  Mat4 mix{};
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) mix.v[i * s + j] = h->dt * (transpose ? h->A[j * s + i] : h->A[i * s + j]);
  auto cls = [&](const Level& Lv, int fine_class) {
    if (&Lv == &h->lev[0]) return fine_class;
    return Lv.nx >= kMgLargeNx ? IRK_K_MG_COARSE : IRK_K_MG_TAIL;
  };
  auto blk = [&](const Level& Lv) { return f64 ? (const C*)Lv.mblk_d : (const C*)Lv.mblk_f; };
  auto interior = [&](const Level& Lv) { return (double)(Lv.nx - 2) * (Lv.nx - 2); };
  auto smooth = [&](Level& Lv, const T* xin, const T* b, T* xout) {
    const double n = interior(Lv);
    KScope k(h, cls(Lv, IRK_K_JACOBI), n * (s * (xin ? 3 : 2) * p + kCoef2 * c + s * s * c),
             n * (xin ? s * (20.0 + 2 * s) + 2.0 * s * s : 2.0 * s * s));
    MG::mmg_smooth(s, st, Lv.nx, P::cf(Lv), Lv.hm, mix, blk(Lv), xin, b, xout, transpose);
  };
  // V(2, 2): one fused kernel per leg (mg2d_legs.cuh) instead of five or six launches.  FP32 / BF16 on
  // every level (the finest one included: memory-bound, the fused legs read b, D and the records once
  // instead of three times); FP64 only below kMgLargeNx nodes per axis (on larger levels the coupled
  // relaxation is FP64-pipe-bound and the halo recomputation costs more than the launches it saves)
  auto fused_leg = [&](int l) {
    if (nu1 != 2 || nu2 != 2) return false;
    if (f64) return l >= 1 && h->lev[l].nx < kMgLargeNx;
    return l >= 1 || x0 == nullptr;
  };
  // per node: residual s (20 + 2 s), sweep that plus the block product 2 s^2
  const double fres = s * (20.0 + 2 * s), fblk = 2.0 * s * s;
  std::vector<T*> cur(L, nullptr);
  const T* bl = b0;
  for (int l = 0; l < L - 1; ++l) {
    Level& Lv = h->lev[l];
    Level& Lc = h->lev[l + 1];
    if (fused_leg(l)) {
      const double n = interior(Lv), nc = interior(Lc);
      KScope k(h, cls(Lv, IRK_K_JACOBI), n * (2 * s * p + kCoef2 * c + s * s * c) + nc * s * p,
               n * (2 * fres + 3 * fblk) + 12.0 * nc * s);
      MG::mmg_down_leg(s, st, Lv.nx, P::cf(Lv), Lv.hm, mix, blk(Lv), transpose, bl, (T*)Lv.xa, Lc.nx, (T*)Lc.b);
      cur[l] = (T*)Lv.xa;
      bl = (const T*)Lc.b;
      continue;
    }
    T* last = (l == 0 && x0) ? x0 : (T*)Lv.xa;
    T* other = (l == 0 && x0) ? (T*)Lv.xa : (T*)Lv.xb;
    T* bufs[2];
    if ((nu1 + nu2) % 2 == 1) {
      bufs[0] = last, bufs[1] = other;
    } else {
      bufs[0] = other, bufs[1] = last;
    }
    int w = 0;
    smooth(Lv, nullptr, bl, bufs[0]);
    for (int k = 1; k < nu1; ++k, w ^= 1) smooth(Lv, bufs[w], bl, bufs[w ^ 1]);
    cur[l] = bufs[w];
    const double nf = interior(Lv), nc = interior(Lc);
    {
      KScope k(h, cls(Lv, IRK_K_RESIDUAL), nf * (3 * s * p + kCoef2 * c), nf * s * (20.0 + 2 * s));
      MG::mmg_residual(s, st, Lv.nx, P::cf(Lv), Lv.hm, mix, cur[l], bl, (T*)Lv.r);
    }
    {
      KScope k(h, cls(Lv, IRK_K_RESTRICT), (nf + nc) * s * p, 12.0 * nc * s);
      MG::restrict_(s, st, Lv.nx, (const T*)Lv.r, Lc.nx, (T*)Lc.b);
    }
    bl = (const T*)Lc.b;
  }
  {  // coarsest level: exact coupled solve
    Level& Lc = h->lev[L - 1];
    T* xc = (L == 1 && x0) ? x0 : (T*)Lc.xa;
    const double nm = (double)s * h->nint;
    KScope k(h, IRK_K_COARSE, nm * nm * c + 2 * nm * p, 2.0 * nm * nm);
    MG::mmg_coarse_solve(s, st, Lc.nx, f64 ? (const C*)h->minv_d : (const C*)h->minv_f, bl, xc, transpose);
    cur[L - 1] = xc;
  }
  for (int l = L - 2; l >= 0; --l) {
    Level& Lv = h->lev[l];
    Level& Lc = h->lev[l + 1];
    const T* bfine = (l == 0) ? b0 : (const T*)Lv.b;
    const double nf = interior(Lv), nc = interior(Lc);
    if (fused_leg(l)) {
      T* xo = (cur[l] == (T*)Lv.xa) ? (T*)Lv.xb : (T*)Lv.xa;
      KScope k(h, cls(Lv, IRK_K_JACOBI), nf * (3 * s * p + kCoef2 * c + s * s * c) + nc * s * p,
               nf * (2 * (fres + fblk) + 5.0 * s));
      // FP32 / BF16: the finest up leg writes the caller's stage vector directly
      ZSink<T> zs{};
      if (!f64 && zo && l == 0 && x0 == nullptr && zo->i < 0) {
        zs = zsink_of<T>(*zo, s);
        zo->done = true;
      }
      MG::mmg_up_leg(s, st, Lv.nx, P::cf(Lv), Lv.hm, mix, blk(Lv), transpose, cur[l], bfine, Lc.nx, cur[l + 1], xo,
                     zs);
      cur[l] = xo;
      continue;
    }
    {
      KScope k(h, cls(Lv, IRK_K_PROLONG), (nc + 2 * nf) * s * p, 5.0 * nf * s);
      MG::prolong_add(s, st, Lc.nx, cur[l + 1], Lv.nx, cur[l]);
    }
    T* last = (l == 0 && x0) ? x0 : (T*)Lv.xa;
    T* other = (l == 0 && x0) ? (T*)Lv.xa : (T*)Lv.xb;
    T* a = cur[l];
    T* bnext = (a == last) ? other : last;
    for (int k = 0; k < nu2; ++k) {
      smooth(Lv, a, bfine, bnext);
      std::swap(a, bnext);
    }
    cur[l] = a;
  }
  h->vcycles += 1;
  return cur[0];
}

// z = P^{-1} v with the configured block preconditioner (v, z: double stage vectors).
// transpose: apply P^T (the triangular sweep runs the other way with A^T couplings
// and every V(nu1, nu2) cycle becomes V(nu2, nu1), its transpose).
template <typename T, typename C>
int precond_apply(irk_handle* h, const double* v, double* z, bool transpose) {
  using MG = MG2<T, C>;
  const int s = h->s;
  const int nu1 = transpose ? h->opt.nu_post : h->opt.nu_pre;
  const int nu2 = transpose ? h->opt.nu_pre : h->opt.nu_post;
  Level& L0 = h->lev[0];
  cudaStream_t st = h->st;
  const double p = sizeof(T), c = sizeof(C), ne = (double)h->ne;
  const bool ia = (h->opt.splitting == IRK_SPLIT_IA);
  if (h->opt.precond == IRK_PC_MONOLITHIC) {
    if constexpr (std::is_same<T, double>::value) {
      mmg_vcycle<T, C>(h, v, z, nu1, nu2, transpose);
    } else {
      {
        KScope k(h, IRK_K_OTHER, ne * (8 + p), 0);
        MG::cast_to(st, v, (T*)L0.b, h->ne);
      }
      ZOut zo{z, -1, 1.0, false};
      T* x = mmg_vcycle<T, C>(h, (const T*)L0.b, nullptr, nu1, nu2, transpose, &zo);
      if (!zo.done) {
        KScope k(h, IRK_K_OTHER, ne * (8 + p), 0);
        MG::cast_from(st, x, z, h->ne);
      }
    }
    CK_LAUNCH();
    return IRK_OK;
  }
  if (h->opt.precond == IRK_PC_DIAG || s == 1) {
    if constexpr (std::is_same<T, double>::value) {
      vcycle<T, C>(h, s, 0, v, z, nu1, nu2);
    } else {
      {
        KScope k(h, IRK_K_OTHER, ne * (8 + p), 0);
        MG::cast_to(st, v, (T*)L0.b, h->ne);
      }
      // the batched cycle's finest up leg writes z, with the IA scaling below folded in
      ZOut zo{z, -1, 1.0, false};
      for (int i = 0; i < s; ++i) zo.sc[i] = ia ? h->Tm[i * s + i] : 1.0;
      T* x = vcycle<T, C>(h, s, 0, (const T*)L0.b, nullptr, nu1, nu2, false, &zo);
      if (zo.done) {
        CK_LAUNCH();
        return IRK_OK;
      }
      KScope k(h, IRK_K_OTHER, ne * (8 + p), 0);
      MG::cast_from(st, x, z, h->ne);
    }
    if (ia) {  // IA diagonal blocks (1/a_ii) M + dt K = (1/a_ii)(M + dt a_ii K): scale the V-cycle output
      Vec8 sc{};
      for (int i = 0; i < s; ++i) sc.v[i] = h->Tm[i * s + i];
      KScope k(h, IRK_K_OTHER, 16.0 * ne, ne);
      launch_stage_scale(s, st, L0.nn, sc, z);
    }
    CK_LAUNCH();
    return IRK_OK;
  }
  // triangular sweep: lower (forward) or upper (backward) in the effective matrix
  bool lower = (h->opt.precond == IRK_PC_LOWER || h->opt.precond == IRK_PC_RANA_LD);
  if (transpose) lower = !lower;
  const bool d3 = (h->dim == 3);
  const C* cf = d3 ? nullptr : Prec<T, C>::cf(L0);
  const double n = d3 ? (double)(L0.nx - 2) * (L0.nx - 2) * (L0.nx - 2) : n_int(L0.nx);
  Cls4 kc{};
  for (int k = 0; k < 4; ++k) kc.v[0][k] = L0.kcls[k];
  // FP64, 2D: the kernel forming a block's right-hand side also writes the first Jacobi sweep from a
  // zero guess (pointwise), into the buffer where the V-cycle's first sweep would land
  const bool fuse_first = !d3 && std::is_same<C, double>::value && nu1 >= 1;
  // (with the scaled finest-level sweeps: into h->x1_d, which the later sweeps read)
  const bool scaled = fuse_first && nu1 == 2 && h->srec_d != nullptr;
  T* x1buf = scaled ? reinterpret_cast<T*>(h->x1_d) : ((nu1 + nu2) % 2 == 1) ? (T*)L0.xa : (T*)L0.xb;
  // FP32 / BF16: the solved stages are read back in precision T (stage-major copies in h->zt)
  T* zt = std::is_same<T, double>::value ? nullptr : (T*)h->zt;
  const size_t zs = L0.nn;
  for (int step = 0; step < s; ++step) {
    const int i = lower ? step : s - 1 - step;
    Vec8 cj{};
    int done = 0;
    for (int j = 0; j < s; ++j) {
      const bool solved = lower ? (j < i) : (j > i);
      // AI: dt (Ap)_ij couples through K; IA: (T^{-1})_ij couples through M
      const double a = ia ? h->Tinv[i * s + j] : (transpose ? h->Ap[j * s + i] : h->Ap[i * s + j]);
      cj.v[j] = solved ? (ia ? a : h->dt * a) : 0.0;
      // reading the unscaled V-cycle outputs (zt): fold in the scale z_j = T_jj x_j (IA)
      if (zt && ia) cj.v[j] *= h->Tm[j * s + j];
      done += (solved && a != 0.0) ? 1 : 0;
    }
    {  // single-stage right-hand side in level-0 b (precision T)
      const C* d1 = fuse_first ? Prec<T, C>::dinv(L0) + L0.nn * s + (size_t)i * L0.nn : nullptr;
      KScope k(h, IRK_K_BLOCK_RHS, n * (8 + done * 8 + (d3 ? 0 : kCoef2 * c) + p + (fuse_first ? c + p : 0)),
               (d3 ? 32.0 : 19.0) * done * n + (fuse_first ? n : 0));
      if (ia && d3) {
        Cls4 mc{};
        for (int q = 0; q < 4; ++q) mc.v[0][q] = L0.mcls[q];
        MG3<T, C>::block_rhs(s, st, L0.nx, mc, v, z, i, cj, (T*)L0.b, zt, zs);
      } else if (ia) {
        MG::block_rhs_mass(s, st, L0.nx, L0.hm, v, z, i, cj, (T*)L0.b, fuse_first ? d1 : nullptr, x1buf, zt, zs);
      } else if (d3) {
        MG3<T, C>::block_rhs(s, st, L0.nx, kc, v, z, i, cj, (T*)L0.b, zt, zs);
      } else {
        MG::block_rhs(s, st, L0.nx, cf, v, z, i, cj, (T*)L0.b, fuse_first ? d1 : nullptr, x1buf, zt, zs);
      }
    }
    const double scale = ia ? h->Tm[i * s + i] : 1.0;
    ZOut zo{z, i, scale, false, zt ? zt + (size_t)i * zs : nullptr};
    T* x = vcycle<T, C>(h, 1, i, (const T*)L0.b, nullptr, nu1, nu2, fuse_first, !d3 ? &zo : nullptr);
    if (zo.done) continue;  // the last sweep (or up leg) wrote scale * x into stage i of z
    KScope k(h, IRK_K_OTHER, n * (p + 8), 0);
    T* zti = zt ? zt + (size_t)i * zs : nullptr;
    if (d3)
      MG3<T, C>::scatter_stage(s, st, L0.nx, x, i, z, scale, zti);
    else
      MG::scatter_stage(s, st, L0.nx, x, i, z, scale, zti);
  }
  CK_LAUNCH();
  return IRK_OK;
}

int precond(irk_handle* h, const double* v, double* z, bool transpose) {
  switch (h->opt.vcycle_prec) {
    case IRK_PREC_FP64: return precond_apply<double, double>(h, v, z, transpose);
    case IRK_PREC_FP32: return precond_apply<float, float>(h, v, z, transpose);
    default: return precond_apply<__nv_bfloat16, float>(h, v, z, transpose);
  }
}

Mat4 mixing(const irk_handle* h, bool transpose) {
  Mat4 m{};
  const int s = h->s;
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) m.v[i * s + j] = h->dt * (transpose ? h->A[j * s + i] : h->A[i * s + j]);
  return m;
}

Cls4 mass_stiff_classes(const Level& L0) {
  Cls4 mk{};
  for (int k = 0; k < 4; ++k) mk.v[0][k] = L0.mcls[k], mk.v[1][k] = L0.kcls[k];
  return mk;
}

Mat4 ia_mixing(const irk_handle* h, bool transpose) {
  Mat4 m{};
  const int s = h->s;
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) m.v[i * s + j] = transpose ? h->Ainv[j * s + i] : h->Ainv[i * s + j];
  return m;
}

int apply_operator(irk_handle* h, const double* x, double* y, bool transpose) {
  const Level& L0 = h->lev[0];
  const int s = h->s;
  if (h->opt.splitting == IRK_SPLIT_IA) {
    const double m = L0.nx - 2;
    const double ni = (h->dim == 3) ? m * m * m : m * m;
    // 2D: the per-stage records of A^{-1}_ii M + dt K, their stencils, the separable mass and the
    // off-diagonal couplings; 3D: class stencils
    KScope k(h, IRK_K_STAGE_APPLY, (double)L0.nn * (16.0 * s + (h->dim == 3 ? 0.0 : 8.0 * kCoef2 * s)),
             ni * s * ((h->dim == 3 ? 30.0 : 27.0) + 2.0 * s));
    if (h->dim == 3)
      launch_stage_apply3_ia(s, h->st, L0.nx, mass_stiff_classes(L0), ia_mixing(h, transpose), h->dt, x, y);
    else
      launch_stage_apply_ia(s, h->st, L0.nx, h->iarec_d, L0.hm, ia_mixing(h, transpose), x, y);
    CK_LAUNCH();
    return IRK_OK;
  }
  if (h->dim == 3) {
    const double m = L0.nx - 2;
    KScope k(h, IRK_K_STAGE_APPLY, (double)L0.nn * 16.0 * s, m * m * m * s * (38.0 + 2.0 * s));
    launch_stage_apply3(s, h->st, L0.nx, mass_stiff_classes(L0), mixing(h, transpose), x, y);
    CK_LAUNCH();
    return IRK_OK;
  }
  KScope k(h, IRK_K_STAGE_APPLY, (double)L0.nn * (16.0 * s + 8.0 * kCoef2), n_int(L0.nx) * s * (28.0 + 2.0 * s));
  launch_stage_apply(s, h->st, L0.nx, L0.cf_d, L0.hm, mixing(h, transpose), x, y);
  CK_LAUNCH();
  return IRK_OK;
}

void multidot(irk_handle* h, const double* V, size_t ld, int count, const double* w, double* out) {
  const double n = (double)h->ne;
  {
    KScope k(h, IRK_K_MULTIDOT, (count + 1.0) * n * 8, 2.0 * count * n);
    launch_multidot(h->st, V, ld, count, w, h->ne, h->partial);
  }
  const double nb = krylov_partial_blocks();
  KScope k(h, IRK_K_OTHER, count * nb * 8, count * nb);
  launch_reduce_partials(h->st, h->partial, count, out);
}

void multi_axpy(irk_handle* h, double* w, const double* V, size_t ld, int count, const double* coef, double sign) {
  const double n = (double)h->ne;
  KScope k(h, IRK_K_AXPY, (count + 2.0) * n * 8, 2.0 * count * n);
  launch_multi_axpy(h->st, w, V, ld, count, coef, sign, h->ne);
}

void scale(irk_handle* h, double* dst, const double* src, const double* denom) {
  KScope k(h, IRK_K_OTHER, 16.0 * h->ne, (double)h->ne);
  launch_scale(h->st, dst, src, denom, h->ne);
}

// ||v||_2 into scal[slot] (device), its square into scal[slot + 1].
int norm2(irk_handle* h, const double* v, int slot) {
  multidot(h, v, 0, 1, v, h->scal + slot + 1);
  KScope k(h, IRK_K_OTHER, 0, 0);
  launch_sqrt_scalar(h->st, h->scal + slot + 1, h->scal + slot);
  CK_LAUNCH();
  return IRK_OK;
}

// ----------------------------------------------------------------------------
// FGMRES (right preconditioned; CGS2, one-pass CGS or DGKS Arnoldi; Givens on the device)
// ----------------------------------------------------------------------------
// One Arnoldi step of FGMRES for basis index j: z_j = P^{-1} v_j, w = S z_j,
// orthogonalisation, Givens update and normalisation; ends by copying
// (|g_{j+1}| / r0, h_{j+1,j}) to pinned host memory.  Uses only device pointers
// and values fixed for the handle, so it can be captured into a CUDA graph.
int arnoldi_step(irk_handle* h, int j, bool transpose) {
  cudaStream_t st = h->st;
  const size_t ne = h->ne;
  const int ldh = h->m + 1;
  double* vj = h->V + (size_t)j * ne;
  double* zj = h->Z + (size_t)j * ne;
  double* w = h->V + (size_t)(j + 1) * ne;
  double* r0p = h->scal + 9;
  TRY(precond(h, vj, zj, transpose));
  TRY(apply_operator(h, zj, w, transpose));
  if (h->opt.orth == IRK_ORTH_CGS2) {
    // classical Gram-Schmidt, twice.  The second pass also sees w' itself (it sits in the
    // slot of V_{j+1}), so it returns ||w'||^2; the Givens kernel takes ||w''|| by
    // Pythagoras and the second update normalises in the same sweep.
    multidot(h, h->V, ne, j + 1, w, h->h1);
    if (j + 1 <= krylov_axpy_dot_max()) {
      {  // w' = w - V h1 and the second pass's dot products (with ||w'||^2 last) from one read of V
        const double n = (double)ne;
        KScope k(h, IRK_K_MULTIDOT, (j + 3.0) * n * 8, 4.0 * (j + 1) * n + 2.0 * n);
        launch_axpy_dot(st, w, h->V, ne, j + 1, h->h1, ne, h->partial);
      }
      const double nb = krylov_partial_blocks();
      KScope k(h, IRK_K_OTHER, (j + 2) * nb * 8, (j + 2) * nb);
      launch_reduce_partials(st, h->partial, j + 2, h->h2);
    } else {
      multi_axpy(h, w, h->V, ne, j + 1, h->h1, -1.0);
      multidot(h, h->V, ne, j + 2, w, h->h2);
    }
    {
      KScope k(h, IRK_K_OTHER, 0, 0);
      launch_givens(st, j, ldh, h->H, h->cs, h->sn, h->g, h->h1, h->h2, nullptr, h->scal + 4, r0p, h->scal + 5, 1,
                    h->scal + 8);
    }
    {
      const double n = (double)ne;
      KScope k(h, IRK_K_AXPY, (j + 3.0) * n * 8, 2.0 * (j + 1) * n + n);
      launch_multi_axpy(st, w, h->V, ne, j + 1, h->h2, -1.0, ne, h->scal + 8);
    }
  } else if (h->opt.orth == IRK_ORTH_CGS) {
    // one pass: h1 = V^T w, w' = w - V h1 with ||w'||^2 reduced in the same sweep, normalise
    multidot(h, h->V, ne, j + 1, w, h->h1);
    const double n = (double)ne;
    {
      KScope k(h, IRK_K_AXPY, (j + 3.0) * n * 8, 2.0 * (j + 1) * n + 2.0 * n);
      launch_axpy_norm(st, w, h->V, ne, j + 1, h->h1, ne, h->partial);
    }
    {
      const double nb = krylov_partial_blocks();
      KScope k(h, IRK_K_OTHER, nb * 8, nb);
      launch_reduce_partials(st, h->partial, 1, h->scal + 3);
    }
    {
      KScope k(h, IRK_K_OTHER, 0, 0);  // h2 holds zeros in this mode (set at create)
      launch_givens(st, j, ldh, h->H, h->cs, h->sn, h->g, h->h1, h->h2, h->scal + 3, h->scal + 4, r0p, h->scal + 5);
    }
    KScope k(h, IRK_K_OTHER, 16.0 * n, n);
    launch_scale(st, w, w, h->scal + 4, ne);
  } else {
    // one pass with ||w||^2 (V_{j+1} is w itself), DGKS test, normalisation fused
    multidot(h, h->V, ne, j + 2, w, h->h1);
    {
      KScope k(h, IRK_K_OTHER, 0, 0);
      launch_orth_decide(st, j, h->h1, h->h2, 0.5, h->iflag, h->scal + 3, h->scal + 8);
    }
    {
      const double n = (double)ne;
      KScope k(h, IRK_K_AXPY, (j + 3.0) * n * 8, 2.0 * (j + 1) * n);
      launch_multi_axpy(st, w, h->V, ne, j + 1, h->h1, -1.0, ne, h->scal + 8);
    }
    {  // second pass, only when the test asked for it (these kernels return at once otherwise)
      KScope k1(h, IRK_K_OTHER, 0, 0);
      launch_multidot(st, h->V, ne, j + 1, w, ne, h->partial, h->iflag);
      KScope k2(h, IRK_K_OTHER, 0, 0);
      launch_reduce_partials(st, h->partial, j + 1, h->h2, h->iflag);
      KScope k3(h, IRK_K_OTHER, 0, 0);
      launch_multi_axpy(st, w, h->V, ne, j + 1, h->h2, -1.0, ne, nullptr, h->iflag);
      KScope k4(h, IRK_K_OTHER, 0, 0);
      launch_multidot(st, w, 0, 1, w, ne, h->partial, h->iflag);
      KScope k5(h, IRK_K_OTHER, 0, 0);
      launch_reduce_partials(st, h->partial, 1, h->scal + 3, h->iflag);
    }
    {
      KScope k(h, IRK_K_OTHER, 0, 0);
      launch_givens(st, j, ldh, h->H, h->cs, h->sn, h->g, h->h1, h->h2, h->scal + 3, h->scal + 4, r0p, h->scal + 5);
    }
    KScope k(h, IRK_K_OTHER, 0, 0);
    launch_scale(st, w, w, h->scal + 4, ne, h->iflag);
  }
  CK_LAUNCH();
  CK(cudaMemcpyAsync(h->pinned + 2, h->scal + 5, 16, cudaMemcpyDeviceToHost, st));
  return IRK_OK;
}

// Capture body() on the private capture stream into G and instantiate it.  The
// instrumentation counters the capture produced are kept as the graph's
// per-replay increment (the capture itself runs nothing).
int capture_graph(irk_handle* h, irk_handle::IterGraph& G, const std::function<int()>& body) {
  const irk_perf before = h->perf;
  const int vc_before = h->vcycles;
  cudaStream_t saved = h->st;
  h->st = h->cap_stream;
  cudaError_t e = cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    h->st = saved;
    return fail(IRK_ECUDA, "cudaStreamBeginCapture failed: %s", cudaGetErrorString(e));
  }
  const int rc = body();
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(h->st, &graph);
  h->st = saved;
  if (rc != IRK_OK) {
    if (graph) cudaGraphDestroy(graph);
    h->perf = before;
    h->vcycles = vc_before;
    return rc;
  }
  if (e != cudaSuccess) return fail(IRK_ECUDA, "cudaStreamEndCapture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&G.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    G.exec = nullptr;
    return fail(IRK_ECUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
  }
  irk_perf d{};
  d.launches = h->perf.launches - before.launches;
  for (int c = 0; c < IRK_K_COUNT; ++c) {
    d.class_launches[c] = h->perf.class_launches[c] - before.class_launches[c];
    d.class_bytes[c] = h->perf.class_bytes[c] - before.class_bytes[c];
    d.class_flops[c] = h->perf.class_flops[c] - before.class_flops[c];
  }
  G.delta = d;
  G.vcycles = h->vcycles - vc_before;
  h->perf = before;
  h->vcycles = vc_before;
  return IRK_OK;
}

// Run body() through its cached graph G (eager launches while kernels are being timed).
int run_graph(irk_handle* h, irk_handle::IterGraph& G, const std::function<int()>& body) {
  if (!h->use_graphs || h->perf_mask != 0) return body();
  if (!G.exec) TRY(capture_graph(h, G, body));
  CK(cudaGraphLaunch(G.exec, h->st));
  h->perf.launches += G.delta.launches;
  for (int c = 0; c < IRK_K_COUNT; ++c) {
    h->perf.class_launches[c] += G.delta.class_launches[c];
    h->perf.class_bytes[c] += G.delta.class_bytes[c];
    h->perf.class_flops[c] += G.delta.class_flops[c];
  }
  h->vcycles += G.vcycles;
  return IRK_OK;
}

int run_arnoldi_step(irk_handle* h, int j, bool transpose) {
  return run_graph(h, h->graphs[transpose ? 1 : 0][j], [h, j, transpose] { return arnoldi_step(h, j, transpose); });
}

// from_x: start from the contents of x instead of zero; the stopping test stays relative to ||rhs||.
int fgmres(irk_handle* h, const double* rhs, double* x, bool transpose, irk_stats* stats, bool from_x = false) {
  Nvtx range("fgmres");
  cudaStream_t st = h->st;
  const size_t ne = h->ne;
  const int m = h->m, ldh = m + 1;
  h->vcycles = 0;
  if (!from_x) CK(cudaMemsetAsync(x, 0, ne * 8, st));
  // r0 = ||rhs|| kept in scal[9] (the reference of the stopping test); scal[0] = beta, scal[1] = beta^2
  TRY(norm2(h, rhs, 0));
  CK(cudaMemcpyAsync(h->scal + 9, h->scal, 8, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(h->pinned, h->scal, 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const double r0 = h->pinned[0];
  if (!std::isfinite(r0)) return fail(IRK_ENONFINITE, "right-hand side norm is %g", r0);
  int its = 0;
  double rel = (r0 == 0.0) ? 0.0 : 1.0;
  bool conv = (r0 == 0.0);
  const double* r = rhs;
  if (from_x && !conv) {  // r = rhs - S x, beta = ||r|| (as at a restart)
    TRY(apply_operator(h, x, h->tmp, transpose));
    {
      KScope k(h, IRK_K_OTHER, 24.0 * ne, (double)ne);
      launch_sub(st, h->tmp, rhs, h->tmp, ne);
    }
    TRY(norm2(h, h->tmp, 0));
    CK(cudaMemcpyAsync(h->pinned, h->scal, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    rel = h->pinned[0] / r0;
    if (!std::isfinite(rel)) return fail(IRK_ENONFINITE, "initial residual is %g", rel);
    conv = rel <= h->opt.rtol;
    r = h->tmp;
    if (rel >= 1.0) {  // the guess is no better than zero (a fast transient between the steps): drop it
      CK(cudaMemsetAsync(x, 0, ne * 8, st));
      TRY(norm2(h, rhs, 0));
      rel = 1.0;
      r = rhs;
    }
  }
  while (!conv && its < h->opt.maxit) {
    scale(h, h->V, r, h->scal);  // V_0 = r / beta
    {
      KScope k(h, IRK_K_OTHER, 0, 0);
      launch_init_g(st, h->g, m + 1, h->scal);
    }
    int J = 0;
    for (int j = 0; j < m; ++j) {
      {
        Nvtx step_range("arnoldi");
        TRY(run_arnoldi_step(h, j, transpose));
      }
      CK(cudaStreamSynchronize(st));
      rel = h->pinned[2];
      const double hn = h->pinned[3];
      ++its;
      J = j + 1;
      if (!std::isfinite(rel) || !std::isfinite(hn))
        return fail(IRK_ENONFINITE, "FGMRES residual estimate is %g at iteration %d", rel, its);
      if (rel <= h->opt.rtol || hn == 0.0) conv = true;
      if (conv || its >= h->opt.maxit) break;
    }
    {  // x += Z y, y = R^{-1} g
      KScope k(h, IRK_K_OTHER, 0, 0);
      launch_trisolve(st, J, ldh, h->H, h->g, h->y);
    }
    multi_axpy(h, x, h->Z, ne, J, h->y, 1.0);
    CK_LAUNCH();
    // one-pass Gram-Schmidt: the estimate |g_{J}| assumes an orthonormal basis, so confirm it
    const bool verify = conv && h->opt.orth == IRK_ORTH_CGS;
    if ((conv && !verify) || (!conv && its >= h->opt.maxit)) break;
    // restart (or verification): r = rhs - S x in tmp, beta = ||r||
    TRY(apply_operator(h, x, h->tmp, transpose));
    {
      KScope k(h, IRK_K_OTHER, 24.0 * ne, (double)ne);
      launch_sub(st, h->tmp, rhs, h->tmp, ne);
    }
    TRY(norm2(h, h->tmp, 0));
    if (verify) {
      CK(cudaMemcpyAsync(h->pinned, h->scal, 8, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      rel = h->pinned[0] / r0;
      if (!std::isfinite(rel)) return fail(IRK_ENONFINITE, "FGMRES true residual is %g", rel);
      if (rel <= h->opt.rtol) break;
      conv = false;
      if (its >= h->opt.maxit) break;
    }
    r = h->tmp;
  }
  if (stats) {
    stats->fgmres_its = its;
    stats->vcycles = h->vcycles;
    stats->rel_resid = rel;
    stats->converged = conv ? 1 : 0;
  }
  if (!conv) return fail(IRK_ENOCONV, "FGMRES stopped at maxit = %d with relative residual %g", its, rel);
  return IRK_OK;
}

// ----------------------------------------------------------------------------
// DIRK path: for lower-triangular A the stage system is block lower triangular,
// so the stages follow one after another (Sec. 2.3):
//   (M + dt a_ii K) k_i = r_i - dt sum_{j<i} a_ij K k_j,
// each solved by conjugate gradients preconditioned with one V-cycle of the same
// block (symmetric positive definite: the V(nu, nu) cycle with Jacobi smoothing is
// symmetric; with nu_pre != nu_post CG still runs but loses that guarantee).
// transpose: the adjoint system, upper triangular in A^T, runs the stages backwards.
// ----------------------------------------------------------------------------
template <typename T, typename C>
void cg_precondition(irk_handle* h, int i, const double* r, double* z, bool transpose) {
  const int nu1 = transpose ? h->opt.nu_post : h->opt.nu_pre;
  const int nu2 = transpose ? h->opt.nu_pre : h->opt.nu_post;
  if constexpr (std::is_same<T, double>::value) {
    vcycle<T, C>(h, 1, i, r, z, nu1, nu2);
  } else {
    using MG = MG2<T, C>;
    Level& L0 = h->lev[0];
    const double n = (double)L0.nn, p = sizeof(T);
    {
      KScope k(h, IRK_K_OTHER, n * (8 + p), 0);
      MG::cast_to(h->st, r, (T*)L0.b, L0.nn);
    }
    T* x = vcycle<T, C>(h, 1, i, (const T*)L0.b, nullptr, nu1, nu2);
    KScope k(h, IRK_K_OTHER, n * (8 + p), 0);
    MG::cast_from(h->st, x, z, L0.nn);
  }
}

void cg_prec(irk_handle* h, int i, const double* r, double* z, bool transpose) {
  switch (h->opt.vcycle_prec) {
    case IRK_PREC_FP64: cg_precondition<double, double>(h, i, r, z, transpose); break;
    case IRK_PREC_FP32: cg_precondition<float, float>(h, i, r, z, transpose); break;
    default: cg_precondition<__nv_bfloat16, float>(h, i, r, z, transpose); break;
  }
}

// dot(a, b) of single-stage vectors into scal[slot]
void dot1(irk_handle* h, const double* a, const double* b, int slot) {
  const size_t n = h->lev[0].nn;
  {
    KScope k(h, IRK_K_MULTIDOT, 16.0 * n, 2.0 * n);
    launch_multidot(h->st, a, 0, 1, b, n, h->partial);
  }
  KScope k(h, IRK_K_OTHER, 0, 0);
  launch_reduce_partials(h->st, h->partial, 1, h->scal + slot);
}

void block_apply(irk_handle* h, int i, const double* x, double* y) {
  const Level& L0 = h->lev[0];
  const double sigma = h->dt * h->A[i * h->s + i];
  if (h->dim == 3) {
    const double m = L0.nx - 2;
    KScope k(h, IRK_K_OTHER, 16.0 * L0.nn, 38.0 * m * m * m);
    launch_block_apply3(h->st, L0.nx, mass_stiff_classes(L0), sigma, x, y);
  } else {
    KScope k(h, IRK_K_OTHER, 16.0 * L0.nn + 8.0 * kCoef2 * L0.nn, 31.0 * n_int(L0.nx));
    launch_block_apply(h->st, L0.nx, L0.cf_d, L0.hm, sigma, x, y);
  }
}

// One PCG iteration for stage i; ends by copying ||r||^2 to pinned host memory.
// scal: 10 rz, 11 pq, 12 alpha, 13 beta, 14 rr, 15 rz_new.
int cg_iteration(irk_handle* h, int i, bool transpose) {
  cudaStream_t st = h->st;
  const size_t n = h->lev[0].nn;
  block_apply(h, i, h->cg_p, h->cg_q);
  dot1(h, h->cg_p, h->cg_q, 11);
  {
    KScope k(h, IRK_K_OTHER, 0, 0);
    launch_cg_alpha(st, h->scal + 10, h->scal + 11, h->scal + 12);
  }
  {
    KScope k(h, IRK_K_AXPY, 48.0 * n, 4.0 * n);
    launch_cg_update_xr(st, h->cg_x, h->cg_r, h->cg_p, h->cg_q, h->scal + 12, n);
  }
  dot1(h, h->cg_r, h->cg_r, 14);
  CK_LAUNCH();
  CK(cudaMemcpyAsync(h->pinned + 4, h->scal + 14, 8, cudaMemcpyDeviceToHost, st));
  cg_prec(h, i, h->cg_r, h->cg_z, transpose);
  dot1(h, h->cg_r, h->cg_z, 15);
  {
    KScope k(h, IRK_K_OTHER, 0, 0);
    launch_cg_beta(st, h->scal + 15, h->scal + 10, h->scal + 13);
  }
  {
    KScope k(h, IRK_K_AXPY, 24.0 * n, 2.0 * n);
    launch_cg_update_p(st, h->cg_p, h->cg_z, h->scal + 13, n);
  }
  CK_LAUNCH();
  return IRK_OK;
}

int dirk_solve(irk_handle* h, const double* rhs, double* k, bool transpose, irk_stats* stats) {
  Nvtx range("dirk_cg");
  cudaStream_t st = h->st;
  const int s = h->s;
  Level& L0 = h->lev[0];
  const size_t nn = L0.nn;
  h->vcycles = 0;
  CK(cudaMemsetAsync(k, 0, h->ne * 8, st));
  int its = 0;
  double worst = 0.0;
  bool conv = true;
  Cls4 kc{};
  for (int c = 0; c < 4; ++c) kc.v[0][c] = L0.kcls[c];
  for (int step = 0; step < s; ++step) {
    const int i = transpose ? s - 1 - step : step;
    Vec8 cj{};
    for (int j = 0; j < s; ++j) {
      const bool solved = transpose ? (j > i) : (j < i);
      cj.v[j] = solved ? h->dt * (transpose ? h->A[j * s + i] : h->A[i * s + j]) : 0.0;
    }
    {  // b = r_i - dt sum_j a_ij K k_j
      KScope kk(h, IRK_K_BLOCK_RHS, (double)nn * 8 * (2 + s), 19.0 * s * (double)nn);
      if (h->dim == 3)
        MG3<double, double>::block_rhs(s, st, L0.nx, kc, rhs, k, i, cj, h->cg_b);
      else
        MG2<double, double>::block_rhs(s, st, L0.nx, L0.cf_d, rhs, k, i, cj, h->cg_b);
    }
    dot1(h, h->cg_b, h->cg_b, 14);
    CK_LAUNCH();
    CK(cudaMemcpyAsync(h->pinned + 4, h->scal + 14, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const double bb = h->pinned[4];
    if (!std::isfinite(bb)) return fail(IRK_ENONFINITE, "stage %d right-hand side norm is %g", i, bb);
    double rel = 0.0;
    if (bb > 0.0) {
      CK(cudaMemsetAsync(h->cg_x, 0, nn * 8, st));
      CK(cudaMemcpyAsync(h->cg_r, h->cg_b, nn * 8, cudaMemcpyDeviceToDevice, st));
      cg_prec(h, i, h->cg_r, h->cg_z, transpose);
      CK(cudaMemcpyAsync(h->cg_p, h->cg_z, nn * 8, cudaMemcpyDeviceToDevice, st));
      dot1(h, h->cg_r, h->cg_z, 10);
      int it = 0;
      rel = 1.0;
      while (it < h->opt.maxit) {
        auto& G = h->cg_graphs[transpose ? 1 : 0][i];
        TRY(run_graph(h, G, [h, i, transpose] { return cg_iteration(h, i, transpose); }));
        CK(cudaStreamSynchronize(st));
        ++it;
        rel = std::sqrt(std::max(h->pinned[4], 0.0) / bb);
        if (!std::isfinite(h->pinned[4])) return fail(IRK_ENONFINITE, "CG residual is %g", h->pinned[4]);
        if (rel <= h->opt.rtol) break;
      }
      its += it;
      if (rel > h->opt.rtol) conv = false;
    }
    worst = std::max(worst, rel);
    KScope kk(h, IRK_K_OTHER, (double)nn * 16, 0);
    if (h->dim == 3)
      MG3<double, double>::scatter_stage(s, st, L0.nx, h->cg_x, i, k);
    else
      MG2<double, double>::scatter_stage(s, st, L0.nx, h->cg_x, i, k);
  }
  CK_LAUNCH();
  if (stats) {
    stats->fgmres_its = its;
    stats->vcycles = h->vcycles;
    stats->rel_resid = worst;
    stats->converged = conv ? 1 : 0;
  }
  if (!conv) return fail(IRK_ENOCONV, "CG stopped at maxit = %d with relative residual %g", h->opt.maxit, worst);
  return IRK_OK;
}

// After work that may have run the multigrid tail kernel: a grid-barrier wait that ran out there is
// reported as IRK_ECUDA (the results of the call are invalid) and the barrier state is cleared.
int tail_status(irk_handle* h) {
  if (!h->tail_used) return IRK_OK;
  int* flag = reinterpret_cast<int*>(h->pinned + 6);
  CK(cudaMemcpyAsync(flag, h->tail_state + 2, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (*flag == 0) return IRK_OK;
  CK(cudaMemsetAsync(h->tail_state, 0, 4 * sizeof(unsigned), h->st));
  CK(cudaStreamSynchronize(h->st));
  return fail(IRK_ECUDA, "a grid barrier of the multigrid tail kernel timed out: the results of this call are invalid");
}

int solve(irk_handle* h, const double* rhs, double* k, bool transpose, irk_stats* stats, bool from_k = false) {
  const int rc = (h->opt.solver == IRK_SOLVER_DIRK_CG) ? dirk_solve(h, rhs, k, transpose, stats)
                                                        : fgmres(h, rhs, k, transpose, stats, from_k);
  const int ts = tail_status(h);
  return ts != IRK_OK ? ts : rc;
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

void irk_default_options(irk_options* o) {
  if (!o) return;
  o->precond = IRK_PC_LOWER;
  o->vcycle_prec = IRK_PREC_FP64;
  o->nu_pre = 2;
  o->nu_post = 2;
  o->omega = 2.0 / 3.0;
  o->rtol = 1e-10;
  o->restart = 50;
  o->maxit = 500;
  o->orth = IRK_ORTH_CGS2;
  o->solver = IRK_SOLVER_FGMRES;
  o->splitting = IRK_SPLIT_AI;
  o->warm_start = 0;
}

const char* irk_last_error(void) { return g_err.c_str(); }

int irk_perf_select(irk_handle* h, unsigned class_mask) {
  if (!h) return fail(IRK_EINVAL, "null handle");
  perf_drain(h, false);
  h->perf = irk_perf{};
  h->perf_mask = class_mask & ((1u << IRK_K_COUNT) - 1);
  return IRK_OK;
}

int irk_perf_read(irk_handle* h, irk_perf* out) {
  if (!h || !out) return fail(IRK_EINVAL, "null argument");
  perf_drain(h, true);
  *out = h->perf;
  return IRK_OK;
}

int irk_create(irk_handle** out, const irk_mesh* mesh, const irk_tableau* tab, double dt, const irk_options* opt,
               void* stream) {
  try {
    g_err.clear();
    return create(out, mesh, tab, dt, opt, stream);
  } catch (const std::bad_alloc&) {
    return fail(IRK_ENOMEM, "host allocation failed");
  } catch (...) {
    return fail(IRK_EINVAL, "unexpected host exception in irk_create");
  }
}

int irk_destroy(irk_handle* h) {
  if (!h) return IRK_OK;
  cudaStreamSynchronize(h->st);
  destroy(h);
  return IRK_OK;
}

int irk_reset_initial_guess(irk_handle* h) {
  if (!h) return fail(IRK_EINVAL, "null handle");
  h->k_from_step = false;
  return IRK_OK;
}

int irk_set_kappa(irk_handle* h, const double* kappa) {
  if (!h) return fail(IRK_EINVAL, "null handle");
  if (h->dim != 2) return fail(IRK_EINVAL, "irk_set_kappa: dim = 3 supports kappa = 1 only");
  if (!kappa) return fail(IRK_EINVAL, "null kappa");
  try {
    const size_t nc = (size_t)h->N * h->N;
    for (size_t i = 0; i < nc; ++i)
      if (!(kappa[i] > 0.0) || !std::isfinite(kappa[i]))
        return fail(IRK_EINVAL, "kappa[%zu] = %g is not positive and finite", i, kappa[i]);
    CK(cudaStreamSynchronize(h->st));
    h->kappa.assign(kappa, kappa + nc);
    return build_operators(h);
  } catch (...) {
    return fail(IRK_ENOMEM, "host allocation failed");
  }
}

int irk_apply_operator(irk_handle* h, const double* x, double* y, int transpose) {
  if (!h || !x || !y) return fail(IRK_EINVAL, "null argument");
  const size_t bytes = h->ne * 8;
  const void* xd;
  void* yd;
  bool yhost;
  TRY(dev_in(h, x, bytes, 0, &xd));
  TRY(dev_out(h, y, bytes, 1, &yd, &yhost));
  TRY(apply_operator(h, (const double*)xd, (double*)yd, transpose != 0));
  if (yhost) TRY(dev_out_finish(h, y, yd, bytes));
  CK(cudaStreamSynchronize(h->st));
  return IRK_OK;
}

int irk_apply_mass(irk_handle* h, const double* x, double* y) {
  if (!h || !x || !y) return fail(IRK_EINVAL, "null argument");
  if (h->dim != 2) return fail(IRK_EINVAL, "irk_apply_mass is implemented for dim = 2");
  const Level& L0 = h->lev[0];
  const size_t bytes = L0.nn * 8;
  const void* xd;
  void* yd;
  bool yhost;
  TRY(dev_in(h, x, bytes, 0, &xd));
  TRY(dev_out(h, y, bytes, 1, &yd, &yhost));
  {
    KScope k(h, IRK_K_OTHER, 16.0 * L0.nn, 11.0 * n_int(L0.nx));
    launch_mass_apply(h->st, L0.nx, L0.hm, (const double*)xd, (double*)yd);
  }
  CK_LAUNCH();
  if (yhost) TRY(dev_out_finish(h, y, yd, bytes));
  CK(cudaStreamSynchronize(h->st));
  return IRK_OK;
}

int irk_apply_preconditioner(irk_handle* h, const double* v, double* z, int transpose) {
  Nvtx range("irk_apply_preconditioner");
  if (!h || !v || !z) return fail(IRK_EINVAL, "null argument");
  if (transpose && h->opt.splitting != IRK_SPLIT_AI)
    return fail(IRK_EINVAL, "the transposed preconditioner needs the AI splitting");
  const size_t bytes = h->ne * 8;
  const void* vd;
  void* zd;
  bool zhost;
  TRY(dev_in(h, v, bytes, 0, &vd));
  TRY(dev_out(h, z, bytes, 1, &zd, &zhost));
  // the triangular sweeps read z for the stages already solved: start from zero
  CK(cudaMemsetAsync(zd, 0, bytes, h->st));
  h->vcycles = 0;
  TRY(precond(h, (const double*)vd, (double*)zd, transpose != 0));
  if (zhost) TRY(dev_out_finish(h, z, zd, bytes));
  CK(cudaStreamSynchronize(h->st));
  return tail_status(h);
}

int irk_solve(irk_handle* h, const double* r, double* k, irk_stats* stats) {
  Nvtx range("irk_solve");
  if (!h || !r || !k) return fail(IRK_EINVAL, "null argument");
  const size_t bytes = h->ne * 8;
  const void* rd;
  void* kd;
  bool khost;
  TRY(dev_in(h, r, bytes, 0, &rd));
  TRY(dev_out(h, k, bytes, 1, &kd, &khost));
  const bool ia = (h->opt.splitting == IRK_SPLIT_IA);
  // IA: w in h->k (not h->tmp, which FGMRES uses for restart residuals)
  if (ia) h->k_from_step = false;
  const int rc = solve(h, (const double*)rd, ia ? h->k : (double*)kd, false, stats);
  if (rc != IRK_OK && rc != IRK_ENOCONV) return rc;
  if (ia) {  // k = (A^{-1} (x) I) w
    KScope kk(h, IRK_K_OTHER, 16.0 * h->ne, 2.0 * h->s * h->ne);
    launch_stage_mix(h->s, h->st, h->lev[0].nn, ia_mixing(h, false), h->k, (double*)kd);
    CK_LAUNCH();
  }
  if (khost) TRY(dev_out_finish(h, k, kd, bytes));
  CK(cudaStreamSynchronize(h->st));
  return rc;
}

int irk_step(irk_handle* h, const double* u_n, const double* f_space, const double* f_coef, const double* f_stages,
             double* u_np1, double* stages_out, irk_stats* stats) {
  Nvtx range("irk_step");
  if (!h || !u_n || !u_np1) return fail(IRK_EINVAL, "null argument");
  const int s = h->s;
  const size_t nn = h->lev[0].nn, nb = nn * 8, sb = h->ne * 8;
  const void *ud, *fd, *fsd;
  void *outd, *kd;
  bool outhost, khost;
  TRY(dev_in(h, u_n, nb, 2, &ud));
  TRY(dev_in(h, f_space, nb, 3, &fd));
  TRY(dev_in(h, f_stages, sb, 4, &fsd));
  TRY(dev_out(h, u_np1, nb, 5, &outd, &outhost));
  TRY(dev_out(h, stages_out, sb, 6, &kd, &khost));
  Vec8 fc{};
  for (int i = 0; i < s; ++i) fc.v[i] = f_coef ? f_coef[i] : 1.0;
  {
    const double nn_d = (double)nn;
    KScope k(h, IRK_K_OTHER, nn_d * (8 + 8 + 8.0 * kCoef2 + 8.0 * s + (fsd ? 8.0 * s : 0.0)),
             n_int(h->lev[0].nx) * (17.0 + 2.0 * s));
    if (h->dim == 3)
      launch_rhs3(s, h->st, h->lev[0].nx, mass_stiff_classes(h->lev[0]), (const double*)ud, (const double*)fd, fc,
                  (const double*)fsd, h->rhs);
    else
      launch_rhs(s, h->st, h->lev[0].nx, h->lev[0].cf_d, (const double*)ud, (const double*)fd, fc,
                 (const double*)fsd, h->rhs);
  }
  CK_LAUNCH();
  // warm start: h->k still holds the previous step's stages (w in the IA form) unless another call replaced them
  const bool warm = h->opt.warm_start && h->k_from_step;
  h->k_from_step = false;
  const int rc = solve(h, h->rhs, h->k, false, stats, warm);
  if (rc != IRK_OK && rc != IRK_ENOCONV) return rc;
  h->k_from_step = true;
  Vec8 bdt{};
  const bool ia = (h->opt.splitting == IRK_SPLIT_IA);
  for (int i = 0; i < s; ++i) bdt.v[i] = h->dt * (ia ? h->bIA[i] : h->b[i]);  // IA: dt (A^{-T} b) . w
  {
    KScope k(h, IRK_K_OTHER, (double)nn * (16.0 + 8.0 * s), 2.0 * s * n_int(h->lev[0].nx));
    if (h->dim == 3)
      launch_rk_update3(s, h->st, h->lev[0].nx, (const double*)ud, h->k, bdt, (double*)outd);
    else
      launch_rk_update(s, h->st, h->lev[0].nx, (const double*)ud, h->k, bdt, (double*)outd);
  }
  CK_LAUNCH();
  if (kd && ia) {  // stages k = (A^{-1} (x) I) w
    KScope kk(h, IRK_K_OTHER, 16.0 * h->ne, 2.0 * s * h->ne);
    launch_stage_mix(s, h->st, nn, ia_mixing(h, false), h->k, (double*)kd);
    CK_LAUNCH();
  } else if (kd) {
    CK(cudaMemcpyAsync(kd, h->k, sb, cudaMemcpyDeviceToDevice, h->st));
  }
  if (outhost) TRY(dev_out_finish(h, u_np1, outd, nb));
  if (khost) TRY(dev_out_finish(h, stages_out, kd, sb));
  CK(cudaStreamSynchronize(h->st));
  return rc;
}

int irk_step_dirichlet(irk_handle* h, const double* u_n, const double* g_stages, const double* f_space,
                       const double* f_coef, const double* f_stages, double* u_np1, double* stages_out,
                       irk_stats* stats) {
  Nvtx range("irk_step_dirichlet");
  if (!h || !u_n || !g_stages || !u_np1) return fail(IRK_EINVAL, "null argument");
  if (!h->ainv_ok) return fail(IRK_EINVAL, "DAE-type boundary conditions need an invertible Butcher matrix");
  const int s = h->s;
  const Level& L0 = h->lev[0];
  const size_t nn = L0.nn, nb = nn * 8, sb = h->ne * 8;
  const bool ia = (h->opt.splitting == IRK_SPLIT_IA);
  const void *ud, *gd, *fd, *fsd;
  void *outd, *kd;
  bool outhost, khost;
  TRY(dev_in(h, u_n, nb, 2, &ud));
  TRY(dev_in(h, g_stages, sb, 7, &gd));
  TRY(dev_in(h, f_space, nb, 3, &fd));
  TRY(dev_in(h, f_stages, sb, 4, &fsd));
  TRY(dev_out(h, u_np1, nb, 5, &outd, &outhost));
  TRY(dev_out(h, stages_out, sb, 6, &kd, &khost));
  if (!h->bnd) TRY(dalloc(&h->bnd, sb));  // its own buffer, not h->tmp: FGMRES restarts use that
  h->k_from_step = false;
  // boundary unknowns of the solved system: k_B = A^{-1} (g - u_n) / dt (AI), w_B = (g - u_n) / dt (IA)
  Mat4 bmix{};
  for (int i = 0; i < s; ++i)
    for (int j = 0; j < s; ++j) bmix.v[i * s + j] = (ia ? double(i == j) : h->Ainv[i * s + j]) / h->dt;
  {
    KScope k(h, IRK_K_OTHER, (double)nn * 8.0 * (1 + 2 * s), 2.0 * s * s * nn);
    if (h->dim == 3)
      launch_bc_stages3(s, h->st, L0.nx, bmix, (const double*)ud, (const double*)gd, h->bnd);
    else
      launch_bc_stages(s, h->st, L0.nx, bmix, (const double*)ud, (const double*)gd, h->bnd);
  }
  CK_LAUNCH();
  // r = F - K u_n (u_n with its boundary values) - S x_B on the interior rows
  Vec8 fc{};
  for (int i = 0; i < s; ++i) fc.v[i] = f_coef ? f_coef[i] : 1.0;
  {
    KScope k(h, IRK_K_OTHER, (double)nn * (8 + 8 + 8.0 * kCoef2 + 8.0 * s + (fsd ? 8.0 * s : 0.0)),
             n_int(L0.nx) * (17.0 + 2.0 * s));
    if (h->dim == 3)
      launch_rhs3(s, h->st, L0.nx, mass_stiff_classes(L0), (const double*)ud, (const double*)fd, fc,
                  (const double*)fsd, h->rhs, 1);
    else
      launch_rhs(s, h->st, L0.nx, L0.cf_d, (const double*)ud, (const double*)fd, fc, (const double*)fsd, h->rhs,
                 1);
  }
  CK_LAUNCH();
  TRY(apply_operator(h, h->bnd, h->k, false));
  {
    KScope k(h, IRK_K_OTHER, 24.0 * h->ne, (double)h->ne);
    launch_sub(h->st, h->rhs, h->rhs, h->k, h->ne);
  }
  CK_LAUNCH();
  const int rc = solve(h, h->rhs, h->k, false, stats);
  if (rc != IRK_OK && rc != IRK_ENOCONV) return rc;
  {
    KScope k(h, IRK_K_OTHER, 24.0 * h->ne, (double)h->ne);
    launch_add(h->st, h->k, h->k, h->bnd, h->ne);
  }
  CK_LAUNCH();
  Vec8 bdt{};
  for (int i = 0; i < s; ++i) bdt.v[i] = h->dt * (ia ? h->bIA[i] : h->b[i]);
  {
    KScope k(h, IRK_K_OTHER, (double)nn * (16.0 + 8.0 * s), 2.0 * s * nn);
    if (h->dim == 3)
      launch_rk_update3(s, h->st, L0.nx, (const double*)ud, h->k, bdt, (double*)outd, 1);
    else
      launch_rk_update(s, h->st, L0.nx, (const double*)ud, h->k, bdt, (double*)outd, 1);
  }
  CK_LAUNCH();
  if (kd && ia) {
    KScope kk(h, IRK_K_OTHER, 16.0 * h->ne, 2.0 * s * h->ne);
    launch_stage_mix(s, h->st, nn, ia_mixing(h, false), h->k, (double*)kd);
    CK_LAUNCH();
  } else if (kd) {
    CK(cudaMemcpyAsync(kd, h->k, sb, cudaMemcpyDeviceToDevice, h->st));
  }
  if (outhost) TRY(dev_out_finish(h, u_np1, outd, nb));
  if (khost) TRY(dev_out_finish(h, stages_out, kd, sb));
  CK(cudaStreamSynchronize(h->st));
  return rc;
}

int irk_step_adjoint(irk_handle* h, const double* u_n, const double* stages, const double* lam_np1, double* lam_n,
                     double* grad_accum, irk_stats* stats) {
  Nvtx range("irk_step_adjoint");
  if (!h || !u_n || !stages || !lam_np1 || !lam_n) return fail(IRK_EINVAL, "null argument");
  if (h->dim != 2) return fail(IRK_EINVAL, "irk_step_adjoint is implemented for dim = 2");
  if (h->opt.splitting != IRK_SPLIT_AI) return fail(IRK_EINVAL, "irk_step_adjoint needs the AI splitting");
  const int s = h->s;
  const size_t nn = h->lev[0].nn, nb = nn * 8, sb = h->ne * 8, gb = (size_t)h->N * h->N * 8;
  const void *ud, *kd, *ld;
  void *lod, *gd = nullptr;
  bool lohost, ghost = false;
  TRY(dev_in(h, u_n, nb, 2, &ud));
  TRY(dev_in(h, stages, sb, 4, &kd));
  TRY(dev_in(h, lam_np1, nb, 3, &ld));
  TRY(dev_out(h, lam_n, nb, 5, &lod, &lohost));
  if (grad_accum) {
    if (is_device_ptr(grad_accum)) {
      gd = grad_accum;
    } else {
      const void* gin;
      TRY(dev_in(h, grad_accum, gb, 7, &gin));  // accumulate onto the caller's values
      gd = (void*)gin;
      ghost = true;
    }
  }
  // rhs_i = dt b_i lam_{n+1}
  Vec8 fc{};
  for (int i = 0; i < s; ++i) fc.v[i] = h->dt * h->b[i];
  {
    KScope k(h, IRK_K_OTHER, (double)nn * (8.0 + 8.0 * s), n_int(h->lev[0].nx) * s);
    launch_rhs(s, h->st, h->lev[0].nx, h->lev[0].cf_d, nullptr, (const double*)ld, fc, nullptr, h->rhs);
  }
  CK_LAUNCH();
  h->k_from_step = false;
  const int rc = solve(h, h->rhs, h->k, true, stats);  // h->k = mu
  if (rc != IRK_OK && rc != IRK_ENOCONV) return rc;
  if (gd) {
    Mat4 dtA = mixing(h, false);
    const double ncell = (double)h->N * h->N;
    KScope k(h, IRK_K_OTHER, ncell * 24.0 + (double)nn * (8.0 + 16.0 * s), ncell * s * (4.0 * (1 + 2 * s) + 36.0));
    launch_cell_gradient(s, h->st, h->N, h->kappa.empty() ? nullptr : h->kappa_d, (const double*)ud,
                         (const double*)kd, dtA, h->k, (double*)gd);
  }
  {
    KScope k(h, IRK_K_OTHER, (double)nn * (24.0 + 8.0 * s + 8.0 * kCoef2), 18.0 * s * n_int(h->lev[0].nx));
    launch_adjoint_lambda(s, h->st, h->lev[0].nx, h->lev[0].cf_d, (const double*)ld, h->k, (double*)lod);
  }
  CK_LAUNCH();
  if (lohost) TRY(dev_out_finish(h, lam_n, lod, nb));
  if (ghost) TRY(dev_out_finish(h, grad_accum, gd, gb));
  CK(cudaStreamSynchronize(h->st));
  return rc;
}

}  // extern "C"

// ============================================================================
// Preconditioner application that allocates nothing.
//
// Some callers cannot allocate device memory at the time they apply the
// preconditioner: host threads that must not enter the allocator (real-time
// loops whose latency a cudaMalloc or an allocator's lock would break), and
// embeddings in a framework that owns all device memory and hands the library a
// fixed budget.  For them, irk_apply_preconditioner_noalloc runs the same V-cycle
// preconditioner as irk_apply_preconditioner, but its multigrid level vectors
// live in one file-scope device array of kNoAllocScratchBytes (16 MiB) instead of
// the handle's buffers.  Every GPU that loads the library holds that array until
// the process exits.  The triangular sweeps still write two buffers the handle
// allocated at create time (the first-sweep buffer x1_d of FP64 cycles and the
// stage-major copies zt of FP32 / BF16 cycles), so calls on one handle must not
// overlap either.
// ============================================================================
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_device_ptr[256] = {};  // device address of g_noalloc_scratch, per device ordinal

// In host code g_noalloc_scratch only names a host-side stand-in, so the
// device address is fetched once per device (with that device current) and
// cached; this is the only set-up the entry point does.
int noalloc_scratch_address(void** out) {
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return fail(IRK_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (g_noalloc_device_ptr[dev] == nullptr) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_device_ptr[dev] = p;
  }
  *out = g_noalloc_device_ptr[dev];
  return IRK_OK;
}

inline size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

}  // namespace

extern "C" int irk_apply_preconditioner_noalloc(irk_handle* h, const double* v, double* z, int transpose) {
  if (!h || !v || !z) return fail(IRK_EINVAL, "null argument");
  if (transpose && h->opt.splitting != IRK_SPLIT_AI)
    return fail(IRK_EINVAL, "the transposed preconditioner needs the AI splitting");
  if (!is_device_ptr(v) || !is_device_ptr(z))
    return fail(IRK_EINVAL, "irk_apply_preconditioner_noalloc takes device pointers only");
  // scratch layout: four level vectors (xa, xb, b, r) per level, 256-byte aligned
  const size_t vb = prec_bytes(h->opt.vcycle_prec);
  size_t need = 0;
  for (const Level& Lv : h->lev) need += 4 * align256(Lv.nn * (size_t)h->s * vb);
  if (need > kNoAllocScratchBytes)
    return fail(IRK_EINVAL, "this handle's V-cycle needs %zu bytes of scratch; the no-allocation entry point has %zu",
                need, kNoAllocScratchBytes);
  void* base = nullptr;
  TRY(noalloc_scratch_address(&base));
  // the array keeps the previous call's contents: level vectors must start with zero boundaries
  CK(cudaMemsetAsync(base, 0, need, h->st));
  CK(cudaMemsetAsync(z, 0, h->ne * 8, h->st));
  // lend the scratch to the handle's levels for this call; instrumentation timing is
  // switched off because it may create CUDA events
  void* saved[16][4];  // levels <= 14 (validated at create)
  for (size_t l = 0; l < h->lev.size(); ++l) {
    saved[l][0] = h->lev[l].xa, saved[l][1] = h->lev[l].xb, saved[l][2] = h->lev[l].b, saved[l][3] = h->lev[l].r;
  }
  const unsigned saved_mask = h->perf_mask;
  unsigned char* cur = static_cast<unsigned char*>(base);
  for (Level& Lv : h->lev) {
    const size_t bytes = align256(Lv.nn * (size_t)h->s * vb);
    Lv.xa = cur, cur += bytes;
    Lv.xb = cur, cur += bytes;
    Lv.b = cur, cur += bytes;
    Lv.r = cur, cur += bytes;
  }
  h->perf_mask = 0;
  h->vcycles = 0;
  const int rc = precond(h, v, z, transpose != 0);
  for (size_t l = 0; l < h->lev.size(); ++l) {
    h->lev[l].xa = saved[l][0], h->lev[l].xb = saved[l][1], h->lev[l].b = saved[l][2], h->lev[l].r = saved[l][3];
  }
  h->perf_mask = saved_mask;
  if (rc != IRK_OK) return rc;
  CK(cudaStreamSynchronize(h->st));
  return tail_status(h);
}
