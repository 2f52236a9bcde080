// Host-side launchers of the solver's CUDA kernels (internal to libirk.so).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>

namespace irk {

struct Vec8;
struct Mat4;

// 3D constant-coefficient stencils: per stage, the values of the four offset classes
// (centre, 6 faces, 12 edges, 8 corners) of a 27-point Q1 stencil.
struct Cls4 {
  double v[4][4];
};

// The small-level tail of a 2D block V(2, 2) cycle run by one cooperative launch (mg2d_tail.cuh):
// the down legs of levels[0 .. levels-1] (finest first), the coarsest solve, the up legs.
constexpr int kTailMaxLevels = 8;
// Where the last finest-level up leg of an FP32 / BF16 cycle writes its result instead of its level
// vector (z == nullptr: the level vector as usual).  One block (i >= 0): stage i of the sf-interleaved FP64
// stage vector z, times scale, and the stage-major copy zt.  All stages of a batched or monolithic cycle
// (i < 0, S == sf): z[p sf + k] = sc[k] * x_k.  Each value is rounded to T first, as the stored iterate was.
template <typename T>
struct ZSink {
  double* z = nullptr;
  int sf = 1;
  int i = 0;
  double scale = 1.0;
  T* zt = nullptr;
  double sc[4] = {1.0, 1.0, 1.0, 1.0};
};

template <typename C>
struct TailSpec {
  int levels;                      // leg levels, 1 .. kTailMaxLevels
  int nx[kTailMaxLevels];          // nodes per axis of each leg level
  const C* rec[kTailMaxLevels];    // B-records of the cycle's first block (stage-major, stride rstride)
  size_t rstride[kTailMaxLevels];
  const C* dinv[kTailMaxLevels];   // omega / diag(B), dstride values per node
  void* b[kTailMaxLevels];         // right-hand sides (b[0] is the input)
  void* xa[kTailMaxLevels];        // down-leg iterates
  void* xb[kTailMaxLevels];        // up-leg results (xb[0] is the output)
  int nxc;                         // coarsest level: nodes per axis
  const C* binv;                   // S dense inverses of the coarsest blocks
  void* bc;                        // coarsest right-hand side and solution
  void* xc;
  unsigned* bar;                   // grid barrier state (two words, zero between launches)
  int* err;                        // set to 1 when a barrier wait ran out
  long long spin_cycles;           // barrier wait limit in SM clock cycles
};

// Multigrid kernels for one precision: storage T, arithmetic C (mg2d.cuh).
template <typename T, typename C>
struct MG2 {
  static void jacobi(int S, cudaStream_t st, int nx, const C* cf, double hm, const Vec8& sigma, const C* dinv,
                     int dstride, const T* xin, const T* b, T* xout);
  static void residual(int S, cudaStream_t st, int nx, const C* cf, double hm, const Vec8& sigma, const T* x,
                       const T* b, T* r);
  // two sweeps from a zero guess in one pass (rec != nullptr: B_i records, else hm M + sigma K)
  static void jacobi2z(int S, cudaStream_t st, int nx, const C* cf, double hm, const Vec8& sigma, const C* rec,
                       size_t rstride, const C* dinv, int dstride, const T* b, T* xout);
  // the same with B_i = M + sigma_i K stored per stage (stage-major records, stride rstride)
  static void jacobi_rec(int S, cudaStream_t st, int nx, const C* rec, size_t rstride, const C* dinv, int dstride,
                         const T* xin, const T* b, T* xout);
  // one block after its first sweep x1: x_out = x1 + sum_k c'_k x_k with the nine scaled planes sr
  // (scaled_jacobi_records_2d); nine FMAs per node
  static void jacobi_scaled(cudaStream_t st, int nx, const C* sr, const T* x1, const T* xin, T* xout);
  // the same sweep writing scale * x_out into stage i of the SF-interleaved FP64 vector z (FP64 only;
  // false, nothing launched, otherwise)
  static bool jacobi_scaled_z(int SF, cudaStream_t st, int nx, const C* sr, const T* x1, const T* xin, int i,
                              double* z, double scale);
  static void residual_rec(int S, cudaStream_t st, int nx, const C* rec, size_t rstride, const T* x, const T* b,
                           T* r);
  static void restrict_(int S, cudaStream_t st, int nxf, const T* rf, int nxc, T* bc);
  static void prolong_add(int S, cudaStream_t st, int nxc, const T* ec, int nxf, T* xf);
  // d1 != nullptr: also x1 = d1 * out (the block V-cycle's first sweep from a zero guess)
  // zt != nullptr: the solved stages from zt + j * zstride (V-cycle outputs in precision T, cj scaled
  // accordingly) instead of the FP64 stage vector z
  static void block_rhs(int SF, cudaStream_t st, int nx, const C* cf, const double* v, const double* z, int i,
                        const Vec8& cj, T* out, const C* d1 = nullptr, T* x1 = nullptr, const T* zt = nullptr,
                        size_t zstride = 0);
  // zt != nullptr: also a copy of x in precision T
  static void scatter_stage(int SF, cudaStream_t st, int nx, const T* x, int i, double* z, double scale = 1.0,
                            T* zt = nullptr);
  // IA form: out = v_i - sum_j cj[j] M z_j
  static void block_rhs_mass(int SF, cudaStream_t st, int nx, double hm, const double* v, const double* z, int i,
                             const Vec8& cj, T* out, const C* d1 = nullptr, T* x1 = nullptr, const T* zt = nullptr,
                             size_t zstride = 0);
  static void cast_to(cudaStream_t st, const double* src, T* dst, size_t n);
  static void cast_from(cudaStream_t st, const T* src, double* dst, size_t n);
  // coarsest level (nxc nodes per axis, (nxc - 2)^2 unknowns in row-major interior order)
  static void coarse_solve(int S, cudaStream_t st, int nxc, const C* binv, const T* b, T* x);
  // fused V(2, 2) legs of a coarse level (mg2d_legs.cuh): x = J(J(0; b)), b_c = P^T (b - B x); and
  // xout = J(J(xin + P e_c; b)) (xout != xin).  rec != nullptr: B_i records, else hm M + sigma K.
  // srec != nullptr (S = 1, with rec): the sweeps use the block's scaled stencil (scaled_jacobi_records_2d)
  static void down_leg(int S, cudaStream_t st, int nxf, const C* cf, double hm, const Vec8& sigma, const C* rec,
                       size_t rstride, const C* dinv, int dstride, const T* b, T* xout, int nxc, T* bc,
                       const C* srec = nullptr);
  // zs.z != nullptr (S = 1): the up leg writes its result into stage zs.i of the FP64 stage vector instead
  static void up_leg(int S, cudaStream_t st, int nxf, const C* cf, double hm, const Vec8& sigma, const C* rec,
                     size_t rstride, const C* dinv, int dstride, const T* xin, const T* b, int nxc, const T* ec,
                     T* xout, const C* srec = nullptr, const ZSink<T>& zs = ZSink<T>{});
  // monolithic multigrid (mmg2d.cuh) on S-interleaved level vectors, mix = dt A (or dt A^T):
  // x_out = x_in + omega D^{-1} (b - S_l x_in) with the per-node s x s inverses dblk (x_in == nullptr:
  // zero guess); r = b - S_l x; exact coarsest solve with the dense inverse of the coupled system.
  // transpose: the relaxation with D^{-T} (pass mix = dt A^T) and the coarsest solve with inv^T
  static void mmg_smooth(int S, cudaStream_t st, int nx, const C* cf, double hm, const Mat4& mix, const C* dblk,
                         const T* xin, const T* b, T* xout, bool transpose = false);
  static void mmg_residual(int S, cudaStream_t st, int nx, const C* cf, double hm, const Mat4& mix, const T* x,
                           const T* b, T* r);
  static void mmg_coarse_solve(int S, cudaStream_t st, int nxc, const C* inv, const T* b, T* x,
                               bool transpose = false);
  // fused V(2, 2) legs of a coarse level of the monolithic cycle (mg2d_legs.cuh), as down_leg / up_leg
  // with the stage-coupled relaxation
  static void mmg_down_leg(int S, cudaStream_t st, int nxf, const C* cf, double hm, const Mat4& mix, const C* dblk,
                           bool transpose, const T* b, T* xout, int nxc, T* bc);
  static void mmg_up_leg(int S, cudaStream_t st, int nxf, const C* cf, double hm, const Mat4& mix, const C* dblk,
                         bool transpose, const T* xin, const T* b, int nxc, const T* ec, T* xout,
                         const ZSink<T>& zs = ZSink<T>{});
  // the tail of S batched blocks (S = 1: one block) as one cooperative launch (mg2d_tail.cuh)
  static cudaError_t tail_cycle(int S, cudaStream_t st, const TailSpec<C>& spec, int dstride);
};

// Coarse levels whose finer grid has at least this many nodes per axis run the fused V-cycle legs
// on large tiles (and count as IRK_K_MG_COARSE); smaller ones use small tiles (IRK_K_MG_TAIL).
constexpr int kMgLargeNx = 513;

// 3D multigrid kernels (mg3d.cuh), constant-coefficient stencils.
template <typename T, typename C>
struct MG3 {
  static void jacobi(int S, cudaStream_t st, int n, const Cls4& bc, const Vec8& dinv, const T* xin, const T* b,
                     T* xout);
  static void residual(int S, cudaStream_t st, int n, const Cls4& bc, const T* x, const T* b, T* r);
  static void jacobi2z(int S, cudaStream_t st, int n, const Cls4& bc, const Vec8& dinv, const T* b, T* xout);
  static void restrict_(int S, cudaStream_t st, int nf, const T* rf, int nc, T* bc);
  static void prolong_add(int S, cudaStream_t st, int nc, const T* ec, int nf, T* xf);
  static void block_rhs(int SF, cudaStream_t st, int n, const Cls4& kc, const double* v, const double* z, int i,
                        const Vec8& cj, T* out, const T* zt = nullptr, size_t zstride = 0);
  static void scatter_stage(int SF, cudaStream_t st, int n, const T* x, int i, double* z, double scale = 1.0,
                            T* zt = nullptr);
  static void coarse_solve(int S, cudaStream_t st, int nint, const C* binv, const int* map, const T* b, T* x);
};

// FP64 3D stage-operator kernels (op3d.cu); mc / kc: mass / stiffness class values in v[0].
void launch_stage_apply3(int S, cudaStream_t st, int n, const Cls4& mk, const Mat4& mix, const double* x, double* y);
void launch_rhs3(int S, cudaStream_t st, int n, const Cls4& mk, const double* u, const double* fsp,
                 const Vec8& fcoef, const double* fst, double* r, int raw_u = 0);
void launch_block_apply3(cudaStream_t st, int n, const Cls4& mk, double sigma, const double* x, double* y);
void launch_stage_apply3_ia(int S, cudaStream_t st, int n, const Cls4& mk, const Mat4& mixM, double dt,
                            const double* x, double* y);
void launch_rk_update3(int S, cudaStream_t st, int n, const double* u, const double* k, const Vec8& bdt, double* out,
                       int all_nodes = 0);
void launch_bc_stages3(int S, cudaStream_t st, int n, const Mat4& ainv_dt, const double* u, const double* g,
                       double* kb);

// FP64 stage-operator kernels (op2d.cu).
void launch_stage_apply(int S, cudaStream_t st, int nx, const double* cf, double hm, const Mat4& mix, const double* x,
                        double* y);
// IA form, crec: per stage the planar records of A^{-1}_ii M + dt K (S blocks); mixM's off-diagonal couples
void launch_stage_apply_ia(int S, cudaStream_t st, int nx, const double* crec, double hm, const Mat4& mixM,
                           const double* x, double* y);
void launch_stage_mix(int S, cudaStream_t st, size_t nodes, const Mat4& mix, const double* in, double* out);
void launch_stage_scale(int S, cudaStream_t st, size_t nodes, const Vec8& scale, double* z);
void launch_rhs(int S, cudaStream_t st, int nx, const double* cf, const double* u, const double* fsp,
                const Vec8& fcoef, const double* fst, double* r, int raw_u = 0);
void launch_rk_update(int S, cudaStream_t st, int nx, const double* u, const double* k, const Vec8& bdt,
                      double* out, int all_nodes = 0);
void launch_bc_stages(int S, cudaStream_t st, int nx, const Mat4& ainv_dt, const double* u, const double* g,
                      double* kb);
void launch_adjoint_lambda(int S, cudaStream_t st, int nx, const double* cf, const double* lam_np1, const double* mu,
                           double* lam_n);
void launch_block_apply(cudaStream_t st, int nx, const double* cf, double hm, double sigma, const double* x,
                        double* y);
void launch_mass_apply(cudaStream_t st, int nx, double hm, const double* x, double* y);
void launch_cell_gradient(int S, cudaStream_t st, int N, const double* kappa, const double* u, const double* k,
                          const Mat4& dtA, const double* mu, double* grad);

// Krylov kernels (krylov.cu), FP64.
int krylov_partial_blocks();
// run_if: optional device flag; the kernel does nothing when *run_if == 0.
void launch_multidot(cudaStream_t st, const double* V, size_t ld, int count, const double* w, size_t n,
                     double* partial, const int* run_if = nullptr);
void launch_reduce_partials(cudaStream_t st, const double* partial, int count, double* out,
                            const int* run_if = nullptr);
// w -= sum_k coef[k] V_k and partial sums of V_k . w (k < count) and w . w (entry count) in one pass,
// for count <= krylov_axpy_dot_max() (else nothing is launched and false returned).
int krylov_axpy_dot_max();
bool launch_axpy_dot(cudaStream_t st, double* w, const double* V, size_t ld, int count, const double* coef, size_t n,
                     double* partial);
// w -= sum_k coef[k] V_k (count <= 128) with the partial sums of the updated w . w (count 1 for reduce_partials)
void launch_axpy_norm(cudaStream_t st, double* w, const double* V, size_t ld, int count, const double* coef,
                      size_t n, double* partial);
void launch_multi_axpy(cudaStream_t st, double* w, const double* V, size_t ld, int count, const double* coef,
                       double sign, size_t n, const double* scale = nullptr, const int* run_if = nullptr);
void launch_scale(cudaStream_t st, double* dst, const double* src, const double* denom, size_t n,
                  const int* run_if = nullptr);
void launch_orth_decide(cudaStream_t st, int j, double* h1, double* h2, double eta2, int* redo, double* hn2,
                        double* inv);
void launch_givens(cudaStream_t st, int j, int ldh, double* H, double* cs, double* sn, double* g, const double* h1,
                   const double* h2, const double* hn2, double* hn_out, const double* r0, double* rel_out,
                   int pythag = 0, double* inv_out = nullptr);
void launch_trisolve(cudaStream_t st, int J, int ldh, const double* H, const double* g, double* y);
void launch_sqrt_scalar(cudaStream_t st, const double* in, double* out);
void launch_cg_alpha(cudaStream_t st, const double* rz, const double* pq, double* alpha);
void launch_cg_beta(cudaStream_t st, const double* rz_new, double* rz_old, double* beta);
void launch_cg_update_xr(cudaStream_t st, double* x, double* r, const double* p, const double* q, const double* alpha,
                         size_t n);
void launch_cg_update_p(cudaStream_t st, double* p, const double* z, const double* beta, size_t n);
void launch_sub(cudaStream_t st, double* out, const double* a, const double* b, size_t n);
void launch_add(cudaStream_t st, double* out, const double* a, const double* b, size_t n);
void launch_init_g(cudaStream_t st, double* g, int m1, const double* beta);

}  // namespace irk
