// FP64 kernels of the outer iteration: the stage operator of Sec. 3,
// eq. block_struct_AI, the right-hand side of Sec. 2 eq. rkheat, the RK update
// (Sec. 2) and the pieces of the discrete adjoint step.
#include "common.cuh"
#include "kernels.h"

#include <algorithm>

namespace irk {

namespace {
constexpr int BX = 32, BY = 8;

inline dim3 all_nodes_grid(int nx) { return dim3((nx + BX - 1) / BX, (nx + BY - 1) / BY); }

// (K u)(p) for a caller-supplied nodal vector whose boundary entries must be read as 0.
__device__ __forceinline__ double k_apply_masked(const double* __restrict__ cf, const double* __restrict__ u, int ix,
                                                 int iy, int nx) {
  const int p = ix + nx * iy;
  auto U = [&](int dx, int dy) {
    const int jx = ix + dx, jy = iy + dy;
    return interior2(jx, jy, nx) ? u[jx + nx * jy] : 0.0;
  };
  return rec_apply_xy<double>(cf, p, nx, U);
}
}  // namespace

// The Q1 mass stencil is separable: 36/h^2 M = [1 4 1] (x) [1 4 1].  The stage-operator kernels
// give each thread two vertically adjacent nodes, so the four row sums x_w + 4 x_c + x_e of rows
// iy - 1 .. iy + 2 serve both: 6 FP64 operations per node and stage instead of 10 (on GB300 the
// FP64 pipe, not memory, bounds these kernels).
template <int S>
__device__ __forceinline__ double row_sum(const double* __restrict__ x, int q, int j) {
  return fma(4.0, x[(size_t)q * S + j], x[(size_t)(q - 1) * S + j]) + x[(size_t)(q + 1) * S + j];
}

// Node pair (ix, iy0), (ix, iy0 + 1) of a thread; both rows exist unless iy0 = nx - 1.
struct NodePair {
  int ix, iy0, p0;
  bool two, in0, in1;
  __device__ NodePair(int nx) {
    ix = blockIdx.x * BX + threadIdx.x;
    iy0 = 2 * (blockIdx.y * BY + threadIdx.y);
    p0 = ix + nx * iy0;
    two = iy0 + 1 < nx;
    const bool col = ix >= 1 && ix <= nx - 2;
    in0 = col && iy0 >= 1 && iy0 <= nx - 2;
    in1 = two && col && iy0 + 1 <= nx - 2;
  }
};

// Unscaled mass stencil of stage j at both nodes of the pair (only called when a node is interior,
// so column ix is interior and rows iy0 - 1 .. iy0 + 2 that exist are in range).
template <int S>
__device__ __forceinline__ void mass_pair(const double* __restrict__ x, const NodePair& q, int nx, int j, double& m0,
                                          double& m1) {
  const double r_m = (q.iy0 >= 1) ? row_sum<S>(x, q.p0 - nx, j) : 0.0;
  const double r_0 = row_sum<S>(x, q.p0, j);
  const double r_1 = q.two ? row_sum<S>(x, q.p0 + nx, j) : 0.0;
  const double r_2 = (q.iy0 + 2 < nx) ? row_sum<S>(x, q.p0 + 2 * nx, j) : 0.0;
  m0 = fma(4.0, r_0, r_m) + r_1;
  m1 = fma(4.0, r_1, r_0) + r_2;
}

inline dim3 pair_grid(int nx) { return dim3((nx + BX - 1) / BX, ((nx + 1) / 2 + BY - 1) / BY); }

// y_i = M x_i + sum_j mix_ij K x_j (mix = dt A or dt A^T) on interior nodes, 0 on the boundary.
// One load of the S interleaved values per stencil point serves every stage; the
// S x S mixing stays in registers.
template <int S>
__global__ void __launch_bounds__(BX* BY) stage_apply_kernel(int nx, const double* __restrict__ cf, double hm, Mat4 mix,
                                                             const double* __restrict__ x, double* __restrict__ y) {
  IRK_PDL_ENTRY;
  const NodePair q(nx);
  if (q.ix >= nx || q.iy0 >= nx) return;
  const bool in[2] = {q.in0, q.in1};
  double mx[2][S];
  if (q.in0 || q.in1) {
#pragma unroll
    for (int j = 0; j < S; ++j) mass_pair<S>(x, q, nx, j, mx[0][j], mx[1][j]);
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    if (r == 1 && !q.two) break;
    const int p = q.p0 + r * nx;
    if (!in[r]) {
#pragma unroll
      for (int i = 0; i < S; ++i) y[(size_t)p * S + i] = 0.0;
      continue;
    }
    double kx[S];
#pragma unroll
    for (int j = 0; j < S; ++j) kx[j] = k_apply<S, double>(cf, x, p, nx, j);
#pragma unroll
    for (int i = 0; i < S; ++i) {
      double acc = hm * mx[r][i];
#pragma unroll
      for (int j = 0; j < S; ++j) acc += mix.v[i * S + j] * kx[j];
      y[(size_t)p * S + i] = acc;
    }
  }
}

// IA form (Sec. 3, eq. block_struct_IA): y_i = sum_j mixM_ij M x_j + dt K x_i (mixM = A^{-1} or A^{-T}),
// with the diagonal term folded into one stencil per stage, C_i = mixM_ii M + dt K (crec: S blocks of the
// five planar record planes, built on the host): y_i = C_i x_i + sum_{j != i} mixM_ij M x_j.  11 FP64
// operations per node and stage instead of 13 (the kernel is FP64-pipe-bound); M x_j from the separable
// mass stencil over node pairs as above.  offMh = mixM h^2/36 with a zero diagonal.
template <int S>
__global__ void __launch_bounds__(BX* BY) stage_apply_ia_kernel(int nx, const double* __restrict__ crec, Mat4 offMh,
                                                                const double* __restrict__ x,
                                                                double* __restrict__ y) {
  IRK_PDL_ENTRY;
  const NodePair q(nx);
  if (q.ix >= nx || q.iy0 >= nx) return;
  const bool in[2] = {q.in0, q.in1};
  const size_t rstride = (size_t)kCoef2 * nx * nx;
  double mx[2][S];
  if constexpr (S > 1) {
    if (q.in0 || q.in1) {
#pragma unroll
      for (int j = 0; j < S; ++j) mass_pair<S>(x, q, nx, j, mx[0][j], mx[1][j]);
    }
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    if (r == 1 && !q.two) break;
    const int p = q.p0 + r * nx;
    if (!in[r]) {
#pragma unroll
      for (int i = 0; i < S; ++i) y[(size_t)p * S + i] = 0.0;
      continue;
    }
#pragma unroll
    for (int i = 0; i < S; ++i) {
      double acc = k_apply<S, double>(crec + (size_t)i * rstride, x, p, nx, i);
#pragma unroll
      for (int j = 0; j < S; ++j)
        if (j != i) acc += offMh.v[i * S + j] * mx[r][j];
      y[(size_t)p * S + i] = acc;
    }
  }
}

// out_i = sum_j mix_ij in_j for every node of a stage vector (the IA back-transform k = (A^{-1} (x) I) w).
template <int S>
__global__ void stage_mix_kernel(size_t nodes, Mat4 mix, const double* __restrict__ in, double* __restrict__ out) {
  IRK_PDL_ENTRY;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nodes; q += (size_t)gridDim.x * blockDim.x) {
    double v[S];
#pragma unroll
    for (int j = 0; j < S; ++j) v[j] = in[q * S + j];
#pragma unroll
    for (int i = 0; i < S; ++i) {
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < S; ++j) acc += mix.v[i * S + j] * v[j];
      out[q * S + i] = acc;
    }
  }
}

// z_i *= scale_i for every node of a stage vector.
template <int S>
__global__ void stage_scale_kernel(size_t nodes, Vec8 scale, double* __restrict__ z) {
  IRK_PDL_ENTRY;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nodes; q += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int i = 0; i < S; ++i) z[q * S + i] *= scale.v[i];
  }
}

// r_i = fcoef_i F^ + F_i - K u_n (Sec. 2 eq. rkheat moved to the right-hand side).
// raw_u != 0: u's boundary entries are Dirichlet data and enter K u_n (DAE-type conditions).
template <int S>
__global__ void __launch_bounds__(BX* BY) rhs_kernel(int nx, const double* __restrict__ cf, const double* __restrict__ u,
                                                     const double* __restrict__ fsp, Vec8 fcoef,
                                                     const double* __restrict__ fst, double* __restrict__ r,
                                                     int raw_u) {
  IRK_PDL_ENTRY;
  const int ix = blockIdx.x * BX + threadIdx.x;
  const int iy = blockIdx.y * BY + threadIdx.y;
  if (ix >= nx || iy >= nx) return;
  const int p = ix + nx * iy;
  if (!interior2(ix, iy, nx)) {
#pragma unroll
    for (int i = 0; i < S; ++i) r[(size_t)p * S + i] = 0.0;
    return;
  }
  const double ku = (u == nullptr) ? 0.0 : (raw_u ? k_apply<1, double>(cf, u, p, nx, 0) : k_apply_masked(cf, u, ix, iy, nx));
  const double f = (fsp != nullptr) ? fsp[p] : 0.0;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    double v = fcoef.v[i] * f - ku;
    if (fst != nullptr) v += fst[(size_t)p * S + i];
    r[(size_t)p * S + i] = v;
  }
}

// u_{n+1} = u_n + sum_i (dt b_i) k_i on interior nodes, 0 on the boundary (all_nodes: everywhere).
template <int S>
__global__ void rk_update_kernel(int nx, const double* __restrict__ u, const double* __restrict__ k, Vec8 bdt,
                                 double* __restrict__ out, int all_nodes) {
  IRK_PDL_ENTRY;
  const int ix = blockIdx.x * BX + threadIdx.x;
  const int iy = blockIdx.y * BY + threadIdx.y;
  if (ix >= nx || iy >= nx) return;
  const int p = ix + nx * iy;
  double v = 0.0;
  if (all_nodes || interior2(ix, iy, nx)) {
    v = u[p];
#pragma unroll
    for (int i = 0; i < S; ++i) v += bdt.v[i] * k[(size_t)p * S + i];
  }
  out[p] = v;
}

// Boundary stage values of DAE-type Dirichlet conditions (Sec. 2.1): on the boundary
// sum_j a_ij k_j = (g_i - u_n) / dt, so k = Ainv_dt (g - u_n) with Ainv_dt = A^{-1} / dt; 0 inside.
template <int S>
__global__ void bc_stages_kernel(int nx, Mat4 ainv_dt, const double* __restrict__ u, const double* __restrict__ g,
                                 double* __restrict__ kb) {
  IRK_PDL_ENTRY;
  const int ix = blockIdx.x * BX + threadIdx.x;
  const int iy = blockIdx.y * BY + threadIdx.y;
  if (ix >= nx || iy >= nx) return;
  const int p = ix + nx * iy;
  const bool bnd = !interior2(ix, iy, nx);
  double d[S];
#pragma unroll
  for (int j = 0; j < S; ++j) d[j] = bnd ? g[(size_t)p * S + j] - u[p] : 0.0;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < S; ++j) acc += ainv_dt.v[i * S + j] * d[j];
    kb[(size_t)p * S + i] = acc;
  }
}

// lam_n = lam_{n+1} - K sum_i mu_i (interior), 0 on the boundary.
template <int S>
__global__ void adjoint_lambda_kernel(int nx, const double* __restrict__ cf, const double* __restrict__ lam1,
                                      const double* __restrict__ mu, double* __restrict__ lam0) {
  IRK_PDL_ENTRY;
  const int ix = blockIdx.x * BX + threadIdx.x;
  const int iy = blockIdx.y * BY + threadIdx.y;
  if (ix >= nx || iy >= nx) return;
  const int p = ix + nx * iy;
  double v = 0.0;
  if (interior2(ix, iy, nx)) {
    double kmu = 0.0;
#pragma unroll
    for (int i = 0; i < S; ++i) kmu += k_apply<S, double>(cf, mu, p, nx, i);
    v = lam1[p] - kmu;
  }
  lam0[p] = v;
}

// y = (M + sigma K) x for one internal single-stage vector (boundary entries zero).
__global__ void block_apply_kernel(int nx, const double* __restrict__ cf, double hm, double sigma,
                                   const double* __restrict__ x, double* __restrict__ y) {
  IRK_PDL_ENTRY;
  const int ix = 1 + blockIdx.x * BX + threadIdx.x;
  const int iy = 1 + blockIdx.y * BY + threadIdx.y;
  if (ix > nx - 2 || iy > nx - 2) return;
  const int p = ix + nx * iy;
  y[p] = hm * m_apply_unscaled<1, double>(x, p, nx, 0) + sigma * k_apply<1, double>(cf, x, p, nx, 0);
}

// y = M x for a caller-supplied nodal vector (boundary entries of x read as 0).
__global__ void mass_apply_kernel(int nx, double hm, const double* __restrict__ x, double* __restrict__ y) {
  IRK_PDL_ENTRY;
  const int ix = blockIdx.x * BX + threadIdx.x;
  const int iy = blockIdx.y * BY + threadIdx.y;
  if (ix >= nx || iy >= nx) return;
  double v = 0.0;
  if (interior2(ix, iy, nx)) {
    auto X = [&](int dx, int dy) {
      const int jx = ix + dx, jy = iy + dy;
      return interior2(jx, jy, nx) ? x[jx + nx * jy] : 0.0;
    };
    const double edge = X(-1, 0) + X(1, 0) + X(0, -1) + X(0, 1);
    const double corner = X(-1, -1) + X(1, -1) + X(-1, 1) + X(1, 1);
    v = hm * (16.0 * X(0, 0) + 4.0 * edge + corner);
  }
  y[ix + nx * iy] = v;
}

// grad[c] += -kappa_c sum_i mu_i|_c^T K_e U_i|_c, U_i = u_n + sum_j (dt a_ij) k_j, with the
// unit-diffusivity bilinear element matrix K_e = [[4,-1,-1,-2],[-1,4,-2,-1],[-1,-2,4,-1],[-2,-1,-1,4]]/6
// (corners ordered (0,0), (1,0), (0,1), (1,1)).  One thread per cell, no atomics.
template <int S>
__global__ void cell_gradient_kernel(int N, const double* __restrict__ kappa, const double* __restrict__ u,
                                     const double* __restrict__ k, Mat4 dtA, const double* __restrict__ mu,
                                     double* __restrict__ grad) {
  IRK_PDL_ENTRY;
  const int cx = blockIdx.x * BX + threadIdx.x;
  const int cy = blockIdx.y * BY + threadIdx.y;
  if (cx >= N || cy >= N) return;
  const int nx = N + 1;
  int q[4], qx[4], qy[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    qx[a] = cx + (a & 1);
    qy[a] = cy + (a >> 1);
    q[a] = qx[a] + nx * qy[a];
  }
  double total = 0.0;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    double U[4], m[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const bool in = interior2(qx[a], qy[a], nx);
      double v = in ? u[q[a]] : 0.0;
#pragma unroll
      for (int j = 0; j < S; ++j) v += dtA.v[i * S + j] * k[(size_t)q[a] * S + j];
      U[a] = in ? v : 0.0;
      m[a] = in ? mu[(size_t)q[a] * S + i] : 0.0;
    }
    const double KU0 = 4 * U[0] - U[1] - U[2] - 2 * U[3];
    const double KU1 = -U[0] + 4 * U[1] - 2 * U[2] - U[3];
    const double KU2 = -U[0] - 2 * U[1] + 4 * U[2] - U[3];
    const double KU3 = -2 * U[0] - U[1] - U[2] + 4 * U[3];
    total += m[0] * KU0 + m[1] * KU1 + m[2] * KU2 + m[3] * KU3;
  }
  const int c = cx + N * cy;
  const double kap = (kappa != nullptr) ? kappa[c] : 1.0;
  grad[c] += -kap * total / 6.0;
}

#define IRK_DISPATCH_S(S, ...)                                \
  switch (S) {                                                \
    case 1: { constexpr int SS = 1; __VA_ARGS__; } break;     \
    case 2: { constexpr int SS = 2; __VA_ARGS__; } break;     \
    case 3: { constexpr int SS = 3; __VA_ARGS__; } break;     \
    case 4: { constexpr int SS = 4; __VA_ARGS__; } break;     \
    default: break;                                           \
  }

void launch_stage_apply(int S, cudaStream_t st, int nx, const double* cf, double hm, const Mat4& mix, const double* x,
                        double* y) {
  IRK_DISPATCH_S(S, launch_k(stage_apply_kernel<SS>, pair_grid(nx), dim3(BX, BY), 0, st, nx, cf, hm, mix, x, y));
}
void launch_stage_apply_ia(int S, cudaStream_t st, int nx, const double* crec, double hm, const Mat4& mixM,
                           const double* x, double* y) {
  Mat4 offMh = mixM;
  for (int i = 0; i < S; ++i)
    for (int j = 0; j < S; ++j) offMh.v[i * S + j] = (i == j) ? 0.0 : offMh.v[i * S + j] * hm;
  IRK_DISPATCH_S(S, launch_k(stage_apply_ia_kernel<SS>, pair_grid(nx), dim3(BX, BY), 0, st, nx, crec, offMh, x, y));
}
void launch_stage_mix(int S, cudaStream_t st, size_t nodes, const Mat4& mix, const double* in, double* out) {
  int blocks = (int)std::min<size_t>((nodes + 255) / 256, 152 * 8);
  IRK_DISPATCH_S(S, launch_k(stage_mix_kernel<SS>, blocks, 256, 0, st, nodes, mix, in, out));
}
void launch_stage_scale(int S, cudaStream_t st, size_t nodes, const Vec8& scale, double* z) {
  int blocks = (int)std::min<size_t>((nodes + 255) / 256, 152 * 8);
  IRK_DISPATCH_S(S, launch_k(stage_scale_kernel<SS>, blocks, 256, 0, st, nodes, scale, z));
}
void launch_rhs(int S, cudaStream_t st, int nx, const double* cf, const double* u, const double* fsp,
                const Vec8& fcoef, const double* fst, double* r, int raw_u) {
  IRK_DISPATCH_S(S, launch_k(rhs_kernel<SS>, all_nodes_grid(nx), dim3(BX, BY), 0, st, nx, cf, u, fsp, fcoef, fst, r, raw_u));
}
void launch_rk_update(int S, cudaStream_t st, int nx, const double* u, const double* k, const Vec8& bdt,
                      double* out, int all_nodes) {
  IRK_DISPATCH_S(S, launch_k(rk_update_kernel<SS>, all_nodes_grid(nx), dim3(BX, BY), 0, st, nx, u, k, bdt, out, all_nodes));
}
void launch_bc_stages(int S, cudaStream_t st, int nx, const Mat4& ainv_dt, const double* u, const double* g,
                      double* kb) {
  IRK_DISPATCH_S(S, launch_k(bc_stages_kernel<SS>, all_nodes_grid(nx), dim3(BX, BY), 0, st, nx, ainv_dt, u, g, kb));
}
void launch_adjoint_lambda(int S, cudaStream_t st, int nx, const double* cf, const double* lam_np1, const double* mu,
                           double* lam_n) {
  IRK_DISPATCH_S(S, launch_k(adjoint_lambda_kernel<SS>, all_nodes_grid(nx), dim3(BX, BY), 0, st, nx, cf, lam_np1, mu, lam_n));
}
void launch_block_apply(cudaStream_t st, int nx, const double* cf, double hm, double sigma, const double* x,
                        double* y) {
  dim3 g((nx - 2 + BX - 1) / BX, (nx - 2 + BY - 1) / BY);
  launch_k(block_apply_kernel, g, dim3(BX, BY), 0, st, nx, cf, hm, sigma, x, y);
}
void launch_mass_apply(cudaStream_t st, int nx, double hm, const double* x, double* y) {
  launch_k(mass_apply_kernel, all_nodes_grid(nx), dim3(BX, BY), 0, st, nx, hm, x, y);
}
void launch_cell_gradient(int S, cudaStream_t st, int N, const double* kappa, const double* u, const double* k,
                          const Mat4& dtA, const double* mu, double* grad) {
  dim3 g((N + BX - 1) / BX, (N + BY - 1) / BY);
  IRK_DISPATCH_S(S, launch_k(cell_gradient_kernel<SS>, g, dim3(BX, BY), 0, st, N, kappa, u, k, dtA, mu, grad));
}

}  // namespace irk
