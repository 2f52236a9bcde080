// FP64 kernels of the outer iteration on 3D Q1 hexahedral grids with kappa = 1:
// the stage operator of Sec. 3, eq. block_struct_AI, the right-hand side of
// Sec. 2 eq. rkheat and the RK update (Sec. 2).  Mass and stiffness are the
// constant 27-point Q1 stencils given by their four offset-class values
// (mk.v[0] = mass classes, mk.v[1] = stiffness classes).
#include "common.cuh"
#include "kernels.h"
#include "mg3d.cuh"

namespace irk {

namespace {
constexpr int AX = 32, AY = 4, AZ = 2;

inline dim3 all_nodes_grid3(int n) { return dim3((n + AX - 1) / AX, (n + AY - 1) / AY, (n + AZ - 1) / AZ); }

#define IRK_3D_ALL_INDEX                              \
  const int ix = blockIdx.x * AX + threadIdx.x;       \
  const int iy = blockIdx.y * AY + threadIdx.y;       \
  const int iz = blockIdx.z * AZ + threadIdx.z;       \
  if (ix >= n || iy >= n || iz >= n) return;          \
  const int p = ix + n * (iy + n * iz);

// Class sums of a caller-supplied nodal vector whose boundary entries must be read as 0.
__device__ __forceinline__ void class_sums3_masked(const double* __restrict__ u, int ix, int iy, int iz, int n,
                                                   double out[4]) {
  out[0] = out[1] = out[2] = out[3] = 0.0;
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int jx = ix + dx, jy = iy + dy, jz = iz + dz;
        const double v = interior3(jx, jy, jz, n) ? u[jx + n * (jy + n * jz)] : 0.0;
        out[(dx != 0) + (dy != 0) + (dz != 0)] += v;
      }
}
}  // namespace

template <int S>
__global__ void __launch_bounds__(AX* AY* AZ) stage_apply3_kernel(int n, Cls4 mk, Mat4 mix,
                                                                  const double* __restrict__ x, double* __restrict__ y) {
  IRK_PDL_ENTRY;
  IRK_3D_ALL_INDEX
  if (!interior3(ix, iy, iz, n)) {
#pragma unroll
    for (int i = 0; i < S; ++i) y[(size_t)p * S + i] = 0.0;
    return;
  }
  double kx[S], mx[S];
#pragma unroll
  for (int j = 0; j < S; ++j) {
    double cs[4];
    class_sums3<S, double>(x, p, n, j, cs);
    mx[j] = class_apply<double>(mk.v[0], cs);
    kx[j] = class_apply<double>(mk.v[1], cs);
  }
#pragma unroll
  for (int i = 0; i < S; ++i) {
    double acc = mx[i];
#pragma unroll
    for (int j = 0; j < S; ++j) acc += mix.v[i * S + j] * kx[j];
    y[(size_t)p * S + i] = acc;
  }
}

template <int S>
__global__ void __launch_bounds__(AX* AY* AZ) stage_apply3_ia_kernel(int n, Cls4 mk, Mat4 mixM, double dt,
                                                                     const double* __restrict__ x,
                                                                     double* __restrict__ y) {
  IRK_PDL_ENTRY;
  IRK_3D_ALL_INDEX
  if (!interior3(ix, iy, iz, n)) {
#pragma unroll
    for (int i = 0; i < S; ++i) y[(size_t)p * S + i] = 0.0;
    return;
  }
  double kx[S], mx[S];
#pragma unroll
  for (int j = 0; j < S; ++j) {
    double cs[4];
    class_sums3<S, double>(x, p, n, j, cs);
    mx[j] = class_apply<double>(mk.v[0], cs);
    kx[j] = class_apply<double>(mk.v[1], cs);
  }
#pragma unroll
  for (int i = 0; i < S; ++i) {
    double acc = dt * kx[i];
#pragma unroll
    for (int j = 0; j < S; ++j) acc += mixM.v[i * S + j] * mx[j];
    y[(size_t)p * S + i] = acc;
  }
}

template <int S>
__global__ void __launch_bounds__(AX* AY* AZ) rhs3_kernel(int n, Cls4 mk, const double* __restrict__ u,
                                                          const double* __restrict__ fsp, Vec8 fcoef,
                                                          const double* __restrict__ fst, double* __restrict__ r,
                                                          int raw_u) {
  IRK_PDL_ENTRY;
  IRK_3D_ALL_INDEX
  if (!interior3(ix, iy, iz, n)) {
#pragma unroll
    for (int i = 0; i < S; ++i) r[(size_t)p * S + i] = 0.0;
    return;
  }
  double ku = 0.0;
  if (u != nullptr) {
    double cs[4];
    if (raw_u)
      class_sums3<1, double>(u, p, n, 0, cs);
    else
      class_sums3_masked(u, ix, iy, iz, n, cs);
    ku = class_apply<double>(mk.v[1], cs);
  }
  const double f = (fsp != nullptr) ? fsp[p] : 0.0;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    double v = fcoef.v[i] * f - ku;
    if (fst != nullptr) v += fst[(size_t)p * S + i];
    r[(size_t)p * S + i] = v;
  }
}

// y = (M + sigma K) x for one internal single-stage vector (boundary entries zero).
__global__ void __launch_bounds__(AX* AY* AZ) block_apply3_kernel(int n, Cls4 mk, double sigma,
                                                                  const double* __restrict__ x, double* __restrict__ y) {
  IRK_PDL_ENTRY;
  const int ix = 1 + blockIdx.x * AX + threadIdx.x;
  const int iy = 1 + blockIdx.y * AY + threadIdx.y;
  const int iz = 1 + blockIdx.z * AZ + threadIdx.z;
  if (ix > n - 2 || iy > n - 2 || iz > n - 2) return;
  const int p = ix + n * (iy + n * iz);
  double cs[4];
  class_sums3<1, double>(x, p, n, 0, cs);
  y[p] = class_apply<double>(mk.v[0], cs) + sigma * class_apply<double>(mk.v[1], cs);
}

template <int S>
__global__ void rk_update3_kernel(int n, const double* __restrict__ u, const double* __restrict__ k, Vec8 bdt,
                                  double* __restrict__ out, int all_nodes) {
  IRK_PDL_ENTRY;
  IRK_3D_ALL_INDEX
  double v = 0.0;
  if (all_nodes || interior3(ix, iy, iz, n)) {
    v = u[p];
#pragma unroll
    for (int i = 0; i < S; ++i) v += bdt.v[i] * k[(size_t)p * S + i];
  }
  out[p] = v;
}

template <int S>
__global__ void bc_stages3_kernel(int n, Mat4 ainv_dt, const double* __restrict__ u, const double* __restrict__ g,
                                  double* __restrict__ kb) {
  IRK_PDL_ENTRY;
  IRK_3D_ALL_INDEX
  const bool bnd = !interior3(ix, iy, iz, n);
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

#define IRK_DISPATCH_S(S, ...)                                \
  switch (S) {                                                \
    case 1: { constexpr int SS = 1; __VA_ARGS__; } break;     \
    case 2: { constexpr int SS = 2; __VA_ARGS__; } break;     \
    case 3: { constexpr int SS = 3; __VA_ARGS__; } break;     \
    case 4: { constexpr int SS = 4; __VA_ARGS__; } break;     \
    default: break;                                           \
  }

void launch_stage_apply3(int S, cudaStream_t st, int n, const Cls4& mk, const Mat4& mix, const double* x, double* y) {
  IRK_DISPATCH_S(S, launch_k(stage_apply3_kernel<SS>, all_nodes_grid3(n), dim3(AX, AY, AZ), 0, st, n, mk, mix, x, y));
}
void launch_stage_apply3_ia(int S, cudaStream_t st, int n, const Cls4& mk, const Mat4& mixM, double dt,
                            const double* x, double* y) {
  IRK_DISPATCH_S(S, launch_k(stage_apply3_ia_kernel<SS>, all_nodes_grid3(n), dim3(AX, AY, AZ), 0, st, n, mk, mixM, dt, x, y));
}
void launch_rhs3(int S, cudaStream_t st, int n, const Cls4& mk, const double* u, const double* fsp,
                 const Vec8& fcoef, const double* fst, double* r, int raw_u) {
  IRK_DISPATCH_S(S, launch_k(rhs3_kernel<SS>, all_nodes_grid3(n), dim3(AX, AY, AZ), 0, st, n, mk, u, fsp, fcoef, fst, r,
                             raw_u));
}
void launch_block_apply3(cudaStream_t st, int n, const Cls4& mk, double sigma, const double* x, double* y) {
  const int m = n - 2;
  dim3 g((m + AX - 1) / AX, (m + AY - 1) / AY, (m + AZ - 1) / AZ);
  launch_k(block_apply3_kernel, g, dim3(AX, AY, AZ), 0, st, n, mk, sigma, x, y);
}
void launch_rk_update3(int S, cudaStream_t st, int n, const double* u, const double* k, const Vec8& bdt, double* out,
                       int all_nodes) {
  IRK_DISPATCH_S(S, launch_k(rk_update3_kernel<SS>, all_nodes_grid3(n), dim3(AX, AY, AZ), 0, st, n, u, k, bdt, out,
                             all_nodes));
}
void launch_bc_stages3(int S, cudaStream_t st, int n, const Mat4& ainv_dt, const double* u, const double* g,
                       double* kb) {
  IRK_DISPATCH_S(S, launch_k(bc_stages3_kernel<SS>, all_nodes_grid3(n), dim3(AX, AY, AZ), 0, st, n, ainv_dt, u, g, kb));
}

}  // namespace irk
