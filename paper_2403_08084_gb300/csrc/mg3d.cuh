// 3D (Q1 hexahedra, kappa = 1) versions of the multigrid and stage kernels.
//
// With a constant coefficient the Q1 mass and stiffness matrices of every level
// are 27-point stencils whose value depends only on how many coordinates of
// the offset are nonzero: class 0 (centre), 1 (6 faces), 2 (12 edges), 3 (8
// corners).  The Galerkin coarse operators of nested uniform grids are the
// same stencils rediscretised with the coarse h, so a level is described by
// four mass and four stiffness class values; B_i = M + sigma_i K by four more.
// Grid: n = N + 1 nodes per axis, node p = ix + n (iy + n iz), interior nodes
// 1 <= ix, iy, iz <= n - 2; stage vectors node-major as in 2D.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace irk {

constexpr int k3X = 32, k3Y = 4, k3Z = 2;

inline dim3 interior_grid3(int n) {
  const int m = n - 2;
  return dim3((m + k3X - 1) / k3X, (m + k3Y - 1) / k3Y, (m + k3Z - 1) / k3Z);
}

__device__ __forceinline__ bool interior3(int ix, int iy, int iz, int n) {
  return ix >= 1 && iy >= 1 && iz >= 1 && ix <= n - 2 && iy <= n - 2 && iz <= n - 2;
}

// Class sums of stage i around p: out[0] centre, out[1] faces, out[2] edges, out[3] corners.
template <int S, typename C, typename T>
__device__ __forceinline__ void class_sums3(const T* __restrict__ x, int p, int n, int i, C out[4]) {
  const int sx = 1, sy = n, sz = n * n;
  auto X = [&](int q) { return ld<C>(x + (size_t)q * S + i); };
  out[0] = X(p);
  out[1] = (X(p - sx) + X(p + sx)) + (X(p - sy) + X(p + sy)) + (X(p - sz) + X(p + sz));
  C e = 0, c = 0;
#pragma unroll
  for (int dz = -1; dz <= 1; dz += 2) {
#pragma unroll
    for (int dy = -1; dy <= 1; dy += 2) {
      e += X(p + dz * sz + dy * sy);  // yz edges
#pragma unroll
      for (int dx = -1; dx <= 1; dx += 2) c += X(p + dz * sz + dy * sy + dx * sx);
    }
#pragma unroll
    for (int dx = -1; dx <= 1; dx += 2) e += X(p + dz * sz + dx * sx);  // xz edges
  }
#pragma unroll
  for (int dy = -1; dy <= 1; dy += 2)
#pragma unroll
    for (int dx = -1; dx <= 1; dx += 2) e += X(p + dy * sy + dx * sx);  // xy edges
  out[2] = e;
  out[3] = c;
}

template <typename C, typename W>
__device__ __forceinline__ C class_apply(const W* w, const C s[4]) {
  return C(w[0]) * s[0] + C(w[1]) * s[1] + C(w[2]) * s[2] + C(w[3]) * s[3];
}

template <typename C>
inline ClsT<C> to_cls(const Cls4& a) {
  ClsT<C> r;
  for (int i = 0; i < kMaxS; ++i)
    for (int k = 0; k < 4; ++k) r.v[i][k] = static_cast<C>(a.v[i][k]);
  return r;
}

#define IRK_3D_INDEX                                          \
  const int ix = 1 + blockIdx.x * k3X + threadIdx.x;          \
  const int iy = 1 + blockIdx.y * k3Y + threadIdx.y;          \
  const int iz = 1 + blockIdx.z * k3Z + threadIdx.z;          \
  if (ix > n - 2 || iy > n - 2 || iz > n - 2) return;         \
  const int p = ix + n * (iy + n * iz);

// Weighted Jacobi x_out = x_in + d_i (b - B_i x_in); d_i = omega / B_i(centre) (constant per level).
template <typename T, typename C, int S>
__global__ void __launch_bounds__(k3X* k3Y* k3Z) jacobi3_kernel(int n, ClsT<C> bc, VecT<C> dinv, const T* __restrict__ xin,
                                                                const T* __restrict__ b, T* __restrict__ xout) {
  IRK_PDL_ENTRY;
  IRK_3D_INDEX
#pragma unroll
  for (int i = 0; i < S; ++i) {
    const C bi = ld<C>(b + (size_t)p * S + i);
    C xn;
    if (xin == nullptr) {
      xn = dinv.v[i] * bi;
    } else {
      C cs[4];
      class_sums3<S, C>(xin, p, n, i, cs);
      xn = cs[0] + dinv.v[i] * (bi - class_apply<C>(bc.v[i], cs));
    }
    st(xout + (size_t)p * S + i, xn);
  }
}

// Two Jacobi sweeps from zero in one pass: with the constant diagonal d of a level,
// x1 = d b and B x1 = d B b, so x2 = d b + d (b - d B b).
template <typename T, typename C, int S>
__global__ void __launch_bounds__(k3X* k3Y* k3Z) jacobi2z3_kernel(int n, ClsT<C> bc, VecT<C> dinv,
                                                                  const T* __restrict__ b, T* __restrict__ xout) {
  IRK_PDL_ENTRY;
  IRK_3D_INDEX
#pragma unroll
  for (int i = 0; i < S; ++i) {
    C cs[4];
    class_sums3<S, C>(b, p, n, i, cs);
    const C d = dinv.v[i];
    st(xout + (size_t)p * S + i, d * cs[0] + d * (cs[0] - d * class_apply<C>(bc.v[i], cs)));
  }
}

template <typename T, typename C, int S>
__global__ void __launch_bounds__(k3X* k3Y* k3Z) residual3_kernel(int n, ClsT<C> bc, const T* __restrict__ x,
                                                                  const T* __restrict__ b, T* __restrict__ r) {
  IRK_PDL_ENTRY;
  IRK_3D_INDEX
#pragma unroll
  for (int i = 0; i < S; ++i) {
    C cs[4];
    class_sums3<S, C>(x, p, n, i, cs);
    st(r + (size_t)p * S + i, ld<C>(b + (size_t)p * S + i) - class_apply<C>(bc.v[i], cs));
  }
}

// b_c = P^T r_f: weights prod_d w(o_d), w(0) = 1, w(+-1) = 1/2 over the 27 fine neighbours.
template <typename T, typename C, int S>
__global__ void __launch_bounds__(k3X* k3Y* k3Z) restrict3_kernel(int nf, const T* __restrict__ rf, int n,
                                                                  T* __restrict__ bc) {
  IRK_PDL_ENTRY;
  IRK_3D_INDEX
  const int q = 2 * ix + nf * (2 * iy + nf * 2 * iz);
  C cs[4];
#pragma unroll
  for (int i = 0; i < S; ++i) {
    class_sums3<S, C>(rf, q, nf, i, cs);
    st(bc + (size_t)p * S + i, cs[0] + C(0.5) * cs[1] + C(0.25) * cs[2] + C(0.125) * cs[3]);
  }
}

// x_f += P e_c (trilinear): the mean of the eight (I0|I1, J0|J1, K0|K1) corner values.
template <typename T, typename C, int S>
__global__ void __launch_bounds__(k3X* k3Y* k3Z) prolong_add3_kernel(int nc, const T* __restrict__ ec, int n,
                                                                     T* __restrict__ xf) {
  IRK_PDL_ENTRY;
  IRK_3D_INDEX
  const int I[2] = {ix >> 1, (ix + 1) >> 1}, J[2] = {iy >> 1, (iy + 1) >> 1}, K[2] = {iz >> 1, (iz + 1) >> 1};
#pragma unroll
  for (int i = 0; i < S; ++i) {
    C v = 0;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int bb = 0; bb < 2; ++bb)
#pragma unroll
        for (int c = 0; c < 2; ++c) v += ld<C>(ec + (size_t)(I[c] + nc * (J[bb] + nc * K[a])) * S + i);
    st(xf + (size_t)p * S + i, ld<C>(xf + (size_t)p * S + i) + C(0.125) * v);
  }
}

// out = v_i - sum_j cj[j] K z_j (triangular preconditioners), K given by its class values kc.
// LOWZ / zt: as for the 2D block_rhs_kernel.
template <typename T, typename C, int SF, bool LOWZ>
__global__ void __launch_bounds__(k3X* k3Y* k3Z) block_rhs3_kernel(int n, ClsT<C> kc, const double* __restrict__ v,
                                                                   const double* __restrict__ z,
                                                                   const T* __restrict__ zt, size_t zstride, int i,
                                                                   VecT<C> cj, unsigned used, T* __restrict__ out) {
  IRK_PDL_ENTRY;
  IRK_3D_INDEX
  C acc = static_cast<C>(v[(size_t)p * SF + i]);
#pragma unroll
  for (int j = 0; j < SF; ++j) {
    if (used & (1u << j)) {
      C cs[4];
      if constexpr (LOWZ)
        class_sums3<1, C>(zt + (size_t)j * zstride, p, n, 0, cs);
      else
        class_sums3<SF, C>(z, p, n, j, cs);
      acc -= cj.v[j] * class_apply<C>(kc.v[0], cs);
    }
  }
  st(out + p, acc);
}

template <typename T, typename C, int SF>
__global__ void __launch_bounds__(k3X* k3Y* k3Z) scatter_stage3_kernel(int n, const T* __restrict__ x, int i,
                                                                       double* __restrict__ z, double scale,
                                                                       T* __restrict__ zt) {
  IRK_PDL_ENTRY;
  IRK_3D_INDEX
  const T xv = x[p];
  z[(size_t)p * SF + i] = scale * static_cast<double>(ld<C>(&xv));
  if (zt != nullptr) zt[p] = xv;
}

template <typename T, typename C>
__global__ void coarse_solve3_kernel(int nint, const C* __restrict__ binv, const int* __restrict__ map,
                                     const T* __restrict__ b, T* __restrict__ x, int S) {
  IRK_PDL_ENTRY;
  extern __shared__ unsigned char smem3_raw[];
  C* bs = reinterpret_cast<C*>(smem3_raw);
  const int i = blockIdx.y;
  for (int c = threadIdx.x; c < nint; c += blockDim.x) bs[c] = ld<C>(b + (size_t)map[c] * S + i);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const C* Bi = binv + (size_t)i * nint * nint;
  for (int r = blockIdx.x * nw + warp; r < nint; r += gridDim.x * nw) {
    C a0 = 0, a1 = 0, a2 = 0, a3 = 0;  // independent chains keep several loads in flight
    const C* row = Bi + (size_t)r * nint;
    int c = lane;
    for (; c + 96 < nint; c += 128) {
      a0 += row[c] * bs[c];
      a1 += row[c + 32] * bs[c + 32];
      a2 += row[c + 64] * bs[c + 64];
      a3 += row[c + 96] * bs[c + 96];
    }
    for (; c < nint; c += 32) a0 += row[c] * bs[c];
    C acc = (a0 + a1) + (a2 + a3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) st(x + (size_t)map[r] * S + i, acc);
  }
}

#define IRK_DISPATCH_S3(S, ...)                               \
  switch (S) {                                                \
    case 1: { constexpr int SS = 1; __VA_ARGS__; } break;     \
    case 2: { constexpr int SS = 2; __VA_ARGS__; } break;     \
    case 3: { constexpr int SS = 3; __VA_ARGS__; } break;     \
    case 4: { constexpr int SS = 4; __VA_ARGS__; } break;     \
    default: break;                                           \
  }

template <typename T, typename C>
void MG3<T, C>::jacobi(int S, cudaStream_t st, int n, const Cls4& bc, const Vec8& dinv, const T* xin, const T* b,
                       T* xout) {
  const ClsT<C> c = to_cls<C>(bc);
  const VecT<C> d = to_vec<C>(dinv);
  IRK_DISPATCH_S3(S, launch_k(jacobi3_kernel<T, C, SS>, interior_grid3(n), dim3(k3X, k3Y, k3Z), 0, st, n, c, d, xin, b, xout));
}
template <typename T, typename C>
void MG3<T, C>::jacobi2z(int S, cudaStream_t st, int n, const Cls4& bc, const Vec8& dinv, const T* b, T* xout) {
  const ClsT<C> c = to_cls<C>(bc);
  const VecT<C> d = to_vec<C>(dinv);
  IRK_DISPATCH_S3(S, launch_k(jacobi2z3_kernel<T, C, SS>, interior_grid3(n), dim3(k3X, k3Y, k3Z), 0, st, n, c, d, b, xout));
}
template <typename T, typename C>
void MG3<T, C>::residual(int S, cudaStream_t st, int n, const Cls4& bc, const T* x, const T* b, T* r) {
  const ClsT<C> c = to_cls<C>(bc);
  IRK_DISPATCH_S3(S, launch_k(residual3_kernel<T, C, SS>, interior_grid3(n), dim3(k3X, k3Y, k3Z), 0, st, n, c, x, b, r));
}
template <typename T, typename C>
void MG3<T, C>::restrict_(int S, cudaStream_t st, int nf, const T* rf, int nc, T* bc) {
  IRK_DISPATCH_S3(S, launch_k(restrict3_kernel<T, C, SS>, interior_grid3(nc), dim3(k3X, k3Y, k3Z), 0, st, nf, rf, nc, bc));
}
template <typename T, typename C>
void MG3<T, C>::prolong_add(int S, cudaStream_t st, int nc, const T* ec, int nf, T* xf) {
  IRK_DISPATCH_S3(S, launch_k(prolong_add3_kernel<T, C, SS>, interior_grid3(nf), dim3(k3X, k3Y, k3Z), 0, st, nc, ec, nf, xf));
}
template <typename T, typename C>
void MG3<T, C>::block_rhs(int SF, cudaStream_t st, int n, const Cls4& kc, const double* v, const double* z, int i,
                          const Vec8& cj, T* out, const T* zt, size_t zstride) {
  unsigned used = 0;
  for (int j = 0; j < SF; ++j)
    if (cj.v[j] != 0.0) used |= 1u << j;
  const ClsT<C> c = to_cls<C>(kc);
  const VecT<C> w = to_vec<C>(cj);
  if (zt != nullptr) {
    IRK_DISPATCH_S3(SF, launch_k(block_rhs3_kernel<T, C, SS, true>, interior_grid3(n), dim3(k3X, k3Y, k3Z), 0, st, n, c,
                                 v, z, zt, zstride, i, w, used, out));
  } else {
    IRK_DISPATCH_S3(SF, launch_k(block_rhs3_kernel<T, C, SS, false>, interior_grid3(n), dim3(k3X, k3Y, k3Z), 0, st, n, c,
                                 v, z, zt, zstride, i, w, used, out));
  }
}
template <typename T, typename C>
void MG3<T, C>::scatter_stage(int SF, cudaStream_t st, int n, const T* x, int i, double* z, double scale, T* zt) {
  IRK_DISPATCH_S3(SF, launch_k(scatter_stage3_kernel<T, C, SS>, interior_grid3(n), dim3(k3X, k3Y, k3Z), 0, st, n, x, i, z,
                               scale, zt));
}
template <typename T, typename C>
void MG3<T, C>::coarse_solve(int S, cudaStream_t st, int nint, const C* binv, const int* map, const T* b, T* x) {
  const int threads = 256, rows_per_block = threads / 32;
  int gx = (nint + rows_per_block - 1) / rows_per_block;
  if (gx > 152 * 4) gx = 152 * 4;
  launch_k(coarse_solve3_kernel<T, C>, dim3(gx, S), threads, sizeof(C) * (size_t)nint, st, nint, binv, map, b, x, S);
}

}  // namespace irk
