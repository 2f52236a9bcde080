// Finest-level 2D kernels of the FP32 / BF16 V-cycles that form the stiffness
// stencil from the per-cell diffusivity on the fly.  Around interior node
// (ix, iy) the cells SW, SE, NW, NE carry kappa; the bilinear element matrix
// kappa/6 [[4,-1,-1,-2],[-1,4,-2,-1],[-1,-2,4,-1],[-2,-1,-1,4]] assembles to
//   6 (K x)_p = 4 (sum kappa) x_p - (k_SE + k_NE) x_E - (k_SW + k_NW) x_W - (k_NW + k_NE) x_N
//               - (k_SW + k_SE) x_S - 2 (k_NE x_NE + k_NW x_NW + k_SW x_SW + k_SE x_SE),
// and the Jacobi diagonal omega / (16 hm + sigma (4/6) sum kappa) follows from the same
// four values.  A sweep then reads 4 bytes of coefficients per node (one kappa per
// cell, shared by four nodes) instead of a 20-byte stencil record and a diagonal.
#pragma once

#include "common.cuh"
#include "kernels.h"
#include "mg2d.cuh"

namespace irk {

template <typename C>
struct Kappa4 {
  C sw, se, nw, ne;
};

template <typename C>
__device__ __forceinline__ Kappa4<C> kappa_around(const C* __restrict__ kap, int ix, int iy, int nx) {
  const int N = nx - 1;
  Kappa4<C> k;
  k.sw = kap[(ix - 1) + N * (iy - 1)];
  k.se = kap[ix + N * (iy - 1)];
  k.nw = kap[(ix - 1) + N * iy];
  k.ne = kap[ix + N * iy];
  return k;
}

// X(dx, dy): the value at the node offset by (dx, dy).
template <typename C, typename F>
__device__ __forceinline__ C k_apply_kappa(const Kappa4<C>& k, F X) {
  C y = C(4) * ((k.sw + k.se) + (k.nw + k.ne)) * X(0, 0);
  y -= (k.se + k.ne) * X(1, 0) + (k.sw + k.nw) * X(-1, 0);
  y -= (k.nw + k.ne) * X(0, 1) + (k.sw + k.se) * X(0, -1);
  y -= C(2) * ((k.ne * X(1, 1) + k.nw * X(-1, 1)) + (k.sw * X(-1, -1) + k.se * X(1, -1)));
  return y * C(1.0 / 6.0);
}

template <typename C, typename F>
__device__ __forceinline__ C m_apply_unscaled_off(F X) {
  C edge = (X(-1, 0) + X(1, 0)) + (X(0, -1) + X(0, 1));
  C corner = (X(-1, -1) + X(1, -1)) + (X(-1, 1) + X(1, 1));
  return C(16) * X(0, 0) + C(4) * edge + corner;
}

template <typename C>
__device__ __forceinline__ C kappa_diag(const Kappa4<C>& k) {
  return C(4.0 / 6.0) * ((k.sw + k.se) + (k.nw + k.ne));
}

#define IRK_2D_INTERIOR_INDEX                                 \
  const int ix = 1 + blockIdx.x * kBX + threadIdx.x;          \
  const int iy = 1 + blockIdx.y * kBY + threadIdx.y;          \
  if (ix > nx - 2 || iy > nx - 2) return;                     \
  const int p = ix + nx * iy;

// v[dy + 1][dx + 1] = stage i of x at the 3 x 3 neighbourhood of p.
template <int S, typename C, typename T>
__device__ __forceinline__ void gather3x3(const T* __restrict__ x, int p, int nx, int i, C v[3][3]) {
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) v[dy + 1][dx + 1] = ld<C>(x + (size_t)(p + dx + nx * dy) * S + i);
}

// 6 K x and the unscaled mass stencil at the centre of a 3 x 3 neighbourhood.
template <typename C>
__device__ __forceinline__ C k3x3(const Kappa4<C>& k, const C v[3][3]) {
  C y = C(4) * ((k.sw + k.se) + (k.nw + k.ne)) * v[1][1];
  y -= (k.se + k.ne) * v[1][2] + (k.sw + k.nw) * v[1][0];
  y -= (k.nw + k.ne) * v[2][1] + (k.sw + k.se) * v[0][1];
  y -= C(2) * ((k.ne * v[2][2] + k.nw * v[2][0]) + (k.sw * v[0][0] + k.se * v[0][2]));
  return y * C(1.0 / 6.0);
}
template <typename C>
__device__ __forceinline__ C m3x3(const C v[3][3]) {
  const C edge = (v[1][0] + v[1][2]) + (v[0][1] + v[2][1]);
  const C corner = (v[0][0] + v[0][2]) + (v[2][0] + v[2][2]);
  return C(16) * v[1][1] + C(4) * edge + corner;
}

// Jacobi sweep (xin == nullptr: zero guess); two_from_zero: x1 = d b formed at the 3 x 3
// neighbourhood (the neighbours' diagonals from a 4 x 4 patch of cells), then one sweep.
template <typename T, typename C, int S>
__global__ void __launch_bounds__(kBX* kBY) jacobi_kappa_kernel(int nx, const C* __restrict__ kap, C hm,
                                                                VecT<C> sigma, C omega, const T* __restrict__ xin,
                                                                const T* __restrict__ b, T* __restrict__ xout,
                                                                int two_from_zero) {
  IRK_PDL_ENTRY;
  IRK_2D_INTERIOR_INDEX
  const int N = nx - 1;
  C kd9[3][3];  // (4/6) sum of kappa around each node of the neighbourhood
  Kappa4<C> k;
  if (two_from_zero) {
    C kp[4][4];  // cells ix-2+cx, iy-2+cy; 0 outside the mesh (only boundary nodes use those)
#pragma unroll
    for (int cy = 0; cy < 4; ++cy)
#pragma unroll
      for (int cx = 0; cx < 4; ++cx) {
        const int gx = ix - 2 + cx, gy = iy - 2 + cy;
        kp[cy][cx] = (gx >= 0 && gy >= 0 && gx < N && gy < N) ? kap[gx + N * gy] : C(0);
      }
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx)
        kd9[dy][dx] = C(4.0 / 6.0) * ((kp[dy][dx] + kp[dy][dx + 1]) + (kp[dy + 1][dx] + kp[dy + 1][dx + 1]));
    k.sw = kp[1][1], k.se = kp[1][2], k.nw = kp[2][1], k.ne = kp[2][2];
  } else {
    k = kappa_around(kap, ix, iy, nx);
    kd9[1][1] = kappa_diag(k);
  }
#pragma unroll
  for (int i = 0; i < S; ++i) {
    const C bi = ld<C>(b + (size_t)p * S + i);
    const C d = __fdividef(omega, C(16) * hm + sigma.v[i] * kd9[1][1]);
    C xn;
    if (two_from_zero) {
      C v[3][3];
      gather3x3<S, C>(b, p, nx, i, v);
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          const bool in = interior2(ix + dx - 1, iy + dy - 1, nx);
          v[dy][dx] = in ? __fdividef(omega, C(16) * hm + sigma.v[i] * kd9[dy][dx]) * v[dy][dx] : C(0);
        }
      const C bx = hm * m3x3<C>(v) + sigma.v[i] * k3x3<C>(k, v);
      xn = v[1][1] + d * (bi - bx);
    } else if (xin == nullptr) {
      xn = d * bi;
    } else {
      C v[3][3];
      gather3x3<S, C>(xin, p, nx, i, v);
      const C bx = hm * m3x3<C>(v) + sigma.v[i] * k3x3<C>(k, v);
      xn = v[1][1] + d * (bi - bx);
    }
    st(xout + (size_t)p * S + i, xn);
  }
}

template <typename T, typename C, int S>
__global__ void __launch_bounds__(kBX* kBY) residual_kappa_kernel(int nx, const C* __restrict__ kap, C hm,
                                                                  VecT<C> sigma, const T* __restrict__ x,
                                                                  const T* __restrict__ b, T* __restrict__ r) {
  IRK_PDL_ENTRY;
  IRK_2D_INTERIOR_INDEX
  const Kappa4<C> k = kappa_around(kap, ix, iy, nx);
#pragma unroll
  for (int i = 0; i < S; ++i) {
    C v[3][3];
    gather3x3<S, C>(x, p, nx, i, v);
    const C bx = hm * m3x3<C>(v) + sigma.v[i] * k3x3<C>(k, v);
    st(r + (size_t)p * S + i, ld<C>(b + (size_t)p * S + i) - bx);
  }
}

// Block right-hand side of the triangular preconditioners with K from kappa.
template <typename T, typename C, int SF>
__global__ void __launch_bounds__(kBX* kBY) block_rhs_kappa_kernel(int nx, const C* __restrict__ kap,
                                                                   const double* __restrict__ v,
                                                                   const double* __restrict__ z, int i,
                                                                   VecT<C> cj, unsigned used, T* __restrict__ out) {
  IRK_PDL_ENTRY;
  IRK_2D_INTERIOR_INDEX
  const Kappa4<C> k = kappa_around(kap, ix, iy, nx);
  C acc = static_cast<C>(v[(size_t)p * SF + i]);
#pragma unroll
  for (int j = 0; j < SF; ++j) {
    if (used & (1u << j)) {
      C w[3][3];
      gather3x3<SF, C>(z, p, nx, j, w);
      acc -= cj.v[j] * k3x3<C>(k, w);
    }
  }
  st(out + p, acc);
}

template <typename T, typename C>
void MG2K<T, C>::jacobi(int S, cudaStream_t st, int nx, const C* kap, double hm, const Vec8& sigma, double omega,
                        const T* xin, const T* b, T* xout, int two_from_zero) {
  dim3 g = interior_grid(nx), blk(kBX, kBY);
  const VecT<C> sg = to_vec<C>(sigma);
  IRK_DISPATCH_S(S, launch_k(jacobi_kappa_kernel<T, C, SS>, g, blk, 0, st, nx, kap, (C)hm, sg, (C)omega, xin, b, xout,
                             two_from_zero));
}
template <typename T, typename C>
void MG2K<T, C>::residual(int S, cudaStream_t st, int nx, const C* kap, double hm, const Vec8& sigma, const T* x,
                          const T* b, T* r) {
  dim3 g = interior_grid(nx), blk(kBX, kBY);
  const VecT<C> sg = to_vec<C>(sigma);
  IRK_DISPATCH_S(S, launch_k(residual_kappa_kernel<T, C, SS>, g, blk, 0, st, nx, kap, (C)hm, sg, x, b, r));
}
template <typename T, typename C>
void MG2K<T, C>::block_rhs(int SF, cudaStream_t st, int nx, const C* kap, const double* v, const double* z, int i,
                           const Vec8& cj, T* out) {
  dim3 g = interior_grid(nx), blk(kBX, kBY);
  unsigned used = 0;
  for (int j = 0; j < SF; ++j)
    if (cj.v[j] != 0.0) used |= 1u << j;
  const VecT<C> c = to_vec<C>(cj);
  IRK_DISPATCH_S(SF, launch_k(block_rhs_kappa_kernel<T, C, SS>, g, blk, 0, st, nx, kap, v, z, i, c, used, out));
}

}  // namespace irk
