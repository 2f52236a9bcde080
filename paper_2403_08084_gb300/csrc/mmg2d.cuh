// Monolithic multigrid for the whole stage system of a 2D level (Sec. 3, monolithic multigrid):
//   S_l x = I (x) M_l x + (dt A) (x) K_l x
// on S-interleaved level vectors (S = s, all stages at once), relaxed by additive Schwarz over
// vertex patches with the stages coupled, which for Q1 is point-block Jacobi: at node p the s x s
// block M_l[p, p] I + dt K_l[p, p] A, whose damped inverse omega D_p^{-1} is stored planar like the
// stencil records (entry (i, j) of node p at dblk[(i S + j) nx^2 + p]).  Transfers reuse the stage-interleaved restriction and prolongation.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace irk {

// x_out = x_in + omega D^{-1} (b - S_l x_in) at interior nodes (x_in == nullptr: zero guess).
// TRANS: the transposed relaxation (D^{-T}; mix is then dt A^T), for the adjoint's transposed cycle.
template <typename T, typename C, int S, bool TRANS>
__global__ void __launch_bounds__(kBX* kBY) mmg_smooth_kernel(int nx, const C* __restrict__ cf, C hm, MatT<C> mix,
                                                              const C* __restrict__ dblk, const T* __restrict__ xin,
                                                              const T* __restrict__ b, T* __restrict__ xout) {
  IRK_PDL_ENTRY;
  const int ix = 1 + blockIdx.x * kBX + threadIdx.x;
  const int iy = 1 + blockIdx.y * kBY + threadIdx.y;
  if (ix > nx - 2 || iy > nx - 2) return;
  const int p = ix + nx * iy;
  C r[S];
  if (xin != nullptr) {
    C kx[S];
#pragma unroll
    for (int j = 0; j < S; ++j) kx[j] = k_apply<S, C>(cf, xin, p, nx, j);
#pragma unroll
    for (int i = 0; i < S; ++i) {
      C sx = hm * m_apply_unscaled<S, C>(xin, p, nx, i);
#pragma unroll
      for (int j = 0; j < S; ++j) sx += mix.v[i * S + j] * kx[j];
      r[i] = ld<C>(b + (size_t)p * S + i) - sx;
    }
  } else {
#pragma unroll
    for (int i = 0; i < S; ++i) r[i] = ld<C>(b + (size_t)p * S + i);
  }
  const size_t n = (size_t)nx * nx;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    C acc = (xin != nullptr) ? ld<C>(xin + (size_t)p * S + i) : C(0);
#pragma unroll
    for (int j = 0; j < S; ++j) acc += dblk[(size_t)(TRANS ? j * S + i : i * S + j) * n + p] * r[j];
    st(xout + (size_t)p * S + i, acc);
  }
}

// r = b - S_l x at interior nodes.
template <typename T, typename C, int S>
__global__ void __launch_bounds__(kBX* kBY) mmg_residual_kernel(int nx, const C* __restrict__ cf, C hm, MatT<C> mix,
                                                                const T* __restrict__ x, const T* __restrict__ b,
                                                                T* __restrict__ r) {
  IRK_PDL_ENTRY;
  const int ix = 1 + blockIdx.x * kBX + threadIdx.x;
  const int iy = 1 + blockIdx.y * kBY + threadIdx.y;
  if (ix > nx - 2 || iy > nx - 2) return;
  const int p = ix + nx * iy;
  C kx[S];
#pragma unroll
  for (int j = 0; j < S; ++j) kx[j] = k_apply<S, C>(cf, x, p, nx, j);
#pragma unroll
  for (int i = 0; i < S; ++i) {
    C sx = hm * m_apply_unscaled<S, C>(x, p, nx, i);
#pragma unroll
    for (int j = 0; j < S; ++j) sx += mix.v[i * S + j] * kx[j];
    st(r + (size_t)p * S + i, ld<C>(b + (size_t)p * S + i) - sx);
  }
}

// Exact coarsest solve of the coupled system with its dense inverse (n = S nint unknowns, interleaved:
// unknown c is stage c % S of interior node c / S).  One warp per row; each lane holds kCoarseChunk row
// entries per chunk in registers (as in coarse_solve_kernel).
template <typename T, typename C, int S>
__global__ void __launch_bounds__(kCoarseThreads) mmg_coarse_solve_kernel(int n, int nxc, const C* __restrict__ inv,
                                                                          const T* __restrict__ b,
                                                                          T* __restrict__ x) {
  IRK_PDL_ENTRY;
  extern __shared__ unsigned char smem_raw[];
  C* bs = reinterpret_cast<C*>(smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.x * (kCoarseThreads / 32) + warp;
  const C* row = inv + (size_t)(r < n ? r : 0) * n;
#pragma unroll 8
  for (int c = threadIdx.x; c < n; c += kCoarseThreads) bs[c] = ld<C>(b + (size_t)coarse_node(c / S, nxc) * S + c % S);
  __syncthreads();
  C acc = 0;
  for (int c0 = 0; c0 < n; c0 += 32 * kCoarseChunk) {
    C a[kCoarseChunk];
#pragma unroll
    for (int k = 0; k < kCoarseChunk; ++k) {
      const int c = c0 + lane + 32 * k;
      a[k] = (r < n && c < n) ? row[c] : C(0);
    }
    C p0 = 0, p1 = 0, p2 = 0, p3 = 0;
#pragma unroll
    for (int k = 0; k < kCoarseChunk; k += 4) {
      const int c = c0 + lane + 32 * k;
      if (c < n) p0 += a[k] * bs[c];
      if (c + 32 < n) p1 += a[k + 1] * bs[c + 32];
      if (c + 64 < n) p2 += a[k + 2] * bs[c + 64];
      if (c + 96 < n) p3 += a[k + 3] * bs[c + 96];
    }
    acc += (p0 + p1) + (p2 + p3);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0 && r < n) st(x + (size_t)coarse_node(r / S, nxc) * S + r % S, acc);
}

// The transposed coarsest solve x = inv^T b: one thread per output r, reading column r of inv
// (coalesced across a warp's consecutive r); b staged in shared memory.
template <typename T, typename C, int S>
__global__ void __launch_bounds__(kCoarseThreads) mmg_coarse_solve_t_kernel(int n, int nxc, const C* __restrict__ inv,
                                                                            const T* __restrict__ b,
                                                                            T* __restrict__ x) {
  IRK_PDL_ENTRY;
  extern __shared__ unsigned char smem_raw[];
  C* bs = reinterpret_cast<C*>(smem_raw);
  for (int c = threadIdx.x; c < n; c += kCoarseThreads) bs[c] = ld<C>(b + (size_t)coarse_node(c / S, nxc) * S + c % S);
  __syncthreads();
  const int r = blockIdx.x * kCoarseThreads + threadIdx.x;
  if (r >= n) return;
  C a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  int c = 0;
  for (; c + 3 < n; c += 4) {
    a0 += inv[(size_t)c * n + r] * bs[c];
    a1 += inv[(size_t)(c + 1) * n + r] * bs[c + 1];
    a2 += inv[(size_t)(c + 2) * n + r] * bs[c + 2];
    a3 += inv[(size_t)(c + 3) * n + r] * bs[c + 3];
  }
  for (; c < n; ++c) a0 += inv[(size_t)c * n + r] * bs[c];
  st(x + (size_t)coarse_node(r / S, nxc) * S + r % S, (a0 + a1) + (a2 + a3));
}

#define IRK_MMG_DISPATCH(S, ...)                              \
  switch (S) {                                                \
    case 1: { constexpr int SS = 1; __VA_ARGS__; } break;     \
    case 2: { constexpr int SS = 2; __VA_ARGS__; } break;     \
    case 3: { constexpr int SS = 3; __VA_ARGS__; } break;     \
    case 4: { constexpr int SS = 4; __VA_ARGS__; } break;     \
    default: break;                                           \
  }

template <typename T, typename C>
void MG2<T, C>::mmg_smooth(int S, cudaStream_t st, int nx, const C* cf, double hm, const Mat4& mix, const C* dblk,
                           const T* xin, const T* b, T* xout, bool transpose) {
  const MatT<C> m = to_mat<C>(mix);
  if (transpose) {
    IRK_MMG_DISPATCH(S, launch_k(mmg_smooth_kernel<T, C, SS, true>, interior_grid(nx), dim3(kBX, kBY), 0, st, nx, cf,
                                 (C)hm, m, dblk, xin, b, xout));
  } else {
    IRK_MMG_DISPATCH(S, launch_k(mmg_smooth_kernel<T, C, SS, false>, interior_grid(nx), dim3(kBX, kBY), 0, st, nx, cf,
                                 (C)hm, m, dblk, xin, b, xout));
  }
}

template <typename T, typename C>
void MG2<T, C>::mmg_residual(int S, cudaStream_t st, int nx, const C* cf, double hm, const Mat4& mix, const T* x,
                             const T* b, T* r) {
  const MatT<C> m = to_mat<C>(mix);
  IRK_MMG_DISPATCH(S, launch_k(mmg_residual_kernel<T, C, SS>, interior_grid(nx), dim3(kBX, kBY), 0, st, nx, cf,
                               (C)hm, m, x, b, r));
}

template <typename T, typename C>
void MG2<T, C>::mmg_coarse_solve(int S, cudaStream_t st, int nxc, const C* inv, const T* b, T* x, bool transpose) {
  const int n = S * (nxc - 2) * (nxc - 2);
  const size_t shm = sizeof(C) * (size_t)n;
  if (transpose) {
    const int g = (n + kCoarseThreads - 1) / kCoarseThreads;  // one thread per output
    IRK_MMG_DISPATCH(S, {
      auto kern = mmg_coarse_solve_t_kernel<T, C, SS>;
      if (shm > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
      launch_k(kern, dim3(g), dim3(kCoarseThreads), shm, st, n, nxc, inv, b, x);
    });
    return;
  }
  const int g = (n + kCoarseThreads / 32 - 1) / (kCoarseThreads / 32);  // one warp per row
  IRK_MMG_DISPATCH(S, {
    auto kern = mmg_coarse_solve_kernel<T, C, SS>;
    if (shm > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    launch_k(kern, dim3(g), dim3(kCoarseThreads), shm, st, n, nxc, inv, b, x);
  });
}

#undef IRK_MMG_DISPATCH

}  // namespace irk
