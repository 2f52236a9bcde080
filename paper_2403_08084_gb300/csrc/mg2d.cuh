// Geometric-multigrid kernels for one diagonal block B = M + sigma K of the
// stage system (Sec. 3.1: "approximate the inverse of this block with a
// standard multigrid method").  Templated on the vector storage type T, the
// arithmetic type C and the number S of stage-interleaved blocks handled in one
// pass (S > 1 batches the independent blocks of the block-diagonal
// preconditioner so that every stencil and coefficient load serves all S).
//
// The launchers at the bottom are explicitly instantiated per precision in
// mg2d_f64.cu / mg2d_f32.cu / mg2d_bf16.cu.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace irk {

constexpr int kBX = 32, kBY = 8;

inline dim3 interior_grid(int nx) {
  int m = nx - 2;
  return dim3((m + kBX - 1) / kBX, (m + kBY - 1) / kBY);
}

// Weighted Jacobi sweep  x_out = x_in + omega D^{-1} (b - B x_in), B = M + sigma_i K.
// dinv holds omega / diag(B) per node and stage with stride dstride; xin == nullptr
// means a zero initial guess (x_out = omega D^{-1} b).
template <typename T, typename C, int S>
__global__ void __launch_bounds__(kBX* kBY) jacobi_kernel(int nx, const C* __restrict__ cf, C hm, VecT<C> sigma,
                                                          const C* __restrict__ dinv, int dstride,
                                                          const T* __restrict__ xin, const T* __restrict__ b,
                                                          T* __restrict__ xout) {
  IRK_PDL_ENTRY;
  const int ix = 1 + blockIdx.x * kBX + threadIdx.x;
  const int iy = 1 + blockIdx.y * kBY + threadIdx.y;
  if (ix > nx - 2 || iy > nx - 2) return;
  const int p = ix + nx * iy;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    const C bi = ld<C>(b + (size_t)p * S + i);
    const C di = dinv[(size_t)p * dstride + i];
    C xn;
    if (xin == nullptr) {
      xn = di * bi;
    } else {
      const C bx = hm * m_apply_unscaled<S, C>(xin, p, nx, i) + sigma.v[i] * k_apply<S, C>(cf, xin, p, nx, i);
      xn = ld<C>(xin + (size_t)p * S + i) + di * (bi - bx);
    }
    st(xout + (size_t)p * S + i, xn);
  }
}

// The same sweep with B_i = M + sigma_i K stored as its own stencil record per
// stage (stage-major: record of stage i at rec + i * rstride): 9 products per
// node instead of separate mass and stiffness stencils.  Used by the FP64
// V-cycle, whose arithmetic (not its memory traffic) bounds it on GB300.
template <typename T, typename C, int S>
__global__ void __launch_bounds__(kBX* kBY) jacobi_rec_kernel(int nx, const C* __restrict__ rec, size_t rstride,
                                                              const C* __restrict__ dinv, int dstride,
                                                              const T* __restrict__ xin, const T* __restrict__ b,
                                                              T* __restrict__ xout) {
  IRK_PDL_ENTRY;
  const int ix = 1 + blockIdx.x * kBX + threadIdx.x;
  const int iy = 1 + blockIdx.y * kBY + threadIdx.y;
  if (ix > nx - 2 || iy > nx - 2) return;
  const int p = ix + nx * iy;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    const C bi = ld<C>(b + (size_t)p * S + i);
    const C di = dinv[(size_t)p * dstride + i];
    const C bx = k_apply<S, C>(rec + (size_t)i * rstride, xin, p, nx, i);
    st(xout + (size_t)p * S + i, ld<C>(xin + (size_t)p * S + i) + di * (bi - bx));
  }
}

// The sweeps after the first, x + d (b - B x) = x1 + sum_k c'_k x_k (x1 = d b, the sweep from zero),
// with the scaled stencil stored as nine planes (centre, E, W, N, S, NE, SW, NW, SE): nine FMAs per node
// where the record form takes eleven FP64 operations (its bound on GB300), for 32 more bytes of
// coalesced record reads.  One stage block.
template <typename T, typename C>
__global__ void __launch_bounds__(kBX* kBY) jacobi_scaled_kernel(int nx, const C* __restrict__ sr,
                                                                 const T* __restrict__ x1, const T* __restrict__ xin,
                                                                 T* __restrict__ xout) {
  IRK_PDL_ENTRY;
  const int ix = 1 + blockIdx.x * kBX + threadIdx.x;
  const int iy = 1 + blockIdx.y * kBY + threadIdx.y;
  if (ix > nx - 2 || iy > nx - 2) return;
  const int p = ix + nx * iy;
  const size_t n = (size_t)nx * nx;
  auto X = [&](int q) { return ld<C>(xin + q); };
  C acc = ld<C>(x1 + p);
  acc = fma(sr[p], X(p), acc);
  acc = fma(sr[n + p], X(p + 1), acc);
  acc = fma(sr[2 * n + p], X(p - 1), acc);
  acc = fma(sr[3 * n + p], X(p + nx), acc);
  acc = fma(sr[4 * n + p], X(p - nx), acc);
  acc = fma(sr[5 * n + p], X(p + nx + 1), acc);
  acc = fma(sr[6 * n + p], X(p - nx - 1), acc);
  acc = fma(sr[7 * n + p], X(p + nx - 1), acc);
  acc = fma(sr[8 * n + p], X(p - nx + 1), acc);
  st(xout + p, acc);
}

// The same sweep writing scale * x_out into stage i of the SF-interleaved FP64 vector z instead of a
// level vector: the last sweep of a block V-cycle in the triangular sweeps (what scatter_stage_kernel
// would write from its output).
template <typename C, int SF>
__global__ void __launch_bounds__(kBX* kBY) jacobi_scaled_z_kernel(int nx, const C* __restrict__ sr,
                                                                   const double* __restrict__ x1,
                                                                   const double* __restrict__ xin, int i,
                                                                   double* __restrict__ z, double scale) {
  IRK_PDL_ENTRY;
  const int ix = 1 + blockIdx.x * kBX + threadIdx.x;
  const int iy = 1 + blockIdx.y * kBY + threadIdx.y;
  if (ix > nx - 2 || iy > nx - 2) return;
  const int p = ix + nx * iy;
  const size_t n = (size_t)nx * nx;
  auto X = [&](int q) { return xin[q]; };
  double acc = x1[p];
  acc = fma(sr[p], X(p), acc);
  acc = fma(sr[n + p], X(p + 1), acc);
  acc = fma(sr[2 * n + p], X(p - 1), acc);
  acc = fma(sr[3 * n + p], X(p + nx), acc);
  acc = fma(sr[4 * n + p], X(p - nx), acc);
  acc = fma(sr[5 * n + p], X(p + nx + 1), acc);
  acc = fma(sr[6 * n + p], X(p - nx - 1), acc);
  acc = fma(sr[7 * n + p], X(p + nx - 1), acc);
  acc = fma(sr[8 * n + p], X(p - nx + 1), acc);
  z[(size_t)p * SF + i] = scale * acc;
}

template <typename T, typename C, int S>
__global__ void __launch_bounds__(kBX* kBY) residual_rec_kernel(int nx, const C* __restrict__ rec, size_t rstride,
                                                                const T* __restrict__ x, const T* __restrict__ b,
                                                                T* __restrict__ r) {
  IRK_PDL_ENTRY;
  const int ix = 1 + blockIdx.x * kBX + threadIdx.x;
  const int iy = 1 + blockIdx.y * kBY + threadIdx.y;
  if (ix > nx - 2 || iy > nx - 2) return;
  const int p = ix + nx * iy;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    const C bx = k_apply<S, C>(rec + (size_t)i * rstride, x, p, nx, i);
    st(r + (size_t)p * S + i, ld<C>(b + (size_t)p * S + i) - bx);
  }
}

// Two weighted-Jacobi sweeps from a zero initial guess in one pass:
// x1 = D^{-1} omega b is formed on the fly at the stencil points, x2 = x1 + d (b - B x1).
// rec == nullptr: B = hm M + sigma K from the stiffness records cf; else the B_i records.
template <typename T, typename C, int S>
__global__ void __launch_bounds__(kBX* kBY) jacobi2z_kernel(int nx, const C* __restrict__ cf, C hm, VecT<C> sigma,
                                                            const C* __restrict__ rec, size_t rstride,
                                                            const C* __restrict__ dinv, int dstride,
                                                            const T* __restrict__ b, T* __restrict__ xout) {
  IRK_PDL_ENTRY;
  const int ix = 1 + blockIdx.x * kBX + threadIdx.x;
  const int iy = 1 + blockIdx.y * kBY + threadIdx.y;
  if (ix > nx - 2 || iy > nx - 2) return;
  const int p = ix + nx * iy;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    auto X1 = [&](int q) { return dinv[(size_t)q * dstride + i] * ld<C>(b + (size_t)q * S + i); };
    C bx;
    if (rec != nullptr)
      bx = k_apply_f<C>(rec + (size_t)i * rstride, p, nx, X1);
    else
      bx = hm * m_apply_unscaled_f<C>(p, nx, X1) + sigma.v[i] * k_apply_f<C>(cf, p, nx, X1);
    const C bi = ld<C>(b + (size_t)p * S + i);
    st(xout + (size_t)p * S + i, X1(p) + dinv[(size_t)p * dstride + i] * (bi - bx));
  }
}

// r = b - B x on interior nodes.
template <typename T, typename C, int S>
__global__ void __launch_bounds__(kBX* kBY) residual_kernel(int nx, const C* __restrict__ cf, C hm, VecT<C> sigma,
                                                            const T* __restrict__ x, const T* __restrict__ b,
                                                            T* __restrict__ r) {
  IRK_PDL_ENTRY;
  const int ix = 1 + blockIdx.x * kBX + threadIdx.x;
  const int iy = 1 + blockIdx.y * kBY + threadIdx.y;
  if (ix > nx - 2 || iy > nx - 2) return;
  const int p = ix + nx * iy;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    const C bx = hm * m_apply_unscaled<S, C>(x, p, nx, i) + sigma.v[i] * k_apply<S, C>(cf, x, p, nx, i);
    st(r + (size_t)p * S + i, ld<C>(b + (size_t)p * S + i) - bx);
  }
}

// b_c = P^T r_f: full weighting (1, 1/2, 1/4) onto coarse interior nodes (the
// transpose of bilinear interpolation, so the coarse operators are Galerkin).
template <typename T, typename C, int S>
__global__ void __launch_bounds__(kBX* kBY) restrict_kernel(int nxf, const T* __restrict__ rf, int nxc,
                                                            T* __restrict__ bc) {
  IRK_PDL_ENTRY;
  const int I = 1 + blockIdx.x * kBX + threadIdx.x;
  const int J = 1 + blockIdx.y * kBY + threadIdx.y;
  if (I > nxc - 2 || J > nxc - 2) return;
  const int q = 2 * I + nxf * 2 * J;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    auto R = [&](int o) { return ld<C>(rf + (size_t)(q + o) * S + i); };
    C v = R(0) + C(0.5) * (R(-1) + R(1) + R(-nxf) + R(nxf)) +
          C(0.25) * (R(-nxf - 1) + R(-nxf + 1) + R(nxf - 1) + R(nxf + 1));
    st(bc + (size_t)(I + nxc * J) * S + i, v);
  }
}

// x_f += P e_c: bilinear interpolation.  Each thread takes the fine nodes ix (odd) and ix + 1 (even)
// of one row, between coarse columns I0 = ix >> 1 and I1 = I0 + 1.  Per parity the interpolant is
// E (even, even), the mean of two coarse values (one odd index) or of four (both odd); written that
// way it is bit-for-bit the four-corner average with repeated corners, in under half the operations.
template <typename T, typename C, int S>
__global__ void __launch_bounds__(kBX* kBY) prolong_add_kernel(int nxc, const T* __restrict__ ec, int nxf,
                                                               T* __restrict__ xf) {
  IRK_PDL_ENTRY;
  const int ix = 1 + 2 * (blockIdx.x * kBX + threadIdx.x);  // odd
  const int iy = 1 + blockIdx.y * kBY + threadIdx.y;
  if (ix > nxf - 2 || iy > nxf - 2) return;
  const bool two = ix + 1 <= nxf - 2;
  const int I0 = ix >> 1, I1 = I0 + 1, J0 = iy >> 1, J1 = (iy + 1) >> 1;
  const int p = ix + nxf * iy;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    auto E = [&](int I, int J) { return ld<C>(ec + (size_t)(I + nxc * J) * S + i); };
    C v_odd, v_even;
    if (J0 == J1) {
      const C a = E(I0, J0), b = E(I1, J0);
      v_odd = C(0.5) * (a + b);
      v_even = b;
    } else {
      const C b0 = E(I1, J0), b1 = E(I1, J1);
      v_odd = C(0.25) * ((E(I0, J0) + b0) + (E(I0, J1) + b1));
      v_even = C(0.5) * (b0 + b1);
    }
    st(xf + (size_t)p * S + i, ld<C>(xf + (size_t)p * S + i) + v_odd);
    if (two) st(xf + (size_t)(p + 1) * S + i, ld<C>(xf + (size_t)(p + 1) * S + i) + v_even);
  }
}

// Right-hand side of one block of the triangular preconditioners:
// out = v_i - sum_j cj[j] K z_j  (cj[j] = dt a_ij for the stages already solved, else 0).
// d1 != nullptr: also x1 = d1 * out, the first Jacobi sweep of the block's V-cycle from a zero guess
// (d1 = omega / diag of the block), so that the V-cycle starts at its second sweep.
// LOWZ (FP32 / BF16 V-cycles): the solved stages are read from zt + j * zstride, a stage-major copy
// of the V-cycle outputs in their own precision, instead of the FP64 stage vector z (no
// double-to-float conversions, which occupy the FP64 pipe on GB300); cj then includes each stage's
// output scale.
template <typename T, typename C, int SF, bool LOWZ>
__global__ void __launch_bounds__(kBX* kBY) block_rhs_kernel(int nx, const C* __restrict__ cf,
                                                             const double* __restrict__ v,
                                                             const double* __restrict__ z,
                                                             const T* __restrict__ zt, size_t zstride, int i,
                                                             VecT<C> cj, unsigned used, T* __restrict__ out,
                                                             const C* __restrict__ d1, T* __restrict__ x1) {
  IRK_PDL_ENTRY;
  const int ix = 1 + blockIdx.x * kBX + threadIdx.x;
  const int iy = 1 + blockIdx.y * kBY + threadIdx.y;
  if (ix > nx - 2 || iy > nx - 2) return;
  const int p = ix + nx * iy;
  C acc = static_cast<C>(v[(size_t)p * SF + i]);
#pragma unroll
  for (int j = 0; j < SF; ++j) {
    if (used & (1u << j)) {
      if constexpr (LOWZ)
        acc -= cj.v[j] * k_apply<1, C>(cf, zt + (size_t)j * zstride, p, nx, 0);
      else
        acc -= cj.v[j] * k_apply<SF, C>(cf, z, p, nx, j);
    }
  }
  st(out + p, acc);
  if (d1 != nullptr) st(x1 + p, d1[p] * ld<C>(out + p));
}

// IA form: out = v_i - sum_j cj[j] M z_j (M: the level's Q1 mass stencil; cjh = cj h^2 / 36).
// The mass stencil is separable, [1 4 1] (x) [1 4 1]: each thread takes two vertically adjacent
// interior nodes and shares the row sums of rows iy - 1 .. iy + 2 between them.
// d1 / x1, LOWZ / zt: as for block_rhs_kernel.
template <typename T, typename C, int SF, bool LOWZ>
__global__ void __launch_bounds__(kBX* kBY) block_rhs_mass_kernel(int nx, const double* __restrict__ v,
                                                                  const double* __restrict__ z,
                                                                  const T* __restrict__ zt, size_t zstride, int i,
                                                                  VecT<C> cjh, unsigned used, T* __restrict__ out,
                                                                  const C* __restrict__ d1, T* __restrict__ x1) {
  IRK_PDL_ENTRY;
  const int ix = 1 + blockIdx.x * kBX + threadIdx.x;
  const int iy0 = 1 + 2 * (blockIdx.y * kBY + threadIdx.y);
  if (ix > nx - 2 || iy0 > nx - 2) return;
  const bool two = iy0 + 1 <= nx - 2;
  const int p0 = ix + nx * iy0;
  C acc0 = static_cast<C>(v[(size_t)p0 * SF + i]);
  C acc1 = two ? static_cast<C>(v[(size_t)(p0 + nx) * SF + i]) : C(0);
#pragma unroll
  for (int j = 0; j < SF; ++j) {
    if (!(used & (1u << j))) continue;
    auto Z = [&](int q) {
      if constexpr (LOWZ)
        return ld<C>(zt + (size_t)j * zstride + q);
      else
        return ld<C>(z + (size_t)q * SF + j);
    };
    auto row = [&](int q) { return fma(C(4), Z(q), Z(q - 1)) + Z(q + 1); };
    const C r_m = row(p0 - nx), r_0 = row(p0), r_1 = row(p0 + nx);
    const C r_2 = (iy0 + 2 <= nx - 1) ? row(p0 + 2 * nx) : C(0);
    acc0 -= cjh.v[j] * (fma(C(4), r_0, r_m) + r_1);
    acc1 -= cjh.v[j] * (fma(C(4), r_1, r_0) + r_2);
  }
  st(out + p0, acc0);
  if (two) st(out + p0 + nx, acc1);
  if (d1 != nullptr) {
    st(x1 + p0, d1[p0] * ld<C>(out + p0));
    if (two) st(x1 + p0 + nx, d1[p0 + nx] * ld<C>(out + p0 + nx));
  }
}

// z[:, i] = scale * x on interior nodes (single-stage x into an SF-interleaved double vector);
// zt != nullptr: also zt[p] = x[p] (the unscaled V-cycle output kept in its own precision).
template <typename T, typename C, int SF>
__global__ void __launch_bounds__(kBX* kBY) scatter_stage_kernel(int nx, const T* __restrict__ x, int i,
                                                                 double* __restrict__ z, double scale,
                                                                 T* __restrict__ zt) {
  IRK_PDL_ENTRY;
  const int ix = 1 + blockIdx.x * kBX + threadIdx.x;
  const int iy = 1 + blockIdx.y * kBY + threadIdx.y;
  if (ix > nx - 2 || iy > nx - 2) return;
  const int p = ix + nx * iy;
  const T xv = x[p];
  z[(size_t)p * SF + i] = scale * static_cast<double>(ld<C>(&xv));
  if (zt != nullptr) zt[p] = xv;
}

template <typename T, typename C>
__global__ void cast_to_kernel(const double* __restrict__ src, T* __restrict__ dst, size_t n) {
  IRK_PDL_ENTRY;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    st(dst + e, static_cast<C>(src[e]));
}
template <typename T, typename C>
__global__ void cast_from_kernel(const T* __restrict__ src, double* __restrict__ dst, size_t n) {
  IRK_PDL_ENTRY;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = static_cast<double>(ld<C>(src + e));
}

// Exact coarsest-level solve x = B_c^{-1} b with a precomputed dense inverse per
// stage (the paper's multigrid uses a direct coarse solve).  blockIdx.y = stage;
// one warp per row.  The solve is a dense matrix-vector product whose matrix
// (7.4 MB in FP64 for a 32 x 32 coarsest mesh) is mostly evicted from L2 between
// V-cycles, so it is latency-bound unless many loads are in flight: each lane first
// issues the loads of its kCoarseChunk row entries (the whole row for up to 1024
// columns) into registers, and only then stages the right-hand side in shared
// memory (independent loads: interior unknown c is node (c % m + 1) + nxc (c / m + 1),
// m = nxc - 2), so the row fetch overlaps the staging.
constexpr int kCoarseChunk = 32;  // row entries per lane held in registers (32 x 32 = 1024 columns)
constexpr int kCoarseThreads = 128;

__device__ __forceinline__ int coarse_node(int c, int nxc) {
  const int m = nxc - 2;
  return (c % m + 1) + nxc * (c / m + 1);
}

// Launched with programmatic serialization: the row loads (the inverse is fixed for the handle)
// are issued before griddepcontrol.wait, so they overlap the previous kernel.
template <typename T, typename C, int S>
__global__ void __launch_bounds__(kCoarseThreads) coarse_solve_kernel(int nint, int nxc, const C* __restrict__ binv,
                                                                      const T* __restrict__ b, T* __restrict__ x) {
  asm volatile("griddepcontrol.launch_dependents;" ::);
  extern __shared__ unsigned char smem_raw[];
  C* bs = reinterpret_cast<C*>(smem_raw);
  const int i = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.x * (kCoarseThreads / 32) + warp;  // one row per warp; the grid covers every row
  const C* row = binv + (size_t)i * nint * nint + (size_t)(r < nint ? r : 0) * nint;
  C acc = 0;
  for (int c0 = 0; c0 < nint; c0 += 32 * kCoarseChunk) {
    C a[kCoarseChunk];
#pragma unroll
    for (int k = 0; k < kCoarseChunk; ++k) {
      const int c = c0 + lane + 32 * k;
      a[k] = (r < nint && c < nint) ? row[c] : C(0);
    }
    if (c0 == 0) {
      asm volatile("griddepcontrol.wait;" ::: "memory");  // b is the previous kernel's output
#pragma unroll 8
      for (int c = threadIdx.x; c < nint; c += kCoarseThreads) bs[c] = ld<C>(b + (size_t)coarse_node(c, nxc) * S + i);
      __syncthreads();
    }
    C p0 = 0, p1 = 0, p2 = 0, p3 = 0;
#pragma unroll
    for (int k = 0; k < kCoarseChunk; k += 4) {
      const int c = c0 + lane + 32 * k;
      if (c < nint) p0 += a[k] * bs[c];
      if (c + 32 < nint) p1 += a[k + 1] * bs[c + 32];
      if (c + 64 < nint) p2 += a[k + 2] * bs[c + 64];
      if (c + 96 < nint) p3 += a[k + 3] * bs[c + 96];
    }
    acc += (p0 + p1) + (p2 + p3);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0 && r < nint) st(x + (size_t)coarse_node(r, nxc) * S + i, acc);
}

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------
#define IRK_DISPATCH_S(S, ...)                 \
  switch (S) {                                 \
    case 1: { constexpr int SS = 1; __VA_ARGS__; } break; \
    case 2: { constexpr int SS = 2; __VA_ARGS__; } break; \
    case 3: { constexpr int SS = 3; __VA_ARGS__; } break; \
    case 4: { constexpr int SS = 4; __VA_ARGS__; } break; \
    default: break;                            \
  }

template <typename T, typename C>
void MG2<T, C>::jacobi(int S, cudaStream_t st, int nx, const C* cf, double hm, const Vec8& sigma, const C* dinv,
                       int dstride, const T* xin, const T* b, T* xout) {
  dim3 g = interior_grid(nx), blk(kBX, kBY);
  const VecT<C> sg = to_vec<C>(sigma);
  IRK_DISPATCH_S(S, launch_k(jacobi_kernel<T, C, SS>, g, blk, 0, st, nx, cf, (C)hm, sg, dinv, dstride, xin, b, xout));
}
template <typename T, typename C>
void MG2<T, C>::jacobi2z(int S, cudaStream_t st, int nx, const C* cf, double hm, const Vec8& sigma, const C* rec,
                         size_t rstride, const C* dinv, int dstride, const T* b, T* xout) {
  dim3 g = interior_grid(nx), blk(kBX, kBY);
  const VecT<C> sg = to_vec<C>(sigma);
  IRK_DISPATCH_S(S, launch_k(jacobi2z_kernel<T, C, SS>, g, blk, 0, st, nx, cf, (C)hm, sg, rec, rstride, dinv, dstride, b, xout));
}
template <typename T, typename C>
void MG2<T, C>::jacobi_rec(int S, cudaStream_t st, int nx, const C* rec, size_t rstride, const C* dinv, int dstride,
                           const T* xin, const T* b, T* xout) {
  dim3 g = interior_grid(nx), blk(kBX, kBY);
  IRK_DISPATCH_S(S, launch_k(jacobi_rec_kernel<T, C, SS>, g, blk, 0, st, nx, rec, rstride, dinv, dstride, xin, b, xout));
}
template <typename T, typename C>
void MG2<T, C>::jacobi_scaled(cudaStream_t st, int nx, const C* sr, const T* x1, const T* xin, T* xout) {
  dim3 g = interior_grid(nx), blk(kBX, kBY);
  launch_k(jacobi_scaled_kernel<T, C>, g, blk, 0, st, nx, sr, x1, xin, xout);
}
template <typename T, typename C>
bool MG2<T, C>::jacobi_scaled_z(int SF, cudaStream_t st, int nx, const C* sr, const T* x1, const T* xin, int i,
                                double* z, double scale) {
  if constexpr (std::is_same<T, double>::value && std::is_same<C, double>::value) {
    dim3 g = interior_grid(nx), blk(kBX, kBY);
    IRK_DISPATCH_S(SF, launch_k(jacobi_scaled_z_kernel<C, SS>, g, blk, 0, st, nx, sr, x1, xin, i, z, scale));
    return true;
  } else {
    return false;
  }
}
template <typename T, typename C>
void MG2<T, C>::residual_rec(int S, cudaStream_t st, int nx, const C* rec, size_t rstride, const T* x, const T* b,
                             T* r) {
  dim3 g = interior_grid(nx), blk(kBX, kBY);
  IRK_DISPATCH_S(S, launch_k(residual_rec_kernel<T, C, SS>, g, blk, 0, st, nx, rec, rstride, x, b, r));
}
template <typename T, typename C>
void MG2<T, C>::residual(int S, cudaStream_t st, int nx, const C* cf, double hm, const Vec8& sigma, const T* x,
                         const T* b, T* r) {
  dim3 g = interior_grid(nx), blk(kBX, kBY);
  const VecT<C> sg = to_vec<C>(sigma);
  IRK_DISPATCH_S(S, launch_k(residual_kernel<T, C, SS>, g, blk, 0, st, nx, cf, (C)hm, sg, x, b, r));
}
template <typename T, typename C>
void MG2<T, C>::restrict_(int S, cudaStream_t st, int nxf, const T* rf, int nxc, T* bc) {
  dim3 g = interior_grid(nxc), blk(kBX, kBY);
  IRK_DISPATCH_S(S, launch_k(restrict_kernel<T, C, SS>, g, blk, 0, st, nxf, rf, nxc, bc));
}
template <typename T, typename C>
void MG2<T, C>::prolong_add(int S, cudaStream_t st, int nxc, const T* ec, int nxf, T* xf) {
  const int m = nxf - 2;
  dim3 g(((m + 1) / 2 + kBX - 1) / kBX, (m + kBY - 1) / kBY), blk(kBX, kBY);  // two nodes per thread in x
  IRK_DISPATCH_S(S, launch_k(prolong_add_kernel<T, C, SS>, g, blk, 0, st, nxc, ec, nxf, xf));
}
template <typename T, typename C>
void MG2<T, C>::block_rhs(int SF, cudaStream_t st, int nx, const C* cf, const double* v, const double* z, int i,
                          const Vec8& cj, T* out, const C* d1, T* x1, const T* zt, size_t zstride) {
  dim3 g = interior_grid(nx), blk(kBX, kBY);
  unsigned used = 0;
  for (int j = 0; j < SF; ++j)
    if (cj.v[j] != 0.0) used |= 1u << j;
  const VecT<C> c = to_vec<C>(cj);
  if (zt != nullptr) {
    IRK_DISPATCH_S(SF, launch_k(block_rhs_kernel<T, C, SS, true>, g, blk, 0, st, nx, cf, v, z, zt, zstride, i, c,
                                used, out, d1, x1));
  } else {
    IRK_DISPATCH_S(SF, launch_k(block_rhs_kernel<T, C, SS, false>, g, blk, 0, st, nx, cf, v, z, zt, zstride, i, c,
                                used, out, d1, x1));
  }
}
template <typename T, typename C>
void MG2<T, C>::scatter_stage(int SF, cudaStream_t st, int nx, const T* x, int i, double* z, double scale, T* zt) {
  dim3 g = interior_grid(nx), blk(kBX, kBY);
  IRK_DISPATCH_S(SF, launch_k(scatter_stage_kernel<T, C, SS>, g, blk, 0, st, nx, x, i, z, scale, zt));
}
template <typename T, typename C>
void MG2<T, C>::block_rhs_mass(int SF, cudaStream_t st, int nx, double hm, const double* v, const double* z, int i,
                               const Vec8& cj, T* out, const C* d1, T* x1, const T* zt, size_t zstride) {
  const int m = nx - 2;
  dim3 g((m + kBX - 1) / kBX, ((m + 1) / 2 + kBY - 1) / kBY), blk(kBX, kBY);  // two rows per thread
  unsigned used = 0;
  Vec8 cjh{};
  for (int j = 0; j < SF; ++j) {
    if (cj.v[j] != 0.0) used |= 1u << j;
    cjh.v[j] = cj.v[j] * hm;
  }
  const VecT<C> c = to_vec<C>(cjh);
  if (zt != nullptr) {
    IRK_DISPATCH_S(SF, launch_k(block_rhs_mass_kernel<T, C, SS, true>, g, blk, 0, st, nx, v, z, zt, zstride, i, c,
                                used, out, d1, x1));
  } else {
    IRK_DISPATCH_S(SF, launch_k(block_rhs_mass_kernel<T, C, SS, false>, g, blk, 0, st, nx, v, z, zt, zstride, i, c,
                                used, out, d1, x1));
  }
}
template <typename T, typename C>
void MG2<T, C>::cast_to(cudaStream_t st, const double* src, T* dst, size_t n) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  launch_k(cast_to_kernel<T, C>, blocks, 256, 0, st, src, dst, n);
}
template <typename T, typename C>
void MG2<T, C>::cast_from(cudaStream_t st, const T* src, double* dst, size_t n) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  launch_k(cast_from_kernel<T, C>, blocks, 256, 0, st, src, dst, n);
}
template <typename T, typename C>
void MG2<T, C>::coarse_solve(int S, cudaStream_t st, int nxc, const C* binv, const T* b, T* x) {
  const int nint = (nxc - 2) * (nxc - 2);
  const int gx = (nint + kCoarseThreads / 32 - 1) / (kCoarseThreads / 32);  // one warp per row
  dim3 g(gx, S);
  size_t shm = sizeof(C) * (size_t)nint;
  IRK_DISPATCH_S(S, launch_k_tail(coarse_solve_kernel<T, C, SS>, g, kCoarseThreads, shm, st, nint, nxc, binv, b, x));
}

}  // namespace irk

#include "mg2d_legs.cuh"
#include "mg2d_tail.cuh"
#include "mmg2d.cuh"
