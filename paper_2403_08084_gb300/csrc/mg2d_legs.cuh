// Fused legs of the 2D V-cycles on the coarse levels, V(2, 2): the block V-cycles of Sec. 3.1 (the
// multigrid approximation of a diagonal block B = M + sigma K) and the monolithic cycle of Sec. 3
// (monolithic multigrid, all stages coupled).
//
// On the coarse levels the six kernels of a level (two pre-sweeps, residual,
// restriction, prolongation, two post-sweeps) each process so few nodes that a
// launch costs more than its work.  Two kernels replace them:
//
//   down leg   x2 = J(J(0; b)), r = b - B x2, b_c = P^T r
//   up leg     y0 = x + P e_c, y2 = J(J(y0; b))
//
// Each block owns a rectangle of fine nodes and recomputes the values its
// stencils need on a halo in shared memory (x1 on a halo of 2 and x2 on a halo
// of 1 for the down leg, y0 on 2 and y1 on 1 for the up leg).  The arithmetic at
// every node is that of the separate kernels (same stencil records, same order of
// operations), and the intermediate vectors kept in shared memory (in the arithmetic
// type C) are rounded to the storage type T as those kernels store them: with BF16
// storage, a residual formed from the unrounded iterate would not belong to the
// iterate that the coarse correction is added to.
//
// The relaxation J is a policy acting on all S stages of a node at once:
//   BlockRelax  independent blocks, x_i += d_i (b_i - B_i x_i) with d_i = omega / diag(B_i); B_i from the
//               stage's record (FP64 V-cycles: REC, stage-major with stride rstride) or hm M + sigma_i K
//               formed from the stiffness records cf (FP32 / BF16);
//   MonoRelax   the monolithic cycle's stage-coupled point-block Jacobi, x += W_p (b - S_l x) with
//               S_l x_i = hm M x_i + sum_j mix_ij K x_j and W_p = omega D_p^{-1} per node (S x S,
//               row-major; TRANS applies W_p^T, for the transposed cycle).
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace irk {

// 36/h^2 (M x) at a node, neighbour values from X(dx, dy); same order as m_apply_unscaled.
template <typename C, typename F>
__device__ __forceinline__ C mass_unscaled_xy(F X) {
  C edge = X(-1, 0) + X(1, 0) + X(0, -1) + X(0, 1);
  C corner = X(-1, -1) + X(1, -1) + X(-1, 1) + X(1, 1);
  return C(16) * X(0, 0) + C(4) * edge + corner;
}

// Independent blocks B_i with their Jacobi scalings.
template <typename C, int S, bool REC>
struct BlockRelax {
  // the two sweeps from zero of the separate kernels (jacobi2z) keep x1 in C
  static constexpr bool kStoreFirst = false;
  const C* rec;    // REC: records of B_0 .. B_{S-1} of this V-cycle, stage-major
  size_t rstride;  // REC: distance between the stages' records
  const C* cf;     // !REC: stiffness records
  C hm;
  VecT<C> sigma;
  const C* dinv;   // omega / diag(B_i): S values per node, node stride dstride
  int dstride;

  template <typename F>
  __device__ __forceinline__ C apply(int i, int p, int nx, F X) const {
    if constexpr (REC) {
      return rec_apply_xy<C>(rec + (size_t)i * rstride, p, nx, X);
    } else {
      return hm * mass_unscaled_xy<C>(X) + sigma.v[i] * rec_apply_xy<C>(cf, p, nx, X);
    }
  }
  // out = J(0; b)
  __device__ __forceinline__ void zero_sweep(int p, int /*nx*/, const C (&b)[S], C (&out)[S]) const {
#pragma unroll
    for (int i = 0; i < S; ++i) out[i] = dinv[(size_t)p * dstride + i] * b[i];
  }
  // out = J(x; b), stage i of the neighbour (dx, dy) of p given by XS(i, dx, dy)
  template <typename XS>
  __device__ __forceinline__ void sweep(int p, int nx, XS xs, const C (&b)[S], C (&out)[S]) const {
#pragma unroll
    for (int i = 0; i < S; ++i) {
      auto X = [&](int dx, int dy) { return xs(i, dx, dy); };
      out[i] = X(0, 0) + dinv[(size_t)p * dstride + i] * (b[i] - apply(i, p, nx, X));
    }
  }
  // out = b - B x
  template <typename XS>
  __device__ __forceinline__ void residual(int p, int nx, XS xs, const C (&b)[S], C (&out)[S]) const {
#pragma unroll
    for (int i = 0; i < S; ++i) {
      auto X = [&](int dx, int dy) { return xs(i, dx, dy); };
      out[i] = b[i] - apply(i, p, nx, X);
    }
  }
};

// One block (S = 1) whose sweeps use the scaled stencil (scaled_jacobi_records_2d: centre, E, W, N, S, NE,
// SW, NW, SE planes): J(x; b) = d b + sum_k c'_k x_k, ten FP64 operations per node instead of eleven; the
// residual keeps B's records.
template <typename C>
struct ScaledRelax {
  static constexpr bool kStoreFirst = false;
  const C* rec;   // B's records (residual)
  const C* sr;    // the nine scaled planes
  const C* dinv;  // d = omega / diag(B) per node

  __device__ __forceinline__ void zero_sweep(int p, int /*nx*/, const C (&b)[1], C (&out)[1]) const {
    out[0] = dinv[p] * b[0];
  }
  template <typename XS>
  __device__ __forceinline__ void sweep(int p, int nx, XS xs, const C (&b)[1], C (&out)[1]) const {
    const size_t n = (size_t)nx * nx;
    C acc = dinv[p] * b[0];
    acc = fma(sr[p], xs(0, 0, 0), acc);
    acc = fma(sr[n + p], xs(0, 1, 0), acc);
    acc = fma(sr[2 * n + p], xs(0, -1, 0), acc);
    acc = fma(sr[3 * n + p], xs(0, 0, 1), acc);
    acc = fma(sr[4 * n + p], xs(0, 0, -1), acc);
    acc = fma(sr[5 * n + p], xs(0, 1, 1), acc);
    acc = fma(sr[6 * n + p], xs(0, -1, -1), acc);
    acc = fma(sr[7 * n + p], xs(0, -1, 1), acc);
    acc = fma(sr[8 * n + p], xs(0, 1, -1), acc);
    out[0] = acc;
  }
  template <typename XS>
  __device__ __forceinline__ void residual(int p, int nx, XS xs, const C (&b)[1], C (&out)[1]) const {
    out[0] = b[0] - rec_apply_xy<C>(rec, p, nx, [&](int dx, int dy) { return xs(0, dx, dy); });
  }
};

// Stage-coupled point-block Jacobi of the monolithic cycle (same arithmetic as mmg_smooth_kernel and
// mmg_residual_kernel).
template <typename C, int S, bool TRANS>
struct MonoRelax {
  // the separate sweeps store x1 in T
  static constexpr bool kStoreFirst = true;
  const C* cf;   // stiffness records
  C hm;
  MatT<C> mix;   // dt A (dt A^T for the transposed cycle)
  const C* W;    // omega D_p^{-1}: entry (i, j) of node p at W[(i S + j) nx^2 + p]

  // y = S_l x at p
  template <typename XS>
  __device__ __forceinline__ void apply_all(int p, int nx, XS xs, C (&y)[S]) const {
    C kx[S];
#pragma unroll
    for (int j = 0; j < S; ++j) kx[j] = rec_apply_xy<C>(cf, p, nx, [&](int dx, int dy) { return xs(j, dx, dy); });
#pragma unroll
    for (int i = 0; i < S; ++i) {
      C v = hm * mass_unscaled_xy<C>([&](int dx, int dy) { return xs(i, dx, dy); });
#pragma unroll
      for (int j = 0; j < S; ++j) v += mix.v[i * S + j] * kx[j];
      y[i] = v;
    }
  }
  // out += W_p r (W_p^T r if TRANS)
  __device__ __forceinline__ void block_add(int p, int nx, const C (&r)[S], C (&out)[S]) const {
    const size_t n = (size_t)nx * nx;
#pragma unroll
    for (int i = 0; i < S; ++i) {
      C acc = out[i];
#pragma unroll
      for (int j = 0; j < S; ++j) acc += W[(size_t)(TRANS ? j * S + i : i * S + j) * n + p] * r[j];
      out[i] = acc;
    }
  }
  __device__ __forceinline__ void zero_sweep(int p, int nx, const C (&b)[S], C (&out)[S]) const {
#pragma unroll
    for (int i = 0; i < S; ++i) out[i] = C(0);
    block_add(p, nx, b, out);
  }
  template <typename XS>
  __device__ __forceinline__ void sweep(int p, int nx, XS xs, const C (&b)[S], C (&out)[S]) const {
    C r[S];
    residual(p, nx, xs, b, r);
#pragma unroll
    for (int i = 0; i < S; ++i) out[i] = xs(i, 0, 0);
    block_add(p, nx, r, out);
  }
  template <typename XS>
  __device__ __forceinline__ void residual(int p, int nx, XS xs, const C (&b)[S], C (&out)[S]) const {
    C sx[S];
    apply_all(p, nx, xs, sx);
#pragma unroll
    for (int i = 0; i < S; ++i) out[i] = b[i] - sx[i];
  }
};

__device__ __forceinline__ bool interior_node(int ix, int iy, int nx) {
  return ix >= 1 && iy >= 1 && ix <= nx - 2 && iy <= nx - 2;
}

// v rounded to the storage type T (the identity when T == C).
template <typename T, typename C>
__device__ __forceinline__ C stored(C v) {
  if constexpr (std::is_same<T, C>::value) {
    return v;
  } else {
    T t;
    st(&t, v);
    return ld<C>(&t);
  }
}

// Loads the S stages of b at node p.
template <typename T, typename C, int S>
__device__ __forceinline__ void load_stages(const T* __restrict__ b, int p, C (&bv)[S]) {
#pragma unroll
  for (int i = 0; i < S; ++i) bv[i] = ld<C>(b + (size_t)p * S + i);
}

// Down leg.  The block owns fine nodes [FX0, FX0 + 2CX) x [FY0, FY0 + 2CY), FX0 = 1 + 2 CX bx, and the
// coarse nodes I in [1 + CX bx, 1 + CX (bx + 1)) (fine node 2I), likewise in y.  Regions (fine, inclusive):
//   x1 on [FX0 - 2, FX0 + 2CX + 2], x2 on [FX0 - 1, FX0 + 2CX + 1], r on [FX0, FX0 + 2CX].
//
// NT threads; every phase loop has a compile-time trip count and is unrolled, so that all the
// global loads of a phase are in flight together (the small levels are latency-bound).
template <typename T, typename C, int S, int CX, int CY, int NT, typename R>
__device__ __forceinline__ void down_leg_tile(int bx, int by, int nxf, const R& relax, const T* __restrict__ b,
                                              T* __restrict__ xout, int nxc, T* __restrict__ bc,
                                              unsigned char* smem) {
  constexpr int W1 = 2 * CX + 5, H1 = 2 * CY + 5;
  constexpr int W2 = 2 * CX + 3, H2 = 2 * CY + 3;
  constexpr int W3 = 2 * CX + 1, H3 = 2 * CY + 1;
  C* X1 = reinterpret_cast<C*>(smem);
  C* X2 = X1 + W1 * H1 * S;
  C* Rr = X2 + W2 * H2 * S;
  const int FX0 = 1 + 2 * CX * bx, FY0 = 1 + 2 * CY * by;

  // x1 = J(0; b), 0 off the interior
#pragma unroll
  for (int t = threadIdx.x; t < W1 * H1; t += NT) {
    const int ix = FX0 - 2 + t % W1, iy = FY0 - 2 + t / W1;
    const int p = ix + nxf * iy;
    C out[S];
    if (interior_node(ix, iy, nxf)) {
      C bv[S];
      load_stages<T, C, S>(b, p, bv);
      relax.zero_sweep(p, nxf, bv, out);
    } else {
#pragma unroll
      for (int i = 0; i < S; ++i) out[i] = C(0);
    }
#pragma unroll
    for (int i = 0; i < S; ++i) X1[t * S + i] = R::kStoreFirst ? stored<T>(out[i]) : out[i];
  }
  __syncthreads();
  // x2 = J(x1; b); the owned part is the leg's smoothed iterate
#pragma unroll
  for (int t = threadIdx.x; t < W2 * H2; t += NT) {
    const int lx = t % W2, ly = t / W2;
    const int ix = FX0 - 1 + lx, iy = FY0 - 1 + ly;
    const bool in = interior_node(ix, iy, nxf);
    const bool own = in && ix >= FX0 && ix < FX0 + 2 * CX && iy >= FY0 && iy < FY0 + 2 * CY;
    const int p = ix + nxf * iy;
    C out[S];
    if (in) {
      C bv[S];
      load_stages<T, C, S>(b, p, bv);
      auto xs = [&](int i, int dx, int dy) { return X1[((ly + 1 + dy) * W1 + (lx + 1 + dx)) * S + i]; };
      relax.sweep(p, nxf, xs, bv, out);
    } else {
#pragma unroll
      for (int i = 0; i < S; ++i) out[i] = C(0);
    }
#pragma unroll
    for (int i = 0; i < S; ++i) {
      X2[t * S + i] = stored<T>(out[i]);
      if (own) st(xout + (size_t)p * S + i, out[i]);
    }
  }
  __syncthreads();
  // r = b - B x2
#pragma unroll
  for (int t = threadIdx.x; t < W3 * H3; t += NT) {
    const int lx = t % W3, ly = t / W3;
    const int ix = FX0 + lx, iy = FY0 + ly;
    const int p = ix + nxf * iy;
    C out[S];
    if (interior_node(ix, iy, nxf)) {
      C bv[S];
      load_stages<T, C, S>(b, p, bv);
      auto xs = [&](int i, int dx, int dy) { return X2[((ly + 1 + dy) * W2 + (lx + 1 + dx)) * S + i]; };
      relax.residual(p, nxf, xs, bv, out);
    } else {
#pragma unroll
      for (int i = 0; i < S; ++i) out[i] = C(0);
    }
#pragma unroll
    for (int i = 0; i < S; ++i) Rr[t * S + i] = stored<T>(out[i]);
  }
  __syncthreads();
  // b_c = P^T r (full weighting), same order as restrict_kernel
#pragma unroll
  for (int t = threadIdx.x; t < CX * CY; t += NT) {
    const int I = 1 + CX * bx + t % CX, J = 1 + CY * by + t / CX;
    if (I > nxc - 2 || J > nxc - 2) continue;
    const int lx = 2 * I - FX0, ly = 2 * J - FY0;  // in [1, 2CX - 1]
#pragma unroll
    for (int i = 0; i < S; ++i) {
      auto Rv = [&](int dx, int dy) { return Rr[((ly + dy) * W3 + (lx + dx)) * S + i]; };
      C v = Rv(0, 0) + C(0.5) * (Rv(-1, 0) + Rv(1, 0) + Rv(0, -1) + Rv(0, 1)) +
            C(0.25) * (Rv(-1, -1) + Rv(1, -1) + Rv(-1, 1) + Rv(1, 1));
      st(bc + (size_t)(I + nxc * J) * S + i, v);
    }
  }
}

template <typename T, typename C, int S, int CX, int CY, int NT, typename R>
__global__ void __launch_bounds__(NT) down_leg_kernel(int nxf, R relax, const T* __restrict__ b,
                                                       T* __restrict__ xout, int nxc, T* __restrict__ bc) {
  IRK_PDL_ENTRY;
  extern __shared__ unsigned char leg_smem[];
  down_leg_tile<T, C, S, CX, CY, NT, R>(blockIdx.x, blockIdx.y, nxf, relax, b, xout, nxc, bc, leg_smem);
}

// Up leg.  The block owns fine nodes [FX0, FX0 + TX) x [FY0, FY0 + TY), FX0 = 1 + TX bx.  Regions:
//   y0 = x + P e_c on [FX0 - 2, FX0 + TX + 1], y1 = J(y0) on [FX0 - 1, FX0 + TX], y2 = J(y1) owned.
// xout must not alias xin (other blocks read xin on their halos).
// With zs.z set (the finest level) y2 goes to the caller's FP64 stage vector instead of xout (ZSink in
// kernels.h): one block, z[p * zs.sf + zs.i] = zs.scale * y2 and zs.zt[p] = y2; all stages (zs.i < 0),
// z[p * S + k] = zs.sc[k] * y2_k; y2 rounded to T first (what the separate scatter or cast of the stored
// iterate wrote).
template <typename T, typename C, int S, int TX, int TY, int NT, typename R>
__device__ __forceinline__ void up_leg_tile(int bx, int by, int nxf, const R& relax, const T* __restrict__ xin,
                                            const T* __restrict__ b, int nxc, const T* __restrict__ ec,
                                            T* __restrict__ xout, unsigned char* smem,
                                            const ZSink<T>& zs = ZSink<T>{}) {
  constexpr int W0 = TX + 4, H0 = TY + 4;
  constexpr int W1 = TX + 2, H1 = TY + 2;
  C* Y0 = reinterpret_cast<C*>(smem);
  C* Y1 = Y0 + W0 * H0 * S;
  const int FX0 = 1 + TX * bx, FY0 = 1 + TY * by;

  // y0 = x + P e_c (bilinear interpolation as in prolong_add_kernel), 0 off the interior
#pragma unroll
  for (int t = threadIdx.x; t < W0 * H0; t += NT) {
    const int ix = FX0 - 2 + t % W0, iy = FY0 - 2 + t / W0;
    const bool in = interior_node(ix, iy, nxf);
    const int p = ix + nxf * iy;
    const int I0 = ix >> 1, I1 = (ix + 1) >> 1, J0 = iy >> 1, J1 = (iy + 1) >> 1;
#pragma unroll
    for (int i = 0; i < S; ++i) {
      C v = C(0);
      if (in) {
        auto E = [&](int I, int J) { return ld<C>(ec + (size_t)(I + nxc * J) * S + i); };
        const C pe = C(0.25) * ((E(I0, J0) + E(I1, J0)) + (E(I0, J1) + E(I1, J1)));
        v = ld<C>(xin + (size_t)p * S + i) + pe;
      }
      Y0[t * S + i] = stored<T>(v);
    }
  }
  __syncthreads();
  // y1 = J(y0; b)
#pragma unroll
  for (int t = threadIdx.x; t < W1 * H1; t += NT) {
    const int lx = t % W1, ly = t / W1;
    const int ix = FX0 - 1 + lx, iy = FY0 - 1 + ly;
    const int p = ix + nxf * iy;
    C out[S];
    if (interior_node(ix, iy, nxf)) {
      C bv[S];
      load_stages<T, C, S>(b, p, bv);
      auto xs = [&](int i, int dx, int dy) { return Y0[((ly + 1 + dy) * W0 + (lx + 1 + dx)) * S + i]; };
      relax.sweep(p, nxf, xs, bv, out);
    } else {
#pragma unroll
      for (int i = 0; i < S; ++i) out[i] = C(0);
    }
#pragma unroll
    for (int i = 0; i < S; ++i) Y1[t * S + i] = stored<T>(out[i]);
  }
  __syncthreads();
  // y2 = J(y1; b) on the owned nodes
#pragma unroll
  for (int t = threadIdx.x; t < TX * TY; t += NT) {
    const int lx = t % TX, ly = t / TX;
    const int ix = FX0 + lx, iy = FY0 + ly;
    if (!interior_node(ix, iy, nxf)) continue;
    const int p = ix + nxf * iy;
    C bv[S], out[S];
    load_stages<T, C, S>(b, p, bv);
    auto xs = [&](int i, int dx, int dy) { return Y1[((ly + 1 + dy) * W1 + (lx + 1 + dx)) * S + i]; };
    relax.sweep(p, nxf, xs, bv, out);
    if (zs.z != nullptr) {
      if (zs.i >= 0) {
        T t;
        st(&t, out[0]);
        zs.z[(size_t)p * zs.sf + zs.i] = zs.scale * static_cast<double>(ld<C>(&t));
        zs.zt[p] = t;
      } else {
#pragma unroll
        for (int i = 0; i < S; ++i) {
          T t;
          st(&t, out[i]);
          zs.z[(size_t)p * S + i] = zs.sc[i] * static_cast<double>(ld<C>(&t));
        }
      }
      continue;
    }
#pragma unroll
    for (int i = 0; i < S; ++i) st(xout + (size_t)p * S + i, out[i]);
  }
}

template <typename T, typename C, int S, int TX, int TY, int NT, typename R>
__global__ void __launch_bounds__(NT) up_leg_kernel(int nxf, R relax, const T* __restrict__ xin,
                                                     const T* __restrict__ b, int nxc, const T* __restrict__ ec,
                                                     T* __restrict__ xout, ZSink<T> zs) {
  IRK_PDL_ENTRY;
  extern __shared__ unsigned char leg_smem[];
  up_leg_tile<T, C, S, TX, TY, NT, R>(blockIdx.x, blockIdx.y, nxf, relax, xin, b, nxc, ec, xout, leg_smem, zs);
}

// ----------------------------------------------------------------------------
// launchers: tile sizes by level size (large levels: fewer halo nodes per owned
// node; small ones: more blocks in flight)
// ----------------------------------------------------------------------------
template <typename K>
inline void leg_smem_attr(K kernel, size_t smem) {
  if (smem > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T, typename C, int S, int CX, int CY, int NT, typename R>
void launch_down_leg(cudaStream_t st, int nxf, const R& relax, const T* b, T* xout, int nxc, T* bc) {
  constexpr int W1 = 2 * CX + 5, H1 = 2 * CY + 5, W2 = 2 * CX + 3, H2 = 2 * CY + 3, W3 = 2 * CX + 1, H3 = 2 * CY + 1;
  const size_t smem = sizeof(C) * S * (size_t)(W1 * H1 + W2 * H2 + W3 * H3);
  auto kern = down_leg_kernel<T, C, S, CX, CY, NT, R>;
  leg_smem_attr(kern, smem);
  const int m = nxf - 2;
  dim3 g((m + 2 * CX - 1) / (2 * CX), (m + 2 * CY - 1) / (2 * CY));
  launch_pdl(CX < 16 ? pdl_mode() >= 1 : pdl_mode() == 2, kern, g, dim3(NT), smem, st, nxf, relax, b, xout, nxc, bc);
}

template <typename T, typename C, int S, int TX, int TY, int NT, typename R>
void launch_up_leg(cudaStream_t st, int nxf, const R& relax, const T* xin, const T* b, int nxc, const T* ec,
                   T* xout, const ZSink<T>& zs) {
  const size_t smem = sizeof(C) * S * (size_t)((TX + 4) * (TY + 4) + (TX + 2) * (TY + 2));
  auto kern = up_leg_kernel<T, C, S, TX, TY, NT, R>;
  leg_smem_attr(kern, smem);
  const int m = nxf - 2;
  dim3 g((m + TX - 1) / TX, (m + TY - 1) / TY);
  launch_pdl(TX < 32 ? pdl_mode() >= 1 : pdl_mode() == 2, kern, g, dim3(NT), smem, st, nxf, relax, xin, b, nxc, ec,
             xout, zs);
}

// Levels whose fine grid has at least kMgLargeNx nodes per axis use the large tiles (fewer halo
// nodes per owned node, for the arithmetic-bound FP64 legs); smaller levels use 8 x 8 owned nodes
// per block so that each phase is one round of loads and there are many blocks in flight.
constexpr int kLegLargeNx = kMgLargeNx;

// Levels with kLegMediumNx <= nxf < kLegLargeNx use 16 x 16 owned nodes per block.
constexpr int kLegMediumNx = 257;

template <typename T, typename C, int S, typename R>
void down_leg_s(cudaStream_t st, int nxf, const R& relax, const T* b, T* xout, int nxc, T* bc) {
  if (nxf >= kLegLargeNx)
    launch_down_leg<T, C, S, 16, 8, 256>(st, nxf, relax, b, xout, nxc, bc);
  else if (nxf >= kLegMediumNx)  // regions 21 x 21, 19 x 19, 17 x 17
    launch_down_leg<T, C, S, 8, 8, 256>(st, nxf, relax, b, xout, nxc, bc);
  else  // regions 13 x 13, 11 x 11, 9 x 9
    launch_down_leg<T, C, S, 4, 4, 192>(st, nxf, relax, b, xout, nxc, bc);
}

template <typename T, typename C, int S, typename R>
void up_leg_s(cudaStream_t st, int nxf, const R& relax, const T* xin, const T* b, int nxc, const T* ec, T* xout,
              const ZSink<T>& zs = ZSink<T>{}) {
  if (nxf >= kLegLargeNx)
    launch_up_leg<T, C, S, 32, 16, 256>(st, nxf, relax, xin, b, nxc, ec, xout, zs);
  else if (nxf >= kLegMediumNx)  // regions 20 x 20, 18 x 18, 16 x 16
    launch_up_leg<T, C, S, 16, 16, 256>(st, nxf, relax, xin, b, nxc, ec, xout, zs);
  else  // regions 12 x 12, 10 x 10, 8 x 8
    launch_up_leg<T, C, S, 8, 8, 160>(st, nxf, relax, xin, b, nxc, ec, xout, zs);
}

#define IRK_LEG_DISPATCH(S, FN, ...)                                  \
  switch (S) {                                                        \
    case 1: FN<T, C, 1>(__VA_ARGS__); break;                          \
    case 2: FN<T, C, 2>(__VA_ARGS__); break;                          \
    case 3: FN<T, C, 3>(__VA_ARGS__); break;                          \
    case 4: FN<T, C, 4>(__VA_ARGS__); break;                          \
    default: break;                                                   \
  }

template <typename T, typename C, int S>
void down_leg_any(cudaStream_t st, int nxf, const C* cf, double hm, const Vec8& sigma, const C* rec, size_t rstride,
                  const C* dinv, int dstride, const T* b, T* xout, int nxc, T* bc, const C* srec) {
  if constexpr (S == 1) {
    if (srec != nullptr && rec != nullptr) {
      ScaledRelax<C> r{rec, srec, dinv};
      down_leg_s<T, C, 1>(st, nxf, r, b, xout, nxc, bc);
      return;
    }
  }
  if (rec != nullptr) {
    BlockRelax<C, S, true> r{rec, rstride, nullptr, C(0), {}, dinv, dstride};
    down_leg_s<T, C, S>(st, nxf, r, b, xout, nxc, bc);
  } else {
    BlockRelax<C, S, false> r{nullptr, 0, cf, (C)hm, to_vec<C>(sigma), dinv, dstride};
    down_leg_s<T, C, S>(st, nxf, r, b, xout, nxc, bc);
  }
}

template <typename T, typename C, int S>
void up_leg_any(cudaStream_t st, int nxf, const C* cf, double hm, const Vec8& sigma, const C* rec, size_t rstride,
                const C* dinv, int dstride, const T* xin, const T* b, int nxc, const T* ec, T* xout, const C* srec,
                const ZSink<T>& zs) {
  if constexpr (S == 1) {
    if (srec != nullptr && rec != nullptr) {
      ScaledRelax<C> r{rec, srec, dinv};
      up_leg_s<T, C, 1>(st, nxf, r, xin, b, nxc, ec, xout);
      return;
    }
  }
  // the stage-vector sink: one block, or all S stages of a batched cycle
  const ZSink<T> z1 = (S == 1 || zs.i < 0) ? zs : ZSink<T>{};
  if (rec != nullptr) {
    BlockRelax<C, S, true> r{rec, rstride, nullptr, C(0), {}, dinv, dstride};
    up_leg_s<T, C, S>(st, nxf, r, xin, b, nxc, ec, xout, z1);
  } else {
    BlockRelax<C, S, false> r{nullptr, 0, cf, (C)hm, to_vec<C>(sigma), dinv, dstride};
    up_leg_s<T, C, S>(st, nxf, r, xin, b, nxc, ec, xout, z1);
  }
}

template <typename T, typename C, int S>
void mmg_down_leg_any(cudaStream_t st, int nxf, const C* cf, double hm, const Mat4& mix, const C* dblk,
                      bool transpose, const T* b, T* xout, int nxc, T* bc) {
  if (transpose) {
    MonoRelax<C, S, true> r{cf, (C)hm, to_mat<C>(mix), dblk};
    down_leg_s<T, C, S>(st, nxf, r, b, xout, nxc, bc);
  } else {
    MonoRelax<C, S, false> r{cf, (C)hm, to_mat<C>(mix), dblk};
    down_leg_s<T, C, S>(st, nxf, r, b, xout, nxc, bc);
  }
}

template <typename T, typename C, int S>
void mmg_up_leg_any(cudaStream_t st, int nxf, const C* cf, double hm, const Mat4& mix, const C* dblk, bool transpose,
                    const T* xin, const T* b, int nxc, const T* ec, T* xout, const ZSink<T>& zs) {
  if (transpose) {
    MonoRelax<C, S, true> r{cf, (C)hm, to_mat<C>(mix), dblk};
    up_leg_s<T, C, S>(st, nxf, r, xin, b, nxc, ec, xout, zs);
  } else {
    MonoRelax<C, S, false> r{cf, (C)hm, to_mat<C>(mix), dblk};
    up_leg_s<T, C, S>(st, nxf, r, xin, b, nxc, ec, xout, zs);
  }
}

template <typename T, typename C>
void MG2<T, C>::down_leg(int S, cudaStream_t st, int nxf, const C* cf, double hm, const Vec8& sigma, const C* rec,
                         size_t rstride, const C* dinv, int dstride, const T* b, T* xout, int nxc, T* bc,
                         const C* srec) {
  IRK_LEG_DISPATCH(S, down_leg_any, st, nxf, cf, hm, sigma, rec, rstride, dinv, dstride, b, xout, nxc, bc, srec)
}

template <typename T, typename C>
void MG2<T, C>::up_leg(int S, cudaStream_t st, int nxf, const C* cf, double hm, const Vec8& sigma, const C* rec,
                       size_t rstride, const C* dinv, int dstride, const T* xin, const T* b, int nxc, const T* ec,
                       T* xout, const C* srec, const ZSink<T>& zs) {
  IRK_LEG_DISPATCH(S, up_leg_any, st, nxf, cf, hm, sigma, rec, rstride, dinv, dstride, xin, b, nxc, ec, xout, srec,
                   zs)
}

template <typename T, typename C>
void MG2<T, C>::mmg_down_leg(int S, cudaStream_t st, int nxf, const C* cf, double hm, const Mat4& mix, const C* dblk,
                             bool transpose, const T* b, T* xout, int nxc, T* bc) {
  IRK_LEG_DISPATCH(S, mmg_down_leg_any, st, nxf, cf, hm, mix, dblk, transpose, b, xout, nxc, bc)
}

template <typename T, typename C>
void MG2<T, C>::mmg_up_leg(int S, cudaStream_t st, int nxf, const C* cf, double hm, const Mat4& mix, const C* dblk,
                           bool transpose, const T* xin, const T* b, int nxc, const T* ec, T* xout,
                           const ZSink<T>& zs) {
  IRK_LEG_DISPATCH(S, mmg_up_leg_any, st, nxf, cf, hm, mix, dblk, transpose, xin, b, nxc, ec, xout, zs)
}

#undef IRK_LEG_DISPATCH

}  // namespace irk
