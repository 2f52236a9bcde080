// Shared device-side definitions of the GB300 stage-coupled RK solver.
//
// Grid conventions (2D, uniform mesh of the unit square with N cells per axis):
//   nx = N + 1 nodes per axis, node p = ix + nx * iy, x fastest; interior nodes
//   have 1 <= ix, iy <= nx - 2.  Every level vector spans the full node grid and
//   keeps zeros on the boundary (homogeneous Dirichlet), so stencils need no
//   bounds logic for interior nodes.  Stage vectors are node-major with the S
//   stage values of a node contiguous: v[p * S + i].
//
// The stiffness operator of a level is stored as a symmetric 9-point stencil,
// five values per node in one record: {D, E, N, NE, NW} = the couplings of p
// with itself, p+1, p+nx, p+nx+1 and p+nx-1.  The couplings towards W, S, SW
// and SE are read from the neighbours' records (symmetry).  The mass matrix of
// a level is the constant Q1 stencil (h^2/36) [1 4 1; 4 16 4; 1 4 1].
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <cstdlib>
#include <type_traits>
#include <utility>

namespace irk {

constexpr int kMaxS = 4;     // IRK_MAX_STAGES
constexpr int kCoef2 = 5;    // stencil record length (2D)

// Small fixed-size arrays passed to kernels by value.
struct Vec8 {
  double v[8];
};
struct Mat4 {
  double v[kMaxS * kMaxS];  // row-major S x S, leading dimension S
};

// Kernel parameters in the kernel's own arithmetic type: on GB300 the FP64 pipe
// runs at 1/64 of the FP32 rate, so even one double-to-float conversion per node
// is visible in an FP32 kernel.
template <typename C>
struct VecT {
  C v[8];
};
template <typename C>
struct ClsT {
  C v[kMaxS][4];
};
template <typename C>
struct MatT {
  C v[kMaxS * kMaxS];
};
template <typename C>
inline MatT<C> to_mat(const Mat4& a) {
  MatT<C> r;
  for (int i = 0; i < kMaxS * kMaxS; ++i) r.v[i] = static_cast<C>(a.v[i]);
  return r;
}
template <typename C>
inline VecT<C> to_vec(const Vec8& a) {
  VecT<C> r;
  for (int i = 0; i < 8; ++i) r.v[i] = static_cast<C>(a.v[i]);
  return r;
}

// ----------------------------------------------------------------------------
// programmatic dependent launch
// ----------------------------------------------------------------------------
// Every kernel of the library starts with IRK_PDL_ENTRY: it waits until the previous
// kernel in the stream has completed and its writes are visible (griddepcontrol.wait),
// then lets the next kernel be scheduled (griddepcontrol.launch_dependents).  A kernel
// launched with programmatic stream serialization can thus be scheduled while its
// predecessor finishes, so its launch latency overlaps that kernel's tail, which is
// most of the cost of the small coarse-level grids.  Without the launch attribute both
// instructions are no-ops.
#define IRK_PDL_ENTRY                                      \
  do {                                                     \
    asm volatile("griddepcontrol.wait;" ::: "memory");     \
    asm volatile("griddepcontrol.launch_dependents;" ::);  \
  } while (0)

// Which launches carry the attribute (environment IRK_PDL): none by default; IRK_PDL=1 puts it
// on the small-level multigrid kernels and the coarsest solve (launch_k_tail), IRK_PDL=2 on every
// launch.  Measured on GB300 (heat2d-1024-radau3 inside CUDA graphs): on every launch the steps
// ran about 4% slower (the dependent kernel's blocks sit on SMs that large kernels still need);
// on the small-level kernels alone it made no difference.
inline int pdl_mode() {
  static const int mode = [] {
    const char* e = getenv("IRK_PDL");
    if (e && e[0] == '2') return 2;
    if (e && e[0] == '1') return 1;
    return 0;
  }();
  return mode;
}

template <typename... KArgs, typename... Args>
inline void launch_pdl(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                       Args&&... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <typename... KArgs, typename... Args>
inline void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                     Args&&... args) {
  launch_pdl(pdl_mode() == 2, kernel, grid, block, smem, stream, std::forward<Args>(args)...);
}

// small-level multigrid kernels and the coarsest solve
template <typename... KArgs, typename... Args>
inline void launch_k_tail(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                          Args&&... args) {
  launch_pdl(pdl_mode() >= 1, kernel, grid, block, smem, stream, std::forward<Args>(args)...);
}

// ----------------------------------------------------------------------------
// precision helpers: storage type T, compute type C
// ----------------------------------------------------------------------------
template <typename C, typename T>
__device__ __forceinline__ C ld(const T* p) {
  return static_cast<C>(*p);
}
template <>
__device__ __forceinline__ float ld<float, __nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}
template <>
__device__ __forceinline__ double ld<double, __nv_bfloat16>(const __nv_bfloat16* p) {
  return static_cast<double>(__bfloat162float(*p));
}

template <typename T, typename C>
__device__ __forceinline__ void st(T* p, C v) {
  *p = static_cast<T>(v);
}
template <>
__device__ __forceinline__ void st<__nv_bfloat16, float>(__nv_bfloat16* p, float v) {
  *p = __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ void st<__nv_bfloat16, double>(__nv_bfloat16* p, double v) {
  *p = __float2bfloat16_rn(static_cast<float>(v));
}

// ----------------------------------------------------------------------------
// 2D stencil primitives at an interior node p
// ----------------------------------------------------------------------------
// Stencil records on the device are planar: coefficient k in {D, E, N, NE, NW} of node q of a level
// with nx nodes per axis is cf[k nx^2 + q] (a warp's loads of one coefficient are then coalesced).
// The symmetric 9-point stencil at p, with the neighbour values given by X(dx, dy).
template <typename C, typename F>
__device__ __forceinline__ C rec_apply_xy(const C* __restrict__ cf, int p, int nx, F X) {
  const size_t n = (size_t)nx * nx;
  C y = cf[p] * X(0, 0);
  y += cf[n + p] * X(1, 0);
  y += cf[n + p - 1] * X(-1, 0);
  y += cf[2 * n + p] * X(0, 1);
  y += cf[2 * n + p - nx] * X(0, -1);
  y += cf[3 * n + p] * X(1, 1);
  y += cf[3 * n + p - nx - 1] * X(-1, -1);
  y += cf[4 * n + p] * X(-1, 1);
  y += cf[4 * n + p - nx + 1] * X(1, -1);
  return y;
}

// (K x)(p) for one stage i of an S-interleaved vector.
template <int S, typename C, typename T>
__device__ __forceinline__ C k_apply(const C* __restrict__ cf, const T* __restrict__ x, int p, int nx, int i) {
  return rec_apply_xy<C>(cf, p, nx, [&](int dx, int dy) { return ld<C>(x + (size_t)(p + dx + nx * dy) * S + i); });
}

// 36/h^2 (M x)(p): the unscaled mass stencil [1 4 1; 4 16 4; 1 4 1].
template <int S, typename C, typename T>
__device__ __forceinline__ C m_apply_unscaled(const T* __restrict__ x, int p, int nx, int i) {
  auto X = [&](int q) { return ld<C>(x + (size_t)q * S + i); };
  C edge = X(p - 1) + X(p + 1) + X(p - nx) + X(p + nx);
  C corner = X(p - nx - 1) + X(p - nx + 1) + X(p + nx - 1) + X(p + nx + 1);
  return C(16) * X(p) + C(4) * edge + corner;
}

// The same 9-point stiffness and mass stencils applied to values produced by a
// functor F(q) (a vector that is never stored).
template <typename C, typename F>
__device__ __forceinline__ C k_apply_f(const C* __restrict__ cf, int p, int nx, F X) {
  return rec_apply_xy<C>(cf, p, nx, [&](int dx, int dy) { return X(p + dx + nx * dy); });
}

template <typename C, typename F>
__device__ __forceinline__ C m_apply_unscaled_f(int p, int nx, F X) {
  C edge = X(p - 1) + X(p + 1) + X(p - nx) + X(p + nx);
  C corner = X(p - nx - 1) + X(p - nx + 1) + X(p + nx - 1) + X(p + nx + 1);
  return C(16) * X(p) + C(4) * edge + corner;
}

__device__ __forceinline__ bool interior2(int ix, int iy, int nx) {
  return ix >= 1 && iy >= 1 && ix <= nx - 2 && iy <= nx - 2;
}

}  // namespace irk
