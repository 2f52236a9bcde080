// FP64 kernels of flexible GMRES (the outer solver of Sec. 4.1): Arnoldi
// multi-dot products and multi-axpys for classical Gram-Schmidt applied twice,
// the Givens update of the Hessenberg column and the triangular solve, all on
// the device so the host never reads the Krylov data.
//
// Reductions are deterministic: every block writes one partial sum per dot
// product and a second kernel adds the partials in a fixed order.
#include "common.cuh"
#include "kernels.h"

#include <cmath>

namespace irk {

namespace {
constexpr int kThreads = 256;
constexpr int kPartialBlocks = 152 * 8;  // partial sums per dot product (8 blocks per SM)
constexpr int kGroup = 8;                // dot products accumulated per pass over w

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Accumulate G dot products V_{k0+g} . w over this thread's elements (G known at compile
// time: no predicated-off FP64 work for partial groups).
template <int G>
__device__ __forceinline__ void multidot_accumulate(const double* __restrict__ V, size_t ld, int k0,
                                                    const double* __restrict__ w, size_t n, double acc[kGroup]) {
  for (size_t e = blockIdx.x * (size_t)kThreads + threadIdx.x; e < n; e += (size_t)gridDim.x * kThreads) {
    const double we = w[e];
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = fma(V[(size_t)(k0 + g) * ld + e], we, acc[g]);
  }
}

// partial[k * nb + blockIdx.x] = sum over this block's elements of V_k[e] w[e],
// for k = blockIdx.y * kGroup + g < count.
__global__ void __launch_bounds__(kThreads) multidot_kernel(const double* __restrict__ V, size_t ld, int count,
                                                            const double* __restrict__ w, size_t n,
                                                            double* __restrict__ partial,
                                                            const int* __restrict__ run_if) {
  IRK_PDL_ENTRY;
  if (run_if != nullptr && *run_if == 0) return;
  __shared__ double red[kThreads / 32][kGroup];
  const int k0 = blockIdx.y * kGroup;
  const int kn = min(kGroup, count - k0);
  double acc[kGroup];
#pragma unroll
  for (int g = 0; g < kGroup; ++g) acc[g] = 0.0;
  switch (kn) {
    case 1: multidot_accumulate<1>(V, ld, k0, w, n, acc); break;
    case 2: multidot_accumulate<2>(V, ld, k0, w, n, acc); break;
    case 3: multidot_accumulate<3>(V, ld, k0, w, n, acc); break;
    case 4: multidot_accumulate<4>(V, ld, k0, w, n, acc); break;
    case 5: multidot_accumulate<5>(V, ld, k0, w, n, acc); break;
    case 6: multidot_accumulate<6>(V, ld, k0, w, n, acc); break;
    case 7: multidot_accumulate<7>(V, ld, k0, w, n, acc); break;
    default: multidot_accumulate<8>(V, ld, k0, w, n, acc); break;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int g = 0; g < kGroup; ++g) {
    if (g < kn) {
      const double v = warp_sum(acc[g]);
      if (lane == 0) red[warp][g] = v;
    }
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int g = 0; g < kGroup; ++g) {
      if (g < kn) {
        double v = (lane < kThreads / 32) ? red[lane][g] : 0.0;
        v = warp_sum(v);
        if (lane == 0) partial[(size_t)(k0 + g) * gridDim.x + blockIdx.x] = v;
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads) reduce_partials_kernel(const double* __restrict__ partial, int nb,
                                                                   double* __restrict__ out,
                                                                   const int* __restrict__ run_if) {
  IRK_PDL_ENTRY;
  if (run_if != nullptr && *run_if == 0) return;
  __shared__ double red[kThreads / 32];
  const int k = blockIdx.x;
  double v = 0.0;
  for (int b = threadIdx.x; b < nb; b += kThreads) v += partial[(size_t)k * nb + b];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = (lane < kThreads / 32) ? red[lane] : 0.0;
    v = warp_sum(v);
    if (lane == 0) out[k] = v;
  }
}

// w = (w + sign * sum_k coef[k] V_k) * scale   (scale == nullptr: 1)
__global__ void __launch_bounds__(kThreads) multi_axpy_kernel(double* __restrict__ w, const double* __restrict__ V,
                                                              size_t ld, int count, const double* __restrict__ coef,
                                                              double sign, size_t n, const double* __restrict__ scale,
                                                              const int* __restrict__ run_if) {
  IRK_PDL_ENTRY;
  if (run_if != nullptr && *run_if == 0) return;
  __shared__ double c[128];
  for (int k = threadIdx.x; k < count; k += kThreads) c[k] = sign * coef[k];
  __syncthreads();
  const double sc = (scale != nullptr) ? *scale : 1.0;
  for (size_t e = blockIdx.x * (size_t)kThreads + threadIdx.x; e < n; e += (size_t)gridDim.x * kThreads) {
    double acc = w[e];
    for (int k = 0; k < count; ++k) acc = fma(c[k], V[(size_t)k * ld + e], acc);
    w[e] = (scale != nullptr) ? acc * sc : acc;
  }
}

// The middle of classical Gram-Schmidt applied twice, in one pass over V:
//   w' = w - sum_k coef[k] V_k   (written back to w), and
//   partial sums of V_k . w' for k < K and of w' . w' (as entry K),
// each thread keeping its K entries of V in registers between the update and the dot
// products (one read of V instead of two).  Layout of partial as in multidot_kernel.
constexpr int kAxpyDotMax = 16;  // largest K handled; the caller falls back to two kernels above

template <int K>
__global__ void __launch_bounds__(kThreads) axpy_dot_kernel(double* __restrict__ w, const double* __restrict__ V,
                                                            size_t ld, const double* __restrict__ coef, size_t n,
                                                            double* __restrict__ partial) {
  IRK_PDL_ENTRY;
  __shared__ double c[K];
  __shared__ double red[kThreads / 32][K + 1];
  if (threadIdx.x < K) c[threadIdx.x] = coef[threadIdx.x];
  __syncthreads();
  double d[K + 1];
#pragma unroll
  for (int k = 0; k <= K; ++k) d[k] = 0.0;
  for (size_t e = blockIdx.x * (size_t)kThreads + threadIdx.x; e < n; e += (size_t)gridDim.x * kThreads) {
    double v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = V[(size_t)k * ld + e];
    double acc = w[e];
#pragma unroll
    for (int k = 0; k < K; ++k) acc = fma(-c[k], v[k], acc);
    w[e] = acc;
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] = fma(v[k], acc, d[k]);
    d[K] = fma(acc, acc, d[K]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k <= K; ++k) {
    const double t = warp_sum(d[k]);
    if (lane == 0) red[warp][k] = t;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k <= K; ++k) {
      double t = (lane < kThreads / 32) ? red[lane][k] : 0.0;
      t = warp_sum(t);
      if (lane == 0) partial[(size_t)k * gridDim.x + blockIdx.x] = t;
    }
  }
}

// w -= sum_k coef[k] V_k, with the partial sums of the updated w . w (layout of multidot_kernel, one product).
__global__ void __launch_bounds__(kThreads) axpy_norm_kernel(double* __restrict__ w, const double* __restrict__ V,
                                                             size_t ld, int count, const double* __restrict__ coef,
                                                             size_t n, double* __restrict__ partial) {
  IRK_PDL_ENTRY;
  __shared__ double c[128];
  __shared__ double red[kThreads / 32];
  for (int k = threadIdx.x; k < count; k += kThreads) c[k] = coef[k];
  __syncthreads();
  double d = 0.0;
  for (size_t e = blockIdx.x * (size_t)kThreads + threadIdx.x; e < n; e += (size_t)gridDim.x * kThreads) {
    double acc = w[e];
    for (int k = 0; k < count; ++k) acc = fma(-c[k], V[(size_t)k * ld + e], acc);
    w[e] = acc;
    d = fma(acc, acc, d);
  }
  d = warp_sum(d);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = d;
  __syncthreads();
  if (warp == 0) {
    d = (lane < kThreads / 32) ? red[lane] : 0.0;
    d = warp_sum(d);
    if (lane == 0) partial[blockIdx.x] = d;
  }
}

// The same update + norm with the basis count K known at compile time: the K loads of an element
// are issued together, U elements per thread per pass (U = 2 for K >= 4: more independent work per
// warp; measured on GB300 10-16% faster than the run-time loop for K >= 4, 20% for K <= 3 with U = 1).
template <int K, int U>
__global__ void __launch_bounds__(kThreads) axpy_norm_k_kernel(double* __restrict__ w, const double* __restrict__ V,
                                                               size_t ld, const double* __restrict__ coef, size_t n,
                                                               double* __restrict__ partial) {
  IRK_PDL_ENTRY;
  __shared__ double c[K];
  __shared__ double red[kThreads / 32];
  if (threadIdx.x < K) c[threadIdx.x] = coef[threadIdx.x];
  __syncthreads();
  double d[U];
#pragma unroll
  for (int u = 0; u < U; ++u) d[u] = 0.0;
  const size_t stride = (size_t)gridDim.x * kThreads;
  size_t e = blockIdx.x * (size_t)kThreads + threadIdx.x;
  for (; e + (U - 1) * stride < n; e += U * stride) {
    double acc[U], v[U][K];
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = w[e + u * stride];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int k = 0; k < K; ++k) v[u][k] = V[(size_t)k * ld + e + u * stride];
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int k = 0; k < K; ++k) acc[u] = fma(-c[k], v[u][k], acc[u]);
      w[e + u * stride] = acc[u];
      d[u] = fma(acc[u], acc[u], d[u]);
    }
  }
  for (; e < n; e += stride) {  // U > 1: the last partial pass
    double acc = w[e];
#pragma unroll
    for (int k = 0; k < K; ++k) acc = fma(-c[k], V[(size_t)k * ld + e], acc);
    w[e] = acc;
    d[0] = fma(acc, acc, d[0]);
  }
  double t = d[0];
#pragma unroll
  for (int u = 1; u < U; ++u) t += d[u];
  t = warp_sum(t);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = t;
  __syncthreads();
  if (warp == 0) {
    t = (lane < kThreads / 32) ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) partial[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kThreads) scale_kernel(double* __restrict__ dst, const double* __restrict__ src,
                                                         const double* __restrict__ denom, size_t n,
                                                         const int* __restrict__ run_if) {
  IRK_PDL_ENTRY;
  if (run_if != nullptr && *run_if == 0) return;
  const double d = *denom;
  const double inv = (d != 0.0) ? 1.0 / d : 0.0;
  for (size_t e = blockIdx.x * (size_t)kThreads + threadIdx.x; e < n; e += (size_t)gridDim.x * kThreads)
    dst[e] = src[e] * inv;
}

// Column j of the Hessenberg matrix is h1 + h2 (the two Gram-Schmidt passes) with
// subdiagonal hn = sqrt(hn2); apply the earlier rotations, form the new one,
// update g and report |g_{j+1}| / r0.  One thread.
// pythag != 0: hn2 is not used; ||w''||^2 = ||w'||^2 - sum_i h2[i]^2 with ||w'||^2 in
// h2[j + 1] (the second pass saw w' itself as basis vector j + 1), and inv_out = 1 / ||w''||
// lets the second update normalise in the same sweep.
__global__ void givens_kernel(int j, int ldh, double* __restrict__ H, double* __restrict__ cs,
                              double* __restrict__ sn, double* __restrict__ g, const double* __restrict__ h1,
                              const double* __restrict__ h2, const double* __restrict__ hn2,
                              double* __restrict__ hn_out, const double* __restrict__ r0p,
                              double* __restrict__ rel_out, int pythag, double* __restrict__ inv_out) {
  IRK_PDL_ENTRY;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* col = H + (size_t)j * ldh;
  for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
  double hn2v;
  if (pythag) {
    double q = 0.0;
    for (int i = 0; i <= j; ++i) q += h2[i] * h2[i];
    hn2v = h2[j + 1] - q;
  } else {
    hn2v = *hn2;
  }
  const double hn = (hn2v < 0.0) ? 0.0 : sqrt(hn2v);  // NaN stays NaN (fmax would hide it)
  col[j + 1] = hn;
  *hn_out = hn;
  for (int i = 0; i < j; ++i) {
    const double a = col[i], b = col[i + 1];
    col[i] = cs[i] * a + sn[i] * b;
    col[i + 1] = -sn[i] * a + cs[i] * b;
  }
  const double a = col[j], b = col[j + 1];
  const double rho = hypot(a, b);
  double c = 1.0, s = 0.0;
  if (rho != 0.0) {
    c = a / rho;
    s = b / rho;
  }
  cs[j] = c;
  sn[j] = s;
  col[j] = rho;
  col[j + 1] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  rel_out[0] = fabs(g[j + 1]) / *r0p;
  rel_out[1] = hn;
  if (inv_out != nullptr) *inv_out = (hn > 0.0) ? 1.0 / hn : 0.0;
}

// Classical Gram-Schmidt with the selective re-orthogonalisation test of Daniel,
// Gragg, Kaufman and Stewart: after one pass w' = w - V h1 the norm follows from
// ||w'||^2 = ||w||^2 - ||h1||^2 (h1 holds V^T w, its entry j+1 holds ||w||^2).  If
// ||w'|| >= eta ||w|| the pass was enough: redo = 0, hn2 = ||w'||^2, inv = 1/||w'||
// (w' is normalised in the same sweep) and h2 = 0.  Otherwise redo = 1 and the
// second pass runs (inv = 1: the normalisation comes after it).  One thread.
__global__ void orth_decide_kernel(int j, double* __restrict__ h1, double* __restrict__ h2, double eta2,
                                   int* __restrict__ redo, double* __restrict__ hn2, double* __restrict__ inv) {
  IRK_PDL_ENTRY;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double wn2 = h1[j + 1];
  double hh = 0.0;
  for (int i = 0; i <= j; ++i) hh += h1[i] * h1[i];
  const double wp2 = wn2 - hh;
  for (int i = 0; i <= j + 1; ++i) h2[i] = 0.0;
  if (wp2 >= eta2 * wn2 && wp2 > 0.0) {
    *redo = 0;
    *hn2 = wp2;
    *inv = 1.0 / sqrt(wp2);
  } else {
    *redo = 1;
    *inv = 1.0;
  }
}

// y = R^{-1} g for the J x J upper-triangular R stored column-major in H.  One thread.
__global__ void trisolve_kernel(int J, int ldh, const double* __restrict__ H, const double* __restrict__ g,
                                double* __restrict__ y) {
  IRK_PDL_ENTRY;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = J - 1; i >= 0; --i) {
    double v = g[i];
    for (int k = i + 1; k < J; ++k) v -= H[(size_t)k * ldh + i] * y[k];
    y[i] = v / H[(size_t)i * ldh + i];
  }
}

__global__ void __launch_bounds__(kThreads) sub_kernel(double* __restrict__ out, const double* __restrict__ a,
                                                       const double* __restrict__ b, size_t n) {
  IRK_PDL_ENTRY;
  for (size_t e = blockIdx.x * (size_t)kThreads + threadIdx.x; e < n; e += (size_t)gridDim.x * kThreads)
    out[e] = a[e] - b[e];
}

__global__ void __launch_bounds__(kThreads) add_kernel(double* __restrict__ out, const double* __restrict__ a,
                                                       const double* __restrict__ b, size_t n) {
  IRK_PDL_ENTRY;
  for (size_t e = blockIdx.x * (size_t)kThreads + threadIdx.x; e < n; e += (size_t)gridDim.x * kThreads)
    out[e] = a[e] + b[e];
}

__global__ void sqrt_scalar_kernel(const double* __restrict__ in, double* __restrict__ out) {
  IRK_PDL_ENTRY;
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const double v = *in;
    *out = (v < 0.0) ? 0.0 : sqrt(v);  // NaN stays NaN
  }
}

__global__ void init_g_kernel(double* __restrict__ g, int m1, const double* __restrict__ beta) {
  IRK_PDL_ENTRY;
  for (int i = threadIdx.x; i < m1; i += blockDim.x) g[i] = (i == 0) ? *beta : 0.0;
}

// Conjugate-gradient pieces with scalars kept on the device.
__global__ void cg_alpha_kernel(const double* __restrict__ rz, const double* __restrict__ pq,
                                double* __restrict__ alpha) {
  IRK_PDL_ENTRY;
  if (threadIdx.x == 0 && blockIdx.x == 0) *alpha = (*pq != 0.0) ? *rz / *pq : 0.0;
}
__global__ void cg_beta_kernel(const double* __restrict__ rz_new, double* __restrict__ rz_old,
                               double* __restrict__ beta) {
  IRK_PDL_ENTRY;
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *beta = (*rz_old != 0.0) ? *rz_new / *rz_old : 0.0;
    *rz_old = *rz_new;
  }
}
// x += alpha p, r -= alpha q
__global__ void __launch_bounds__(kThreads) cg_update_xr_kernel(double* __restrict__ x, double* __restrict__ r,
                                                                const double* __restrict__ p,
                                                                const double* __restrict__ q,
                                                                const double* __restrict__ alpha, size_t n) {
  IRK_PDL_ENTRY;
  const double a = *alpha;
  for (size_t e = blockIdx.x * (size_t)kThreads + threadIdx.x; e < n; e += (size_t)gridDim.x * kThreads) {
    x[e] = fma(a, p[e], x[e]);
    r[e] = fma(-a, q[e], r[e]);
  }
}
// p = z + beta p
__global__ void __launch_bounds__(kThreads) cg_update_p_kernel(double* __restrict__ p, const double* __restrict__ z,
                                                               const double* __restrict__ beta, size_t n) {
  IRK_PDL_ENTRY;
  const double b = *beta;
  for (size_t e = blockIdx.x * (size_t)kThreads + threadIdx.x; e < n; e += (size_t)gridDim.x * kThreads)
    p[e] = fma(b, p[e], z[e]);
}

int grid_for(size_t n) {
  size_t b = (n + kThreads - 1) / kThreads;
  if (b > (size_t)kPartialBlocks) b = kPartialBlocks;
  return b < 1 ? 1 : (int)b;
}
}  // namespace

int krylov_partial_blocks() { return kPartialBlocks; }
int krylov_axpy_dot_max() { return kAxpyDotMax; }

void launch_multidot(cudaStream_t st, const double* V, size_t ld, int count, const double* w, size_t n,
                     double* partial, const int* run_if) {
  dim3 g(kPartialBlocks, (count + kGroup - 1) / kGroup);
  launch_k(multidot_kernel, g, kThreads, 0, st, V, ld, count, w, n, partial, run_if);
}
void launch_reduce_partials(cudaStream_t st, const double* partial, int count, double* out, const int* run_if) {
  launch_k(reduce_partials_kernel, count, kThreads, 0, st, partial, kPartialBlocks, out, run_if);
}
void launch_multi_axpy(cudaStream_t st, double* w, const double* V, size_t ld, int count, const double* coef,
                       double sign, size_t n, const double* scale, const int* run_if) {
  launch_k(multi_axpy_kernel, grid_for(n), kThreads, 0, st, w, V, ld, count, coef, sign, n, scale, run_if);
}
void launch_axpy_norm(cudaStream_t st, double* w, const double* V, size_t ld, int count, const double* coef,
                      size_t n, double* partial) {
#define IRK_AXPY_NORM(K, U) \
  case K: launch_k(axpy_norm_k_kernel<K, U>, kPartialBlocks, kThreads, 0, st, w, V, ld, coef, n, partial); return;
  switch (count) {
    IRK_AXPY_NORM(1, 1) IRK_AXPY_NORM(2, 1) IRK_AXPY_NORM(3, 1) IRK_AXPY_NORM(4, 2) IRK_AXPY_NORM(5, 2)
    IRK_AXPY_NORM(6, 2) IRK_AXPY_NORM(7, 2) IRK_AXPY_NORM(8, 2) IRK_AXPY_NORM(9, 2) IRK_AXPY_NORM(10, 2)
    IRK_AXPY_NORM(11, 2) IRK_AXPY_NORM(12, 2) IRK_AXPY_NORM(13, 2) IRK_AXPY_NORM(14, 2) IRK_AXPY_NORM(15, 2)
    IRK_AXPY_NORM(16, 2)
    default: launch_k(axpy_norm_kernel, kPartialBlocks, kThreads, 0, st, w, V, ld, count, coef, n, partial);
  }
#undef IRK_AXPY_NORM
}
bool launch_axpy_dot(cudaStream_t st, double* w, const double* V, size_t ld, int count, const double* coef, size_t n,
                     double* partial) {
#define IRK_AXPY_DOT(K) \
  case K: launch_k(axpy_dot_kernel<K>, kPartialBlocks, kThreads, 0, st, w, V, ld, coef, n, partial); return true;
  switch (count) {
    IRK_AXPY_DOT(1) IRK_AXPY_DOT(2) IRK_AXPY_DOT(3) IRK_AXPY_DOT(4) IRK_AXPY_DOT(5) IRK_AXPY_DOT(6)
    IRK_AXPY_DOT(7) IRK_AXPY_DOT(8) IRK_AXPY_DOT(9) IRK_AXPY_DOT(10) IRK_AXPY_DOT(11) IRK_AXPY_DOT(12)
    IRK_AXPY_DOT(13) IRK_AXPY_DOT(14) IRK_AXPY_DOT(15) IRK_AXPY_DOT(16)
    default: return false;
  }
#undef IRK_AXPY_DOT
}
void launch_scale(cudaStream_t st, double* dst, const double* src, const double* denom, size_t n, const int* run_if) {
  launch_k(scale_kernel, grid_for(n), kThreads, 0, st, dst, src, denom, n, run_if);
}
void launch_orth_decide(cudaStream_t st, int j, double* h1, double* h2, double eta2, int* redo, double* hn2,
                        double* inv) {
  launch_k(orth_decide_kernel, 1, 32, 0, st, j, h1, h2, eta2, redo, hn2, inv);
}
void launch_givens(cudaStream_t st, int j, int ldh, double* H, double* cs, double* sn, double* g, const double* h1,
                   const double* h2, const double* hn2, double* hn_out, const double* r0, double* rel_out, int pythag,
                   double* inv_out) {
  launch_k(givens_kernel, 1, 32, 0, st, j, ldh, H, cs, sn, g, h1, h2, hn2, hn_out, r0, rel_out, pythag, inv_out);
}
void launch_trisolve(cudaStream_t st, int J, int ldh, const double* H, const double* g, double* y) {
  launch_k(trisolve_kernel, 1, 32, 0, st, J, ldh, H, g, y);
}
void launch_sub(cudaStream_t st, double* out, const double* a, const double* b, size_t n) {
  launch_k(sub_kernel, grid_for(n), kThreads, 0, st, out, a, b, n);
}
void launch_cg_alpha(cudaStream_t st, const double* rz, const double* pq, double* alpha) {
  launch_k(cg_alpha_kernel, 1, 32, 0, st, rz, pq, alpha);
}
void launch_cg_beta(cudaStream_t st, const double* rz_new, double* rz_old, double* beta) {
  launch_k(cg_beta_kernel, 1, 32, 0, st, rz_new, rz_old, beta);
}
void launch_cg_update_xr(cudaStream_t st, double* x, double* r, const double* p, const double* q, const double* alpha,
                         size_t n) {
  launch_k(cg_update_xr_kernel, grid_for(n), kThreads, 0, st, x, r, p, q, alpha, n);
}
void launch_cg_update_p(cudaStream_t st, double* p, const double* z, const double* beta, size_t n) {
  launch_k(cg_update_p_kernel, grid_for(n), kThreads, 0, st, p, z, beta, n);
}
void launch_add(cudaStream_t st, double* out, const double* a, const double* b, size_t n) {
  launch_k(add_kernel, grid_for(n), kThreads, 0, st, out, a, b, n);
}
void launch_sqrt_scalar(cudaStream_t st, const double* in, double* out) { launch_k(sqrt_scalar_kernel, 1, 32, 0, st, in, out); }
void launch_init_g(cudaStream_t st, double* g, int m1, const double* beta) { launch_k(init_g_kernel, 1, 128, 0, st, g, m1, beta); }

}  // namespace irk
