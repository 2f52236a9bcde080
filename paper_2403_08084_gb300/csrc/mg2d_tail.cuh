// The small-level tail of a 2D block V(2, 2) cycle (Sec. 3.1: the multigrid approximation of a diagonal
// block B = M + sigma K) in one persistent, cooperatively launched kernel.
//
// On the levels below kMgLargeNx nodes per axis each fused leg (mg2d_legs.cuh) and the coarsest solve
// is a launch of a few microseconds whose cost is mostly latency; run as separate kernels they are seven
// or more dependent launches per V-cycle.  Here every block of one resident grid walks the same
// sequence of phases,
//
//   down legs on the tail levels (finest first), coarsest dense solve, up legs (coarsest first),
//
// processing the tiles of a phase in a grid-stride loop, with a grid-wide barrier between phases.
// The tiles are those of the separate kernels (16 x 16 fine nodes per down-leg tile on levels of at
// least kLegMediumNx nodes per axis, 8 x 8 below) and the coarsest solve uses the coarse kernel's
// summation order, so the results are bitwise those of the separate launches.
//
// Every barrier wait is bounded (TailArgs::spin SM clock cycles).  A block whose wait runs out sets the
// error flag and returns; the blocks still running then run out at their next barrier, so the kernel
// always ends.  The host reads the flag after the call, reports IRK_ECUDA and clears the barrier state.
// The launch is cooperative, which guarantees that all blocks are resident at once.
//
// Measured on GB300 (1024^2 and 2048^2 workloads, FP64 and FP32 cycles): 52 / 38 us per FP64 / FP32
// tail against about 36 / 28 us for the seven separate launches replayed in a CUDA graph, so the
// library runs this kernel only when asked to (environment IRK_TAIL=1).
#pragma once

#include "mg2d_legs.cuh"

namespace irk {

constexpr int kTailThreads = 256;

template <typename T, typename C, int S>
struct TailArgs {
  int levels;  // leg levels, finest first
  int nx[kTailMaxLevels];
  BlockRelax<C, S, true> relax[kTailMaxLevels];
  T* b[kTailMaxLevels];   // b[0]: the input right-hand side; b[l > 0]: written by the down leg of l - 1
  T* xa[kTailMaxLevels];  // down-leg iterates
  T* xb[kTailMaxLevels];  // up-leg results; xb[0] is the tail's output
  int nxc, nint;          // coarsest level
  const C* binv;          // S dense inverses, nint x nint, row-major
  T* bc;                  // coarsest right-hand side (written by the last down leg)
  T* xc;                  // coarsest solution
  unsigned* bar;          // barrier state: arrivals, generation (both zero between launches)
  int* err;               // set to 1 when a barrier wait ran out
  long long spin;         // barrier wait limit in SM clock cycles
};

// Grid-wide barrier with a bounded wait; false when this block's wait ran out (the error flag is set).
__device__ __forceinline__ bool tail_grid_sync(unsigned* bar, int* err, long long spin) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {  // last to arrive: reset the count, open the barrier
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (clock64() - t0 > spin) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// v[l] for a runtime level l, read with constant offsets (no local-memory copy of the argument arrays).
template <typename X>
__device__ __forceinline__ X pick(const X (&v)[kTailMaxLevels], int l) {
  static_assert(kTailMaxLevels == 8, "pick() lists every level");
  switch (l) {
    case 0: return v[0];
    case 1: return v[1];
    case 2: return v[2];
    case 3: return v[3];
    case 4: return v[4];
    case 5: return v[5];
    case 6: return v[6];
    default: return v[7];
  }
}

template <typename T, typename C, int S>
__global__ void __launch_bounds__(kTailThreads) tail_cycle_kernel(TailArgs<T, C, S> a) {
  using R = BlockRelax<C, S, true>;
  extern __shared__ unsigned char tail_smem[];
  const int G = gridDim.x;
  // down legs: x_l = J(J(0; b_l)), b_{l+1} = P^T (b_l - B x_l)
  for (int l = 0; l < a.levels; ++l) {
    const int nxf = pick(a.nx, l), m = nxf - 2, nxc = (nxf - 1) / 2 + 1;
    const R relax = pick(a.relax, l);
    T* bl = pick(a.b, l);
    T* xl = pick(a.xa, l);
    T* bc = (l + 1 < a.levels) ? pick(a.b, l + 1) : a.bc;
    if (nxf >= kLegMediumNx) {
      const int tx = (m + 15) / 16;
      for (int t = blockIdx.x; t < tx * tx; t += G) {
        down_leg_tile<T, C, S, 8, 8, kTailThreads, R>(t % tx, t / tx, nxf, relax, bl, xl, nxc, bc, tail_smem);
        __syncthreads();
      }
    } else {
      const int tx = (m + 7) / 8;
      for (int t = blockIdx.x; t < tx * tx; t += G) {
        down_leg_tile<T, C, S, 4, 4, kTailThreads, R>(t % tx, t / tx, nxf, relax, bl, xl, nxc, bc, tail_smem);
        __syncthreads();
      }
    }
    if (!tail_grid_sync(a.bar, a.err, a.spin)) return;
  }
  // coarsest level: x_c = B_c^{-1} b_c, one row per warp (the order of coarse_solve_kernel)
  {
    C* bs = reinterpret_cast<C*>(tail_smem);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * (kTailThreads / 32) + warp, nw = G * (kTailThreads / 32);
    const int nint = a.nint;
    for (int i = 0; i < S; ++i) {
      __syncthreads();
      for (int c = threadIdx.x; c < nint; c += kTailThreads) bs[c] = ld<C>(a.bc + (size_t)coarse_node(c, a.nxc) * S + i);
      __syncthreads();
      const C* Bi = a.binv + (size_t)i * nint * nint;
      for (int r = gw; r < nint; r += nw) {
        const C* row = Bi + (size_t)r * nint;
        C acc = 0;
        for (int c0 = 0; c0 < nint; c0 += 32 * kCoarseChunk) {
          C p0 = 0, p1 = 0, p2 = 0, p3 = 0;
#pragma unroll
          for (int k = 0; k < kCoarseChunk; k += 4) {
            const int c = c0 + lane + 32 * k;
            if (c < nint) p0 += row[c] * bs[c];
            if (c + 32 < nint) p1 += row[c + 32] * bs[c + 32];
            if (c + 64 < nint) p2 += row[c + 64] * bs[c + 64];
            if (c + 96 < nint) p3 += row[c + 96] * bs[c + 96];
          }
          acc += (p0 + p1) + (p2 + p3);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) st(a.xc + (size_t)coarse_node(r, a.nxc) * S + i, acc);
      }
    }
  }
  if (!tail_grid_sync(a.bar, a.err, a.spin)) return;
  // up legs: xb_l = J(J(xa_l + P e; b_l)), e the next coarser level's result
  for (int l = a.levels - 1; l >= 0; --l) {
    const int nxf = pick(a.nx, l), m = nxf - 2, nxc = (nxf - 1) / 2 + 1;
    const R relax = pick(a.relax, l);
    const T* xin = pick(a.xa, l);
    const T* bl = pick(a.b, l);
    T* xo = pick(a.xb, l);
    const T* ec = (l + 1 < a.levels) ? pick(a.xb, l + 1) : a.xc;
    if (nxf >= kLegMediumNx) {
      const int tx = (m + 15) / 16;
      for (int t = blockIdx.x; t < tx * tx; t += G) {
        up_leg_tile<T, C, S, 16, 16, kTailThreads, R>(t % tx, t / tx, nxf, relax, xin, bl, nxc, ec, xo, tail_smem);
        __syncthreads();
      }
    } else {
      const int tx = (m + 7) / 8;
      for (int t = blockIdx.x; t < tx * tx; t += G) {
        up_leg_tile<T, C, S, 8, 8, kTailThreads, R>(t % tx, t / tx, nxf, relax, xin, bl, nxc, ec, xo, tail_smem);
        __syncthreads();
      }
    }
    if (l > 0 && !tail_grid_sync(a.bar, a.err, a.spin)) return;
  }
}

// Shared memory of the tail kernel: the largest phase (leg halos of the tile sizes present, or the
// coarse right-hand side).
template <typename C, int S>
size_t tail_smem_bytes(const TailSpec<C>& sp) {
  bool medium = false, small = false;
  for (int l = 0; l < sp.levels; ++l) (sp.nx[l] >= kLegMediumNx ? medium : small) = true;
  size_t b = sizeof(C) * (size_t)(sp.nxc - 2) * (sp.nxc - 2);
  auto mx = [&](size_t v) { b = v > b ? v : b; };
  if (medium) {
    mx(sizeof(C) * S * (size_t)(21 * 21 + 19 * 19 + 17 * 17));  // down leg, 8 x 8 coarse nodes
    mx(sizeof(C) * S * (size_t)(20 * 20 + 18 * 18));            // up leg, 16 x 16 fine nodes
  }
  if (small) {
    mx(sizeof(C) * S * (size_t)(13 * 13 + 11 * 11 + 9 * 9));
    mx(sizeof(C) * S * (size_t)(12 * 12 + 10 * 10));
  }
  return b;
}

inline int device_sm_count() {
  static thread_local int dev_cached = -1, n_cached = 1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != dev_cached) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    n_cached = n > 0 ? n : 1;
    dev_cached = dev;
  }
  return n_cached;
}

template <typename T, typename C, int S>
cudaError_t launch_tail_cycle(cudaStream_t st, const TailSpec<C>& sp, int dstride) {
  TailArgs<T, C, S> a{};
  a.levels = sp.levels;
  int tiles = 1;
  for (int l = 0; l < sp.levels; ++l) {
    a.nx[l] = sp.nx[l];
    a.relax[l] = BlockRelax<C, S, true>{sp.rec[l], sp.rstride[l], nullptr, C(0), {}, sp.dinv[l], dstride};
    a.b[l] = static_cast<T*>(sp.b[l]);
    a.xa[l] = static_cast<T*>(sp.xa[l]);
    a.xb[l] = static_cast<T*>(sp.xb[l]);
    const int m = sp.nx[l] - 2, edge = sp.nx[l] >= kLegMediumNx ? 16 : 8;
    const int t = ((m + edge - 1) / edge) * ((m + edge - 1) / edge);
    tiles = t > tiles ? t : tiles;
  }
  a.nxc = sp.nxc;
  a.nint = (sp.nxc - 2) * (sp.nxc - 2);
  a.binv = sp.binv;
  a.bc = static_cast<T*>(sp.bc);
  a.xc = static_cast<T*>(sp.xc);
  a.bar = sp.bar;
  a.err = sp.err;
  a.spin = sp.spin_cycles;
  const int coarse_blocks = (a.nint + kTailThreads / 32 - 1) / (kTailThreads / 32);
  tiles = coarse_blocks > tiles ? coarse_blocks : tiles;
  auto kern = tail_cycle_kernel<T, C, S>;
  const size_t smem = tail_smem_bytes<C, S>(sp);
  if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // resident blocks per SM for this shared memory size, queried once per instantiation and size
  static thread_local size_t q_smem = 0;
  static thread_local int q_blocks = 0;
  if (q_smem != smem || q_blocks == 0) {
    int nb = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kTailThreads, smem);
    if (e != cudaSuccess) return e;
    q_smem = smem;
    q_blocks = nb > 0 ? nb : 1;
  }
  int grid = q_blocks * device_sm_count();
  if (grid > tiles) grid = tiles;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kTailThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <typename T, typename C>
cudaError_t MG2<T, C>::tail_cycle(int S, cudaStream_t st, const TailSpec<C>& sp, int dstride) {
  switch (S) {
    case 1: return launch_tail_cycle<T, C, 1>(st, sp, dstride);
    case 2: return launch_tail_cycle<T, C, 2>(st, sp, dstride);
    case 3: return launch_tail_cycle<T, C, 3>(st, sp, dstride);
    case 4: return launch_tail_cycle<T, C, 4>(st, sp, dstride);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace irk
