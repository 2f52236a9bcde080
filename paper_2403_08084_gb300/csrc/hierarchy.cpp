// Host-side construction of the multigrid hierarchy: level stencils,
// Galerkin coarse operators, Jacobi diagonals and the exact coarsest-level
// inverse (Sec. 3.1: each diagonal block M + dt a_ii K is approximated by one
// multigrid V-cycle).
#include "hierarchy.h"

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <thread>
#include <utility>

namespace irk {

namespace {
enum { kD = 0, kE = 1, kN = 2, kNE = 3, kNW = 4, kRec = 5 };

// K(a, b) for nodes a = (ax, ay), b = a + (dx, dy), |dx|, |dy| <= 1, from records.
inline double coupling(const std::vector<double>& cf, int nx, int ax, int ay, int dx, int dy) {
  const size_t a = (size_t)ax + (size_t)nx * ay;
  auto R = [&](size_t node, int k) { return cf[node * kRec + k]; };
  if (dx == 0 && dy == 0) return R(a, kD);
  if (dx == 1 && dy == 0) return R(a, kE);
  if (dx == -1 && dy == 0) return R(a - 1, kE);
  if (dx == 0 && dy == 1) return R(a, kN);
  if (dx == 0 && dy == -1) return R(a - nx, kN);
  if (dx == 1 && dy == 1) return R(a, kNE);
  if (dx == -1 && dy == -1) return R(a - nx - 1, kNE);
  if (dx == -1 && dy == 1) return R(a, kNW);
  return R(a + 1 - nx, kNW);  // (1, -1)
}

// Record slot holding K(I, J) for J = I + (dx, dy) if (dx, dy) is a forward
// direction or the node itself; -1 for the four backward directions.
inline int forward_slot(int dx, int dy) {
  if (dx == 0 && dy == 0) return kD;
  if (dx == 1 && dy == 0) return kE;
  if (dx == 0 && dy == 1) return kN;
  if (dx == 1 && dy == 1) return kNE;
  if (dx == -1 && dy == 1) return kNW;
  return -1;
}

// Coarse parents of fine index i (1D linear interpolation): returns count.
inline int parents(int i, int* idx, double* w) {
  if ((i & 1) == 0) {
    idx[0] = i / 2;
    w[0] = 1.0;
    return 1;
  }
  idx[0] = (i - 1) / 2;
  idx[1] = (i + 1) / 2;
  w[0] = w[1] = 0.5;
  return 2;
}

inline bool interior(int ix, int iy, int nx) { return ix >= 1 && iy >= 1 && ix <= nx - 2 && iy <= nx - 2; }
}  // namespace

void stiffness_records_2d(int N, const double* kappa, std::vector<double>& cf) {
  const int nx = N + 1;
  cf.assign((size_t)nx * nx * kRec, 0.0);
  for (int cy = 0; cy < N; ++cy) {
    for (int cx = 0; cx < N; ++cx) {
      const double k = kappa ? kappa[(size_t)cx + (size_t)N * cy] : 1.0;
      const size_t p0 = (size_t)cx + (size_t)nx * cy, p1 = p0 + 1, p2 = p0 + nx, p3 = p2 + 1;
      // bilinear element matrix kappa/6 [[4,-1,-1,-2],[-1,4,-2,-1],[-1,-2,4,-1],[-2,-1,-1,4]]
      for (size_t p : {p0, p1, p2, p3}) cf[p * kRec + kD] += 4.0 * k / 6.0;
      cf[p0 * kRec + kE] += -k / 6.0;   // p0 - p1
      cf[p2 * kRec + kE] += -k / 6.0;   // p2 - p3
      cf[p0 * kRec + kN] += -k / 6.0;   // p0 - p2
      cf[p1 * kRec + kN] += -k / 6.0;   // p1 - p3
      cf[p0 * kRec + kNE] += -2.0 * k / 6.0;  // p0 - p3
      cf[p1 * kRec + kNW] += -2.0 * k / 6.0;  // p1 - p2
    }
  }
}

void galerkin_coarsen_2d(int Nf, const std::vector<double>& cff, std::vector<double>& cfc) {
  const int Nc = Nf / 2, nxf = Nf + 1, nxc = Nc + 1;
  cfc.assign((size_t)nxc * nxc * kRec, 0.0);
  int pax[2], pay[2], pbx[2], pby[2];
  double wax[2], way[2], wbx[2], wby[2];
  for (int ay = 0; ay < nxf; ++ay) {
    const int nay = parents(ay, pay, way);
    for (int ax = 0; ax < nxf; ++ax) {
      const int nax = parents(ax, pax, wax);
      for (int dy = -1; dy <= 1; ++dy) {
        const int by = ay + dy;
        if (by < 0 || by >= nxf) continue;
        const int nby = parents(by, pby, wby);
        for (int dx = -1; dx <= 1; ++dx) {
          const int bx = ax + dx;
          if (bx < 0 || bx >= nxf) continue;
          const double v = coupling(cff, nxf, ax, ay, dx, dy);
          if (v == 0.0) continue;
          const int nbx = parents(bx, pbx, wbx);
          for (int ia = 0; ia < nay; ++ia)
            for (int ja = 0; ja < nax; ++ja)
              for (int ib = 0; ib < nby; ++ib)
                for (int jb = 0; jb < nbx; ++jb) {
                  const int slot = forward_slot(pbx[jb] - pax[ja], pby[ib] - pay[ia]);
                  if (slot < 0) continue;  // counted from the symmetric pair
                  const size_t I = (size_t)pax[ja] + (size_t)nxc * pay[ia];
                  cfc[I * kRec + slot] += wax[ja] * way[ia] * v * wbx[jb] * wby[ib];
                }
        }
      }
    }
  }
}

void block_records_2d(int N, const std::vector<double>& cf, double hm, const double* sigma, int S,
                      std::vector<double>& rec) {
  const size_t nn = (size_t)(N + 1) * (N + 1);
  rec.assign(nn * kRec * S, 0.0);
  const double mass[kRec] = {16.0 * hm, 4.0 * hm, 4.0 * hm, hm, hm};  // D, E, N, NE, NW
  for (int i = 0; i < S; ++i)
    for (size_t p = 0; p < nn; ++p)
      for (int k = 0; k < kRec; ++k) rec[((size_t)i * nn + p) * kRec + k] = mass[k] + sigma[i] * cf[p * kRec + k];
}

void jacobi_inverse_diag_2d(int N, const std::vector<double>& cf, double hm, const double* sigma, int S,
                            double omega, std::vector<double>& dinv) {
  const int nx = N + 1;
  dinv.assign((size_t)nx * nx * S, 0.0);
  for (int iy = 1; iy < nx - 1; ++iy)
    for (int ix = 1; ix < nx - 1; ++ix) {
      const size_t p = (size_t)ix + (size_t)nx * iy;
      for (int i = 0; i < S; ++i) dinv[p * S + i] = omega / (16.0 * hm + sigma[i] * cf[p * kRec + kD]);
    }
}

void scaled_jacobi_records_2d(int N, const double* rec, const double* dinv, double* out) {
  const int nx = N + 1;
  const size_t nn = (size_t)nx * nx;
  for (size_t q = 0; q < 9 * nn; ++q) out[q] = 0.0;
  for (int iy = 1; iy < nx - 1; ++iy)
    for (int ix = 1; ix < nx - 1; ++ix) {
      const size_t p = (size_t)ix + (size_t)nx * iy;
      const double d = dinv[p];
      auto R = [&](size_t q, int k) { return rec[q * kRec + k]; };
      // B_pk for the neighbours (dx, dy), from the symmetric records
      const int dx[9] = {0, 1, -1, 0, 0, 1, -1, -1, 1};
      const int dy[9] = {0, 0, 0, 1, -1, 1, -1, 1, -1};
      const double b[9] = {R(p, kD),          R(p, 1), R(p - 1, 1),      R(p, 2),         R(p - nx, 2),
                           R(p, 3),           R(p - nx - 1, 3),          R(p, 4),         R(p - nx + 1, 4)};
      out[p] = 1.0 - d * b[0];
      for (int k = 1; k < 9; ++k) {
        const int jx = ix + dx[k], jy = iy + dy[k];
        const bool inner = jx >= 1 && jy >= 1 && jx <= nx - 2 && jy <= nx - 2;
        out[(size_t)k * nn + p] = inner ? -d * b[k] : 0.0;
      }
    }
}

void interior_nodes_2d(int N, std::vector<int>& map) {
  const int nx = N + 1;
  map.clear();
  for (int iy = 1; iy < nx - 1; ++iy)
    for (int ix = 1; ix < nx - 1; ++ix) map.push_back(ix + nx * iy);
}

bool mmg_block_inverses_2d(int N, const std::vector<double>& cf, double hm, const double* A, int s, double dt,
                           double omega, std::vector<double>& dblk) {
  const int nx = N + 1;
  dblk.assign((size_t)nx * nx * s * s, 0.0);
  std::vector<double> D((size_t)s * s), W((size_t)s * 2 * s);
  for (int iy = 1; iy < nx - 1; ++iy)
    for (int ix = 1; ix < nx - 1; ++ix) {
      const size_t p = (size_t)ix + (size_t)nx * iy;
      const double m = 16.0 * hm, k = cf[p * kRec + kD];
      // Gauss-Jordan with partial pivoting on [D | I], D = m I + dt k A
      for (int i = 0; i < s; ++i)
        for (int j = 0; j < 2 * s; ++j)
          W[(size_t)i * 2 * s + j] = (j < s) ? (i == j ? m : 0.0) + dt * k * A[i * s + j] : (j - s == i ? 1.0 : 0.0);
      for (int c = 0; c < s; ++c) {
        int piv = c;
        for (int r = c + 1; r < s; ++r)
          if (std::fabs(W[(size_t)r * 2 * s + c]) > std::fabs(W[(size_t)piv * 2 * s + c])) piv = r;
        const double d = W[(size_t)piv * 2 * s + c];
        if (!(std::fabs(d) > 0.0) || !std::isfinite(d)) return false;
        if (piv != c)
          for (int j = 0; j < 2 * s; ++j) std::swap(W[(size_t)c * 2 * s + j], W[(size_t)piv * 2 * s + j]);
        for (int j = 0; j < 2 * s; ++j) W[(size_t)c * 2 * s + j] /= d;
        for (int r = 0; r < s; ++r) {
          if (r == c) continue;
          const double f = W[(size_t)r * 2 * s + c];
          for (int j = 0; j < 2 * s; ++j) W[(size_t)r * 2 * s + j] -= f * W[(size_t)c * 2 * s + j];
        }
      }
      for (int i = 0; i < s; ++i)
        for (int j = 0; j < s; ++j) dblk[p * s * s + (size_t)i * s + j] = omega * W[(size_t)i * 2 * s + s + j];
    }
  return true;
}

bool mmg_coarse_inverse_2d(int N, const std::vector<double>& cf, double hm, const double* A, int s, double dt,
                           std::vector<double>& inv) {
  const int nx = N + 1, m = nx - 2, nint = m * m, n = s * nint;
  // assemble the interleaved system densely (its band: |row - col| <= s (m + 1) + s - 1)
  std::vector<double> F((size_t)n * n, 0.0);
  for (int iy = 1; iy < nx - 1; ++iy)
    for (int ix = 1; ix < nx - 1; ++ix) {
      const int q = (ix - 1) + m * (iy - 1);
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int jx = ix + dx, jy = iy + dy;
          if (!interior(jx, jy, nx)) continue;
          const int qc = (jx - 1) + m * (jy - 1);
          const double mv = hm * ((dx == 0 ? 4.0 : 1.0) * (dy == 0 ? 4.0 : 1.0));
          const double kv = coupling(cf, nx, ix, iy, dx, dy);
          for (int i = 0; i < s; ++i)
            for (int j = 0; j < s; ++j)
              F[(size_t)(q * s + i) * n + (qc * s + j)] = (i == j ? mv : 0.0) + dt * A[i * s + j] * kv;
        }
    }
  // Banded LU with partial pivoting in the scheme of LAPACK's band solver: the interchange at step k
  // swaps only the not yet eliminated columns, so column k of L keeps the multipliers of the rows as
  // they stood at step k and the forward solve replays interchange and elimination step by step.
  const int bl = s * (m + 1) + s - 1;  // lower bandwidth; row interchanges widen the upper one to 2 bl
  const int bu = 2 * bl;
  std::vector<int> perm(n);
  for (int k = 0; k < n; ++k) {
    const int rmax = std::min(n - 1, k + bl), cmax = std::min(n - 1, k + bu);
    int piv = k;
    for (int r = k + 1; r <= rmax; ++r)
      if (std::fabs(F[(size_t)r * n + k]) > std::fabs(F[(size_t)piv * n + k])) piv = r;
    const double d = F[(size_t)piv * n + k];
    if (!(std::fabs(d) > 0.0) || !std::isfinite(d)) return false;
    perm[k] = piv;
    if (piv != k)
      for (int c = k; c <= cmax; ++c) std::swap(F[(size_t)k * n + c], F[(size_t)piv * n + c]);
    for (int r = k + 1; r <= rmax; ++r) {
      const double f = F[(size_t)r * n + k] / d;
      F[(size_t)r * n + k] = f;
      if (f == 0.0) continue;
      for (int c = k + 1; c <= cmax; ++c) F[(size_t)r * n + c] -= f * F[(size_t)k * n + c];
    }
  }
  // columns of the inverse, spread over the host's threads
  inv.assign((size_t)n * n, 0.0);
  auto solve_columns = [&](int c0, int c1) {
    std::vector<double> y(n);
    for (int col = c0; col < c1; ++col) {
      std::fill(y.begin(), y.end(), 0.0);
      y[col] = 1.0;
      for (int k = 0; k < n; ++k) {
        if (perm[k] != k) std::swap(y[k], y[perm[k]]);
        const double yk = y[k];
        if (yk == 0.0) continue;
        const int rmax = std::min(n - 1, k + bl);
        for (int r = k + 1; r <= rmax; ++r) y[r] -= F[(size_t)r * n + k] * yk;
      }
      for (int r = n - 1; r >= 0; --r) {
        double v = y[r];
        const int cmax = std::min(n - 1, r + bu);
        for (int c = r + 1; c <= cmax; ++c) v -= F[(size_t)r * n + c] * y[c];
        y[r] = v / F[(size_t)r * n + r];
      }
      for (int r = 0; r < n; ++r) inv[(size_t)r * n + col] = y[r];
    }
  };
  const int nt = std::max(1, std::min(32, (int)std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t) pool.emplace_back(solve_columns, (int)((long long)n * t / nt), (int)((long long)n * (t + 1) / nt));
  for (auto& th : pool) th.join();
  return true;
}

bool dense_block_inverse_2d(int N, const std::vector<double>& cf, double hm, double sigma,
                            const std::vector<int>& map, std::vector<double>& inv) {
  const int nx = N + 1;
  const int n = (int)map.size();
  std::vector<int> pos((size_t)nx * nx, -1);
  for (int c = 0; c < n; ++c) pos[map[c]] = c;
  // B = M + sigma K on interior nodes, M = hm [1 4 1; 4 16 4; 1 4 1]
  std::vector<double> B((size_t)n * n, 0.0);
  for (int r = 0; r < n; ++r) {
    const int p = map[r], ix = p % nx, iy = p / nx;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int jx = ix + dx, jy = iy + dy;
        if (!interior(jx, jy, nx)) continue;
        const int c = pos[jx + nx * jy];
        const double m = hm * ((dx == 0 ? 4.0 : 1.0) * (dy == 0 ? 4.0 : 1.0));
        B[(size_t)r * n + c] = m + sigma * coupling(cf, nx, ix, iy, dx, dy);
      }
  }
  const int bw = nx - 1;  // |row - col| <= nx - 1 for the 9-point stencil in interior numbering
  if (sigma >= 0.0) {
    // M + sigma K is symmetric positive definite: banded LU without pivoting keeps the band.
    std::vector<double> F = B;
    bool ok = true;
    for (int k = 0; k < n && ok; ++k) {
      const double piv = F[(size_t)k * n + k];
      if (!(piv > 0.0) || !std::isfinite(piv)) {
        ok = false;
        break;
      }
      const int rmax = std::min(n - 1, k + bw);
      for (int r = k + 1; r <= rmax; ++r) {
        const double f = F[(size_t)r * n + k] / piv;
        if (f == 0.0) continue;
        F[(size_t)r * n + k] = f;
        for (int c = k + 1; c <= rmax; ++c) F[(size_t)r * n + c] -= f * F[(size_t)k * n + c];
      }
    }
    if (ok) {
      inv.assign((size_t)n * n, 0.0);
      std::vector<double> y(n);
      for (int col = 0; col < n; ++col) {
        std::fill(y.begin(), y.end(), 0.0);
        y[col] = 1.0;
        for (int r = col + 1; r < n; ++r) {  // L y = e_col (unit lower, band)
          double v = y[r];
          for (int c = std::max(col, r - bw); c < r; ++c) v -= F[(size_t)r * n + c] * y[c];
          y[r] = v;
        }
        for (int r = n - 1; r >= 0; --r) {  // U x = y
          double v = y[r];
          const int cmax = std::min(n - 1, r + bw);
          for (int c = r + 1; c <= cmax; ++c) v -= F[(size_t)r * n + c] * y[c];
          y[r] = v / F[(size_t)r * n + r];
        }
        for (int r = 0; r < n; ++r) inv[(size_t)r * n + col] = y[r];
      }
      return true;
    }
  }
  // General case: Gauss-Jordan elimination with partial pivoting on [B | I].
  inv.assign((size_t)n * n, 0.0);
  for (int r = 0; r < n; ++r) inv[(size_t)r * n + r] = 1.0;
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = std::fabs(B[(size_t)k * n + k]);
    for (int r = k + 1; r < n; ++r) {
      const double v = std::fabs(B[(size_t)r * n + k]);
      if (v > best) best = v, piv = r;
    }
    if (!(best > 0.0) || !std::isfinite(best)) return false;
    if (piv != k) {
      for (int c = 0; c < n; ++c) {
        std::swap(B[(size_t)k * n + c], B[(size_t)piv * n + c]);
        std::swap(inv[(size_t)k * n + c], inv[(size_t)piv * n + c]);
      }
    }
    const double d = 1.0 / B[(size_t)k * n + k];
    double* Bk = &B[(size_t)k * n];
    double* Ik = &inv[(size_t)k * n];
    for (int c = 0; c < n; ++c) Bk[c] *= d, Ik[c] *= d;
    for (int r = 0; r < n; ++r) {
      if (r == k) continue;
      const double f = B[(size_t)r * n + k];
      if (f == 0.0) continue;
      double* Br = &B[(size_t)r * n];
      double* Ir = &inv[(size_t)r * n];
      for (int c = 0; c < n; ++c) Br[c] -= f * Bk[c];
      for (int c = 0; c < n; ++c) Ir[c] -= f * Ik[c];
    }
  }
  return true;
}

void q1_classes_3d(double h, double mass[4], double stiff[4]) {
  // 1D linear elements: m(0) = 4h/6, m(1) = h/6; k(0) = 2/h, k(1) = -1/h.  The Q1 matrices are
  // M = m (x) m (x) m and K = k (x) m (x) m + m (x) k (x) m + m (x) m (x) k.
  const double m0 = 4.0 * h / 6.0, m1 = h / 6.0, k0 = 2.0 / h, k1 = -1.0 / h;
  for (int nz = 0; nz <= 3; ++nz) {
    const int z = 3 - nz;
    mass[nz] = std::pow(m1, nz) * std::pow(m0, z);
    double kv = 0.0;
    if (nz > 0) kv += nz * k1 * std::pow(m1, nz - 1) * std::pow(m0, z);
    if (z > 0) kv += z * k0 * std::pow(m1, nz) * std::pow(m0, z - 1);
    stiff[nz] = kv;
  }
}

void interior_nodes_3d(int N, std::vector<int>& map) {
  const int n = N + 1;
  map.clear();
  for (int iz = 1; iz < n - 1; ++iz)
    for (int iy = 1; iy < n - 1; ++iy)
      for (int ix = 1; ix < n - 1; ++ix) map.push_back(ix + n * (iy + n * iz));
}

bool dense_block_inverse_3d(int N, const double mass[4], const double stiff[4], double sigma,
                            const std::vector<int>& map, std::vector<double>& inv) {
  const int n = N + 1, m = n - 2;
  const int cnt = (int)map.size();
  auto idx = [&](int ix, int iy, int iz) { return (ix - 1) + m * ((iy - 1) + m * (iz - 1)); };
  std::vector<double> B((size_t)cnt * cnt, 0.0);
  for (int iz = 1; iz <= m; ++iz)
    for (int iy = 1; iy <= m; ++iy)
      for (int ix = 1; ix <= m; ++ix) {
        const int r = idx(ix, iy, iz);
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              const int jx = ix + dx, jy = iy + dy, jz = iz + dz;
              if (!interior(jx, jy, n) || jz < 1 || jz > m) continue;
              const int cls = (dx != 0) + (dy != 0) + (dz != 0);
              B[(size_t)r * cnt + idx(jx, jy, jz)] = mass[cls] + sigma * stiff[cls];
            }
      }
  // Gauss-Jordan with partial pivoting (the coarsest 3D level is small)
  inv.assign((size_t)cnt * cnt, 0.0);
  for (int r = 0; r < cnt; ++r) inv[(size_t)r * cnt + r] = 1.0;
  for (int k = 0; k < cnt; ++k) {
    int piv = k;
    double best = std::fabs(B[(size_t)k * cnt + k]);
    for (int r = k + 1; r < cnt; ++r)
      if (std::fabs(B[(size_t)r * cnt + k]) > best) best = std::fabs(B[(size_t)r * cnt + k]), piv = r;
    if (!(best > 0.0) || !std::isfinite(best)) return false;
    if (piv != k)
      for (int c = 0; c < cnt; ++c) {
        std::swap(B[(size_t)k * cnt + c], B[(size_t)piv * cnt + c]);
        std::swap(inv[(size_t)k * cnt + c], inv[(size_t)piv * cnt + c]);
      }
    const double d = 1.0 / B[(size_t)k * cnt + k];
    for (int c = 0; c < cnt; ++c) B[(size_t)k * cnt + c] *= d, inv[(size_t)k * cnt + c] *= d;
    for (int r = 0; r < cnt; ++r) {
      if (r == k) continue;
      const double f = B[(size_t)r * cnt + k];
      if (f == 0.0) continue;
      for (int c = 0; c < cnt; ++c) B[(size_t)r * cnt + c] -= f * B[(size_t)k * cnt + c];
      for (int c = 0; c < cnt; ++c) inv[(size_t)r * cnt + c] -= f * inv[(size_t)k * cnt + c];
    }
  }
  (void)map;
  return true;
}

}  // namespace irk
