// Test infrastructure: C entry points over the library's host-side hierarchy builders
// (paper_2403_08084_gb300/csrc/hierarchy.cpp), compiled by tests/test_host_hierarchy.py with the
// system C++ compiler so that the CPU tests can compare what they build with the oracle's
// assembled matrices.  Not part of the library.
#include <cstring>
#include <vector>

#include "hierarchy.h"

namespace {
void copy_out(const std::vector<double>& v, double* out) { std::memcpy(out, v.data(), v.size() * sizeof(double)); }
std::vector<double> records_in(int N, const double* cf) {
  const size_t nn = (size_t)(N + 1) * (N + 1);
  return std::vector<double>(cf, cf + nn * 5);
}
}  // namespace

extern "C" {

void shim_stiffness_records(int N, const double* kappa, double* out) {
  std::vector<double> cf;
  irk::stiffness_records_2d(N, kappa, cf);
  copy_out(cf, out);
}

void shim_galerkin_coarsen(int Nf, const double* cff, double* out) {
  std::vector<double> cfc;
  irk::galerkin_coarsen_2d(Nf, records_in(Nf, cff), cfc);
  copy_out(cfc, out);
}

void shim_block_records(int N, const double* cf, double hm, const double* sigma, int S, double* out) {
  std::vector<double> rec;
  irk::block_records_2d(N, records_in(N, cf), hm, sigma, S, rec);
  copy_out(rec, out);
}

void shim_jacobi_inverse_diag(int N, const double* cf, double hm, const double* sigma, int S, double omega,
                              double* out) {
  std::vector<double> dinv;
  irk::jacobi_inverse_diag_2d(N, records_in(N, cf), hm, sigma, S, omega, dinv);
  copy_out(dinv, out);
}

void shim_scaled_jacobi_records(int N, const double* rec, const double* dinv, double* out) {
  irk::scaled_jacobi_records_2d(N, rec, dinv, out);
}

int shim_dense_block_inverse(int N, const double* cf, double hm, double sigma, double* out) {
  std::vector<int> map;
  irk::interior_nodes_2d(N, map);
  std::vector<double> inv;
  if (!irk::dense_block_inverse_2d(N, records_in(N, cf), hm, sigma, map, inv)) return 0;
  copy_out(inv, out);
  return 1;
}

int shim_mmg_block_inverses(int N, const double* cf, double hm, const double* A, int s, double dt, double omega,
                            double* out) {
  std::vector<double> dblk;
  if (!irk::mmg_block_inverses_2d(N, records_in(N, cf), hm, A, s, dt, omega, dblk)) return 0;
  copy_out(dblk, out);
  return 1;
}

int shim_mmg_coarse_inverse(int N, const double* cf, double hm, const double* A, int s, double dt, double* out) {
  std::vector<double> inv;
  if (!irk::mmg_coarse_inverse_2d(N, records_in(N, cf), hm, A, s, dt, inv)) return 0;
  copy_out(inv, out);
  return 1;
}

void shim_q1_classes_3d(double h, double* mass, double* stiff) { irk::q1_classes_3d(h, mass, stiff); }

int shim_dense_block_inverse_3d(int N, const double* mass, const double* stiff, double sigma, double* out) {
  std::vector<int> map;
  irk::interior_nodes_3d(N, map);
  std::vector<double> inv;
  if (!irk::dense_block_inverse_3d(N, mass, stiff, sigma, map, inv)) return 0;
  copy_out(inv, out);
  return 1;
}

}  // extern "C"
