// Host-side construction of the multigrid hierarchy (plain C++, no CUDA).
#pragma once

#include <vector>

namespace irk {

// Level-0 stiffness stencil records {D, E, N, NE, NW} per node of the full
// (N+1)^2 grid, assembled cell by cell from the bilinear element matrix with
// per-cell diffusivity (kappa == nullptr: kappa = 1).
void stiffness_records_2d(int N, const double* kappa, std::vector<double>& cf);

// Galerkin coarse stencil P^T K_f P (P = bilinear interpolation on the full
// grid) from fine records with Nf cells per axis to Nf/2.
void galerkin_coarsen_2d(int Nf, const std::vector<double>& cff, std::vector<double>& cfc);

// Stencil records of B_i = M + sigma_i K for each stage, stage-major
// (S blocks of (N+1)^2 records); M is the Q1 mass stencil hm [1 4 1; 4 16 4; 1 4 1].
void block_records_2d(int N, const std::vector<double>& cf, double hm, const double* sigma, int S,
                      std::vector<double>& rec);

// omega / diag(M + sigma_i K) at interior nodes (0 on the boundary), node-major
// with S values per node; hm = h^2/36.
void jacobi_inverse_diag_2d(int N, const std::vector<double>& cf, double hm, const double* sigma, int S,
                            double omega, std::vector<double>& dinv);

// Weighted Jacobi for one block B after its first sweep (Sec. 3.1's smoother, rewritten): with
// d = omega / diag(B) and x1 = d b the sweep from a zero guess,
//   x + d (b - B x) = x1 + sum_k c'_k x_k,   c'_centre = 1 - d B_pp,   c'_k = -d B_pk (k != p),
// nine products per node instead of nine plus two.  rec: B's records {D, E, N, NE, NW} per node (node-major,
// (N+1)^2 records); dinv: d per node; out: nine planes of (N+1)^2 values, neighbour order centre, E, W, N, S,
// NE, SW, NW, SE; zero at boundary nodes and for couplings to boundary nodes.
void scaled_jacobi_records_2d(int N, const double* rec, const double* dinv, double* out);

// Interior node ids of an N-cell grid (x fastest) and the dense inverse of
// M + sigma K restricted to them (row-major, nint x nint).  Returns false if the
// matrix is singular to working precision.
void interior_nodes_2d(int N, std::vector<int>& map);
bool dense_block_inverse_2d(int N, const std::vector<double>& cf, double hm, double sigma,
                            const std::vector<int>& map, std::vector<double>& inv);

// Monolithic multigrid (stage-coupled point-block Jacobi): omega (M[p,p] I + dt K[p,p] A)^{-1} per
// node (row-major s x s, 0 on the boundary), node-major.  Returns false if a block is singular.
bool mmg_block_inverses_2d(int N, const std::vector<double>& cf, double hm, const double* A, int s, double dt,
                           double omega, std::vector<double>& dblk);

// Dense inverse of the coupled coarsest system I (x) M + dt A (x) K on the interior nodes, unknowns
// interleaved (row q s + i: stage i of interior node q, x fastest); banded LU with partial pivoting.
// Returns false if the matrix is singular to working precision.
bool mmg_coarse_inverse_2d(int N, const std::vector<double>& cf, double hm, const double* A, int s, double dt,
                           std::vector<double>& inv);

// 3D, kappa = 1: values of the Q1 mass and stiffness 27-point stencils on a grid
// of spacing h by offset class (number of nonzero offset coordinates 0..3).
void q1_classes_3d(double h, double mass[4], double stiff[4]);

// Interior node ids of an N^3-cell grid and the dense inverse of M + sigma K
// (constant-coefficient classes) restricted to them.
void interior_nodes_3d(int N, std::vector<int>& map);
bool dense_block_inverse_3d(int N, const double mass[4], const double stiff[4], double sigma,
                            const std::vector<int>& map, std::vector<double>& inv);

}  // namespace irk
