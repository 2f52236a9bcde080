// Instantiation of the 2D and 3D multigrid kernels for vectors stored as double.
#include "mg2d.cuh"
#include "mg3d.cuh"

namespace irk {
template struct MG2<double, double>;
template struct MG3<double, double>;
}  // namespace irk
