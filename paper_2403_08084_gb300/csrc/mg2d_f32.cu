// Instantiation of the 2D and 3D multigrid kernels for vectors stored as float.
#include "mg2d.cuh"
#include "mg3d.cuh"

namespace irk {
template struct MG2<float, float>;
template struct MG3<float, float>;
}  // namespace irk
