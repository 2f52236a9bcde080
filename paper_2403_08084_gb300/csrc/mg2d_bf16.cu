// Instantiation of the 2D and 3D multigrid kernels for vectors stored as __nv_bfloat16.
#include "mg2d.cuh"
#include "mg3d.cuh"

namespace irk {
template struct MG2<__nv_bfloat16, float>;
template struct MG3<__nv_bfloat16, float>;
}  // namespace irk
