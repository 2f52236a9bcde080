// Instantiation of the multigrid kernels for vectors stored as float.
#include "mg2d.cuh"

namespace irk {
template struct MG2<float, float>;
}  // namespace irk
