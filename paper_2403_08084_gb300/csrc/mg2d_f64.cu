// Instantiation of the multigrid kernels for vectors stored as double.
#include "mg2d.cuh"

namespace irk {
template struct MG2<double, double>;
}  // namespace irk
