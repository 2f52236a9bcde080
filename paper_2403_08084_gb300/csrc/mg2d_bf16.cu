// Instantiation of the multigrid kernels for vectors stored as __nv_bfloat16.
#include "mg2d.cuh"

namespace irk {
template struct MG2<__nv_bfloat16, float>;
}  // namespace irk
