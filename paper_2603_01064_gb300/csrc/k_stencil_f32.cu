// Stencil residual kernels (k_stencil.cuh) for float level vectors.
#include "k_stencil.cuh"

namespace nmg {
template bool launch_stencil_residual<float, false>(const Band2D<float>&, int, const float*, const float*,
                                                    float*, double*, const int*, int, int, cudaStream_t, int*);
template bool launch_stencil_residual<float, true>(const Band2D<float>&, int, const float*, const float*,
                                                   float*, double*, const int*, int, int, cudaStream_t, int*);
template int stencil_strip_parts<float>(const Band2D<float>&);
}  // namespace nmg
