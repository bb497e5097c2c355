// Stencil residual kernels (k_stencil.cuh) for double level vectors.
#include "k_stencil.cuh"

namespace nmg {
template bool launch_stencil_residual<double, false>(const Band2D<double>&, int, const double*, const double*,
                                                     double*, double*, const int*, int, int, cudaStream_t, int*);
template bool launch_stencil_residual<double, true>(const Band2D<double>&, int, const double*, const double*,
                                                    double*, double*, const int*, int, int, cudaStream_t, int*);
template int stencil_strip_parts<double>(const Band2D<double>&);
}  // namespace nmg
