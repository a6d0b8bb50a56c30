// The stencil kernels instantiated for FP64 storage and arithmetic.
#include "stencil_impl.cuh"

namespace qcd {

int dispatch_f64(const StencilCall &sc, const StencilArgs &A, dim3 grid, dim3 block, cudaStream_t s, int v)
{
    return dispatch<QCD_F64>(sc, A, grid, block, s, v);
}

}  // namespace qcd
