// The stencil kernels instantiated for FP16 storage and arithmetic.
#include "stencil_impl.cuh"

namespace qcd {

int dispatch_f16(const StencilCall &sc, const StencilArgs &A, dim3 grid, dim3 block, cudaStream_t s, int v)
{
    return dispatch<QCD_F16>(sc, A, grid, block, s, v);
}

}  // namespace qcd
