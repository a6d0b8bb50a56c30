// The stencil kernels instantiated for DF64 (float-pair) storage and arithmetic.
#include "stencil_impl.cuh"

namespace qcd {

int dispatch_df64(const StencilCall &sc, const StencilArgs &A, dim3 grid, dim3 block, cudaStream_t s, int v)
{
    return dispatch<QCD_DF64>(sc, A, grid, block, s, v);
}

}  // namespace qcd
