// The stencil kernels instantiated for FP32 storage and arithmetic.
#include "stencil_impl.cuh"

namespace qcd {

int dispatch_f32(const StencilCall &sc, const StencilArgs &A, dim3 grid, dim3 block, cudaStream_t s, int v)
{
    return dispatch<QCD_F32>(sc, A, grid, block, s, v);
}

int dispatch_f32_rg(const StencilCall &sc, const StencilArgs &A, int bx, cudaStream_t s, int v)
{
    return dispatch_rg<QCD_F32>(sc, A, bx, s, v);
}

}  // namespace qcd
