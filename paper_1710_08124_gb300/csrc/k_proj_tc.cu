// Tensor-core (tcgen05) projection GEMM with the fused selection epilogue.
#include "epll_internal.cuh"

namespace epll {

epll_status launch_select_bf16(epll_gmm *g, const float *xhat, int H, int W, const int *anchors,
                               int n, float tau, cudaStream_t st)
{
    (void)g; (void)xhat; (void)H; (void)W; (void)anchors; (void)n; (void)tau; (void)st;
    set_error("BF16 selection not built");
    return EPLL_EUNSUPPORTED;
}

}  // namespace epll
