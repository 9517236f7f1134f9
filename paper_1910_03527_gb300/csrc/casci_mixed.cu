// a5-a6 in mixed precision, the warp solver's float32 launch (anchored refinement).
#include "casci_dev.cuh"

namespace mbe {

template <int DPL>
static int launch_warp_mixed_t(mbe_ctx *ctx, const BatchArgs &a, int b, const MixLayout &L)
{
    const size_t smem = (size_t)L.bytes * a.warps;
    MBE_CHECK(smem <= ctx->smem_optin, MBE_EUNSUPPORTED, "casci_batch: mixed warp solver needs %zu B shared memory",
              smem);
    MBE_CU(cudaFuncSetAttribute(k_casci_warp_mixed<DPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    MBE_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_casci_warp_mixed<DPL>, a.warps * 32, smem));
    if (per_sm < 1) per_sm = 1;
    k_casci_warp_mixed<DPL><<<ctx->sm_count * per_sm, a.warps * 32, smem, ctx->stream>>>(a, b, L);
    MBE_CU(cudaGetLastError());
    ++ctx->launches;
    return MBE_OK;
}

int launch_warp_mixed_dpl(mbe_ctx *ctx, const BatchArgs &a, int b, const MixLayout &L, int dpl)
{
    switch (dpl) {
    case 1: return launch_warp_mixed_t<1>(ctx, a, b, L);
    case 2: return launch_warp_mixed_t<2>(ctx, a, b, L);
    case 4: return launch_warp_mixed_t<4>(ctx, a, b, L);
    case 8: return launch_warp_mixed_t<8>(ctx, a, b, L);
    default: return launch_warp_mixed_t<13>(ctx, a, b, L);
    }
}

}  // namespace mbe
