// a5-a6, the warp solver's float64 launches (all phases, or the float64 redo of
// the tuples the mixed launch flagged).
#include "casci_dev.cuh"

namespace mbe {

template <int DPL, int MODE>
static int launch_warp_mode(mbe_ctx *ctx, const BatchArgs &a, int b, const WarpLayout &L, size_t smem)
{
    MBE_CU(cudaFuncSetAttribute(k_casci_warp<DPL, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    MBE_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_casci_warp<DPL, MODE>, a.warps * 32, smem));
    if (per_sm < 1) per_sm = 1;
    k_casci_warp<DPL, MODE><<<ctx->sm_count * per_sm, a.warps * 32, smem, ctx->stream>>>(a, b, L);
    MBE_CU(cudaGetLastError());
    ++ctx->launches;
    return MBE_OK;
}

// One warp-solver bucket: in mixed mode (energies only) the mixed launch and the
// float64 launch that redoes the tuples it flagged, timed as one.
template <int DPL>
static int launch_warp(mbe_ctx *ctx, const BatchArgs &a, int b, const Bucket &bk)
{
    WarpLayout L = warp_layout(a.n, bk.max_ns, bk.max_r, bk.max_n, a.rdm != 0);
    size_t smem = (size_t)L.bytes * a.warps;
    MBE_CHECK(smem <= ctx->smem_optin, MBE_EUNSUPPORTED, "casci_batch: warp solver needs %zu B shared memory",
              smem);
    TimedLaunch tl(ctx, a.order, 0, DPL);
    int rc;
    if (a.pstate != nullptr) {
        const MixLayout LM = mix_layout(a.n, bk.max_ns, bk.max_r, bk.max_n);
        if ((rc = launch_warp_mixed_dpl(ctx, a, b, LM, DPL))) return rc;
        if ((rc = launch_warp_mode<DPL, WM_F64>(ctx, a, b, L, smem))) return rc;
    } else {
        if ((rc = launch_warp_mode<DPL, WM_ALL>(ctx, a, b, L, smem))) return rc;
    }
    return tl.done();
}

int launch_warp_bucket(mbe_ctx *ctx, const BatchArgs &a, int b, const Bucket &bk)
{
    switch (bk.dpl) {
    case 1: return launch_warp<1>(ctx, a, b, bk);
    case 2: return launch_warp<2>(ctx, a, b, bk);
    case 4: return launch_warp<4>(ctx, a, b, bk);
    case 8: return launch_warp<8>(ctx, a, b, bk);
    default: return launch_warp<13>(ctx, a, b, bk);
    }
}

}  // namespace mbe
