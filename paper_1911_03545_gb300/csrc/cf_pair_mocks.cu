// cf_pair_mocks.cu -- instances of the pair kernel for DD(rp, pi) of observed positions
// (Appendix A.2.1; see cf_pair.cuh).  Non-periodic only, direct form only (run_mocks).
#include "cf_pair.cuh"

using namespace cfpair;

// global histograms, per-warp histograms with fixed-point sums, or per-warp with FP64 sums
template <bool W, bool R, bool LO>
static cudaError_t launch_mocks(const CfPairCfg &c, const CfPairArgs &a, int num_sms, cudaStream_t st, int *grid_out,
                                int *warps_out)
{
    if (c.ghist) return launch_variant<KIND_MOCKS, W, R, false, LO, false, true>(c, a, num_sms, st, grid_out, warps_out);
    if constexpr (W || R)
        if (a.fxw != 0.f || a.fxr != 0.f)
            return launch_variant<KIND_MOCKS, W, R, false, LO, false, false, true>(c, a, num_sms, st, grid_out,
                                                                               warps_out);
    return launch_variant<KIND_MOCKS, W, R, false, LO, false, false>(c, a, num_sms, st, grid_out, warps_out);
}

#define CF_L(W, R, LO) return launch_mocks<W, R, LO>(c, a, num_sms, st, grid_out, warps_out)

cudaError_t cfp_launch_mocks(const CfPairCfg &c, const CfPairArgs &a, int num_sms, cudaStream_t st, int *grid_out,
                             int *warps_out)
{
    if (c.wrap || c.variant == 2) return cudaErrorInvalidValue;
    if (c.weighted) {
        if (c.ravg) { if (c.lo) CF_L(true, true, true); else CF_L(true, true, false); }
        CF_L(true, false, false);
    }
    if (c.ravg) { if (c.lo) CF_L(false, true, true); else CF_L(false, true, false); }
    CF_L(false, false, false);
}
