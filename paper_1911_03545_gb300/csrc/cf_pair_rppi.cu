// cf_pair_rppi.cu -- instances of the pair kernel for kind "rppi" (see cf_pair.cuh).
#include "cf_pair.cuh"

using namespace cfpair;

#define CF_L(W, R, WR, LO) return launch_one<KIND_RPPI, W, R, WR, LO>(c, a, num_sms, st, grid_out, warps_out)

cudaError_t cfp_launch_rppi(const CfPairCfg &c, const CfPairArgs &a, int num_sms, cudaStream_t st, int *grid_out,
                          int *warps_out)
{
    if (c.wrap) {
        if (c.weighted) {
            if (c.ravg) { if (c.lo) CF_L(true, true, true, true); else CF_L(true, true, true, false); }
            CF_L(true, false, true, false);
        }
        if (c.ravg) { if (c.lo) CF_L(false, true, true, true); else CF_L(false, true, true, false); }
        CF_L(false, false, true, false);
    }
    if (c.weighted) {
        if (c.ravg) { if (c.lo) CF_L(true, true, false, true); else CF_L(true, true, false, false); }
        CF_L(true, false, false, false);
    }
    if (c.ravg) { if (c.lo) CF_L(false, true, false, true); else CF_L(false, true, false, false); }
    CF_L(false, false, false, false);
}
