// cf_pair_theta.cu -- instances of the pair kernel for kind "theta" (see cf_pair.cuh).
#include "cf_pair.cuh"

using namespace cfpair;

#define CF_L(W, R, WR, LO) return launch_one<KIND_THETA, W, R, WR, LO>(c, a, num_sms, st, grid_out, warps_out)

cudaError_t cfp_launch_theta(const CfPairCfg &c, const CfPairArgs &a, int num_sms, cudaStream_t st, int *grid_out,
                          int *warps_out)
{
    if (c.weighted) {
        if (c.ravg) { if (c.lo) CF_L(true, true, false, true); else CF_L(true, true, false, false); }
        CF_L(true, false, false, false);
    }
    if (c.ravg) { if (c.lo) CF_L(false, true, false, true); else CF_L(false, true, false, false); }
    CF_L(false, false, false, false);
}
