// gemm_tc.cu -- tensor-core (tcgen05) GEMM path; filled in below.
#include "common.cuh"

namespace dmrg {

bool tc_available(dmrg_ctx *) { return false; }

dmrg_status gemm_3xtf32(dmrg_ctx *, int, int, int, double, const double *, long long, long long, long long,
                        const double *, long long, long long, long long, double, double *, long long, long long,
                        long long, int)
{
    return DMRG_EUNSUPPORTED;
}

}  // namespace dmrg
