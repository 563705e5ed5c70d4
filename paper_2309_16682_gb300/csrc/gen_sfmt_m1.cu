// gen_sfmt_m1.cu -- V-SFMT19937 generation kernels for M = 1 lanes.
#include "gen_sfmt.cuh"

namespace vmt {
cudaError_t launch_generate_sfmt_1(const GenArgs& a, bool ragged, cudaStream_t s)
{
    return dev::launch_sfmt_m<1>(a, ragged, s);
}
}  // namespace vmt
