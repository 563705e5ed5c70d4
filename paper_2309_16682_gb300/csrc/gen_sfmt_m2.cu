// gen_sfmt_m2.cu -- V-SFMT19937 generation kernels for M = 2 lanes.
#include "gen_sfmt.cuh"

namespace vmt {
cudaError_t launch_generate_sfmt_2(const GenArgs& a, bool ragged, cudaStream_t s)
{
    return dev::launch_sfmt_m<2>(a, ragged, s);
}
}  // namespace vmt
