// gen_sfmt_m4.cu -- V-SFMT19937 generation kernels for M = 4 lanes.
#include "gen_sfmt.cuh"

namespace vmt {
cudaError_t launch_generate_sfmt_4(const GenArgs& a, bool ragged, cudaStream_t s)
{
    return dev::launch_sfmt_m<4>(a, ragged, s);
}
}  // namespace vmt
