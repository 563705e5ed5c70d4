// gen_sfmt_m16.cu -- V-SFMT19937 generation kernels for M = 16 lanes.
#include "gen_sfmt.cuh"

namespace vmt {
cudaError_t launch_generate_sfmt_16(const GenArgs& a, bool ragged, cudaStream_t s)
{
    return dev::launch_sfmt_m<16>(a, ragged, s);
}
}  // namespace vmt
