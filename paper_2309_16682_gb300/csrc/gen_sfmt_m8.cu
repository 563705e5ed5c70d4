// gen_sfmt_m8.cu -- V-SFMT19937 generation kernels for M = 8 lanes.
#include "gen_sfmt.cuh"

namespace vmt {
cudaError_t launch_generate_sfmt_8(const GenArgs& a, bool ragged, cudaStream_t s)
{
    return dev::launch_sfmt_m<8>(a, ragged, s);
}
}  // namespace vmt
