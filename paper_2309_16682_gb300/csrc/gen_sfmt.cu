// gen_sfmt.cu -- lane-count dispatch of the V-SFMT19937 generation kernels
// (gen_sfmt.cuh, instantiated in gen_sfmt_m*.cu).
#include "vmt_internal.hpp"

namespace vmt {
cudaError_t launch_generate_sfmt_1(const GenArgs& a, bool ragged, cudaStream_t s);
cudaError_t launch_generate_sfmt_2(const GenArgs& a, bool ragged, cudaStream_t s);
cudaError_t launch_generate_sfmt_4(const GenArgs& a, bool ragged, cudaStream_t s);
cudaError_t launch_generate_sfmt_8(const GenArgs& a, bool ragged, cudaStream_t s);
cudaError_t launch_generate_sfmt_16(const GenArgs& a, bool ragged, cudaStream_t s);

cudaError_t launch_generate_sfmt(int lanes, const GenArgs& a, bool ragged, cudaStream_t s)
{
    switch (lanes) {
    case 1: return launch_generate_sfmt_1(a, ragged, s);
    case 2: return launch_generate_sfmt_2(a, ragged, s);
    case 4: return launch_generate_sfmt_4(a, ragged, s);
    case 8: return launch_generate_sfmt_8(a, ragged, s);
    case 16: return launch_generate_sfmt_16(a, ragged, s);
    }
    return cudaErrorInvalidValue;
}
}  // namespace vmt
