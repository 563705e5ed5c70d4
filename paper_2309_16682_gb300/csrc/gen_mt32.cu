// gen_mt32.cu -- the V-MT19937-32 instances of the generation kernels
// (gen_mt_kernel.cuh), compiled apart from the MT19937-64 ones.
#include "gen_mt_kernel.cuh"

namespace vmt {

cudaError_t launch_generate_mt32(int lanes, int t, bool ip, bool m1, const GenArgs& a, cudaStream_t s)
{
    using namespace dev;
    if (m1) return a.seg[0].dtype == VMT_U32 ? launch_mt1<MT32, VMT_U32>(a, s) : launch_mt1<MT32, VMT_F32>(a, s);
    switch (lanes) {
    case 1: return launch_mt<MT32, 1, 1, 256>(a, s);
    case 2: return launch_mt<MT32, 2, 2, 256>(a, s);
    case 4: return launch_mt<MT32, 4, 4, 256>(a, s);
    case 8:
        if (ip) return launch_mt<MT32, 8, 4, 256, true>(a, s);
        return t == 512 ? launch_mt<MT32, 8, 4, 512>(a, s) : launch_mt<MT32, 8, 4, 256>(a, s);
    case 16:
        if (ip) return launch_mt<MT32, 16, 4, 256, true>(a, s);
        return t == 1024 ? launch_mt<MT32, 16, 4, 1024>(a, s) : launch_mt<MT32, 16, 4, 512>(a, s);
    }
    return cudaErrorInvalidValue;
}

int read_generate_timeout_mt32(bool reset) { return dev::read_timeout_flag(reset); }

}  // namespace vmt
