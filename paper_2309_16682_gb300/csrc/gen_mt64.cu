// gen_mt64.cu -- the V-MT19937-64 instances of the generation kernels
// (gen_mt_kernel.cuh), compiled apart from the MT19937-32 ones.
#include "gen_mt_kernel.cuh"

namespace vmt {

cudaError_t launch_generate_mt64(int lanes, int t, bool ip, bool m1, const GenArgs& a, cudaStream_t s)
{
    using namespace dev;
    if (m1) {
        const int d = a.seg[0].dtype;
        return d == VMT_U64 ? launch_mt1<MT64, VMT_U64>(a, s)
                            : (d == VMT_F64 ? launch_mt1<MT64, VMT_F64>(a, s) : launch_mt1<MT64, VMT_F32>(a, s));
    }
    switch (lanes) {
    case 1: return launch_mt<MT64, 1, 1, 256>(a, s);
    case 2: return launch_mt<MT64, 2, 2, 256>(a, s);
    case 4: return ip ? launch_mt<MT64, 4, 2, 256, true>(a, s) : launch_mt<MT64, 4, 2, 256>(a, s);
    case 8:
        if (ip) return launch_mt<MT64, 8, 2, 256, true>(a, s);
        return t == 512 ? launch_mt<MT64, 8, 2, 512>(a, s) : launch_mt<MT64, 8, 2, 256>(a, s);
    case 16:
        if (ip) return launch_mt<MT64, 16, 2, 256, true>(a, s);
        return t == 1024 ? launch_mt<MT64, 16, 2, 1024>(a, s) : launch_mt<MT64, 16, 2, 512>(a, s);
    }
    return cudaErrorInvalidValue;
}

int read_generate_timeout_mt64(bool reset) { return dev::read_timeout_flag(reset); }

}  // namespace vmt
