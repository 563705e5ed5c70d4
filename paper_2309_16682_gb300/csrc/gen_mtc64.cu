// gen_mtc64.cu -- instantiations of the chain-form generation kernel for
// V-MT19937-64 (the configurations of kKernelCfgs with form kChain).
#include "gen_mtc.cuh"

namespace vmt {

// cudaErrorNotSupported when the configuration or the call's output pattern
// is not compiled (the caller then takes the phase form)
cudaError_t launch_generate_mtc64(int lanes, int lpc, int threads, int store, const GenArgs& a, cudaStream_t s)
{
    using namespace dev;
    const int key = ((lanes * 32 + lpc) * 2048 + threads) * 32 + store;
#define VMT_MTC(M, L, T, S, MINB) \
    case ((M * 32 + L) * 2048 + T) * 32 + S: return launch_mtc<MT64, M, L, S / 8, T, MINB>(a, s);
    switch (key) {
        VMT_MTC(16, 4, 160, 16, 6)
        VMT_MTC(16, 8, 320, 16, 3)
        VMT_MTC(8, 4, 160, 16, 6)
        VMT_MTC(8, 8, 320, 16, 3)
        VMT_MTC(8, 4, 160, 8, 6)
        VMT_MTC(4, 4, 160, 16, 6)
    }
#undef VMT_MTC
    return cudaErrorNotSupported;
}

}  // namespace vmt
