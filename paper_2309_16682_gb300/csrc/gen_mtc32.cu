// gen_mtc32.cu -- instantiations of the chain-form generation kernel for
// V-MT19937-32 (the configurations of kKernelCfgs with form kChain).
#include "gen_mtc.cuh"

namespace vmt {

// cudaErrorNotSupported when the configuration or the call's output pattern
// is not compiled (the caller then takes the phase form)
cudaError_t launch_generate_mtc32(int lanes, int lpc, int threads, int store, const GenArgs& a, cudaStream_t s)
{
    using namespace dev;
    const int key = ((lanes * 32 + lpc) * 2048 + threads) * 32 + store;
#define VMT_MTC(M, L, T, S, MINB) \
    case ((M * 32 + L) * 2048 + T) * 32 + S: return launch_mtc<MT32, M, L, S / 4, T, MINB>(a, s);
    switch (key) {
        VMT_MTC(16, 8, 256, 16, 5)
        VMT_MTC(16, 16, 512, 16, 2)
        VMT_MTC(16, 8, 128, 16, 5)
        VMT_MTC(16, 8, 256, 8, 5)
        VMT_MTC(8, 8, 256, 16, 4)
        VMT_MTC(8, 8, 128, 16, 5)
        VMT_MTC(4, 4, 128, 16, 8)
    }
#undef VMT_MTC
    return cudaErrorNotSupported;
}

}  // namespace vmt
