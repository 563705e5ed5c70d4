// gen_mt.cu -- dispatch of the V-MT19937-32 / V-MT19937-64 generation
// kernels.  The tuning table's configuration (gen_args.hpp) selects the phase
// form or its in-place variant (gen_mt_kernel.cuh, instantiated per variant
// in gen_mt32.cu and gen_mt64.cu) or the chain form (gen_mtc32.cu,
// gen_mtc64.cu); a single-lane call of one output type from word 0 goes to
// the warp-per-generator kernel.
#include "gen_args.hpp"
#include "pass_cut.hpp"
#include "vmt_internal.hpp"

namespace vmt {

// per variant (gen_mt32.cu, gen_mt64.cu): threads = the phase form's CTA
// size (0: its default), in_place = the in-place variant, m1 = the
// warp-per-generator kernel
cudaError_t launch_generate_mt32(int lanes, int threads, bool in_place, bool m1, const GenArgs& a, cudaStream_t s);
cudaError_t launch_generate_mt64(int lanes, int threads, bool in_place, bool m1, const GenArgs& a, cudaStream_t s);
int read_generate_timeout_mt32(bool reset);
int read_generate_timeout_mt64(bool reset);
cudaError_t launch_generate_mtc32(int lanes, int lpc, int threads, int store, const GenArgs& a, cudaStream_t s);
cudaError_t launch_generate_mtc64(int lanes, int lpc, int threads, int store, const GenArgs& a, cudaStream_t s);

// 1 if a generation kernel gave up on a bounded wait since the last reset
int read_generate_timeout(bool reset)
{
    const int a = read_generate_timeout_mt32(reset), b = read_generate_timeout_mt64(reset);
    if (a < 0 || b < 0) return -1;
    return a | b;
}

namespace {
// true when the warp kernel takes the call: one segment from word 0 of a type
// that takes one generator word per output
bool m1_eligible(int variant, const GenArgs& a)
{
    if (a.nseg != 1 || a.seg[0].wbeg != 0) return false;
    const int d = a.seg[0].dtype;
    return variant == VMT_MT19937_64 ? (d == VMT_U64 || d == VMT_F64 || d == VMT_F32) : (d == VMT_U32 || d == VMT_F32);
}
}  // namespace

int pass_cut(int variant, int lanes, int index, int* out)
{
    const KernelCfg* cfg = kernel_cfg(variant, lanes, index);
    if (!cfg || cfg->form == kChain) return -1;
    const int n = variant == VMT_MT19937_32 ? 624 : 312, m = variant == VMT_MT19937_32 ? 397 : 156;
    const int vw = variant == VMT_MT19937_32 ? (lanes < 4 ? lanes : 4) : (lanes < 2 ? lanes : 2);
    const int rv = lanes / vw, nv = n * rv, dv = (n - m) * rv;
    const int step = pass_step(nv, dv, cfg->threads);
    out[0] = nv;
    out[1] = step;
    out[2] = rv;
    out[3] = (n - m) * rv;
    out[4] = m * rv;
    out[5] = cfg->threads;
    out[6] = cfg->form == kInPlace;
    out[7] = early_first_preload(nv, step, rv);
    return 0;
}

cudaError_t launch_generate_mt(int variant, int lanes, const GenArgs& a_in, cudaStream_t s)
{
    GenArgs a = a_in;
    a.k = kShiftK;   // the tempering's multipliers travel as kernel parameters
    const bool m1 = lanes == 1 && m1_eligible(variant, a);
    // a.kcfg selects among the compiled configurations of (variant, lanes)
    const KernelCfg* cfg = kernel_cfg(variant, lanes, a.kcfg);
    if (!cfg) cfg = kernel_cfg(variant, lanes, 0);
    int t = 0;        // CTA size of the phase form (0: its default)
    bool ip = false;  // in-place phase form
    if (!m1 && cfg && cfg->form == kChain) {
        // unit launches (per-generator positions) keep one CTA per generator
        if (!a.units || cfg->lpc == lanes) {
            const cudaError_t e = variant == VMT_MT19937_32
                                      ? launch_generate_mtc32(lanes, cfg->lpc, cfg->threads, cfg->store, a, s)
                                      : launch_generate_mtc64(lanes, cfg->lpc, cfg->threads, cfg->store, a, s);
            if (e != cudaErrorNotSupported) return e;
        }
    } else if (cfg) {
        t = cfg->threads;
        ip = cfg->form == kInPlace;
    }
    if (variant == VMT_MT19937_32) return launch_generate_mt32(lanes, t, ip, m1, a, s);
    if (variant == VMT_MT19937_64) return launch_generate_mt64(lanes, t, ip, m1, a, s);
    return cudaErrorInvalidValue;
}

}  // namespace vmt
