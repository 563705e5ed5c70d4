// pass_cut.hpp -- how a block of eq. (stepnomod) is cut into passes (the
// MT generation kernels' schedule), as constexpr functions that the kernels
// and the host (vmt_tune_pass_cut) share.
#pragma once

namespace vmt {

// Passes of the block twist.  A pass may hold up to (n-m) M / VW vectors (no
// vector of it depends on another of it); with T threads a pass of s vectors
// costs ceil(s / T) item slots per thread and one barrier.  Two cuts:
//   * phase form: the row ranges [0, n-m), [n-m, 2(n-m)), [2(n-m), n);
//   * wave form: passes of the largest multiple of T that fits, so that no
//     thread idles at a barrier while others finish an extra item.
// The cheaper one is taken, a barrier counted as 0.4 item slots (measured:
// MT19937-32, 16 lanes, 512 threads, 5 slots + 5 barriers beat 6 + 3, and
// MT19937-64, 8 lanes, 256 threads, 6 slots + 2 barriers beat 5 + 5).
__host__ __device__ constexpr int pass_slots(int nv, int step, int t)
{
    int s = 0;
    for (int v = 0; v < nv; v += step) s += ((nv - v < step ? nv - v : step) + t - 1) / t;
    return s;
}

__host__ __device__ constexpr int pass_step(int nv, int dv, int t)
{
    if (t > dv) return dv;
    const int wave = t * (dv / t);
    const int cost_wave = 10 * pass_slots(nv, wave, t) + 4 * ((nv + wave - 1) / wave);
    const int cost_phase = 10 * pass_slots(nv, dv, t) + 4 * ((nv + dv - 1) / dv);
    return cost_wave < cost_phase ? wave : dv;
}

// In place: true when the rows that the first pass's x_{k+1} operands come
// from (vectors rv .. step + rv - 1) are not written by the block's last pass
// (from vector v_last on), so that those operands for the next block can be
// loaded during the last pass, before its barrier.
__host__ __device__ constexpr bool early_first_preload(int nv, int step, int rv)
{
    return step + rv <= (nv - 1) / step * step;
}

}  // namespace vmt
