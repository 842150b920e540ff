// vp_fel.cuh -- FEL field update from per-tile partial sums (Sec. IV.B, dA/dz = <exp(-i Phi)>),
// shared by the standalone finalize kernels and the step kernel's last CTA.
//
// Drift-kick-drift in time: A^{n+1/2} = A^n + h/2 b^n, the push uses A^{n+1/2}, b^{n+1} =
// <exp(-i theta)> of the new weights, A^{n+1} = A^{n+1/2} + h/2 b^{n+1}. The partials
// (sum w, sum w cos theta, sum w sin theta) are summed by kFinThreads threads in a fixed
// order (a strided pass, then a tree), so the result does not depend on which block runs it
// or on scheduling: a simulation stepped alone or in a batch gets the same bits.
#pragma once

#include "vp_internal.h"

namespace vp {

constexpr int kFinThreads = 256;

// Every thread of the block calls it (it synchronises the block), with any block size: the
// sums run over kFinThreads virtual lanes v (lane v adds the partials v, v + kFinThreads, ...,
// then a tree over the lanes), each thread taking the lanes t, t + blockDim.x, ..., so the
// order of every addition is the same for any block size. s: 3 * kFinThreads doubles of shared
// memory. Partials are read through L2 (other CTAs of the same launch may have written them).
__device__ __forceinline__ void fel_finalize_core(const double *part, int nparts, double *state,
                                                  double *hist, int hist_cap, double dt, int init,
                                                  int rk4, double *s)
{
    const int t = threadIdx.x, nt = blockDim.x;
    for (int v = t; v < kFinThreads; v += nt) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int k = v; k < nparts; k += kFinThreads) {
            a0 += __ldcg(part + 3 * k);
            a1 += __ldcg(part + 3 * k + 1);
            a2 += __ldcg(part + 3 * k + 2);
        }
        s[v] = a0;
        s[kFinThreads + v] = a1;
        s[2 * kFinThreads + v] = a2;
    }
    __syncthreads();
    for (int o = kFinThreads / 2; o > 0; o >>= 1) {
        for (int v = t; v < o; v += nt)
            for (int q = 0; q < 3; ++q) s[q * kFinThreads + v] += s[q * kFinThreads + v + o];
        __syncthreads();
    }
    if (t != 0) return;
    const double sw = s[0];
    const double b_re = s[kFinThreads] / sw, b_im = -s[2 * kFinThreads] / sw;
    state[ST_B_RE] = b_re;
    state[ST_B_IM] = b_im;
    if (init) {
        // A^0 already stored; A^{1/2} = A^0 + h/2 b^0
        state[ST_AH_RE] = state[ST_A_RE] + 0.5 * dt * b_re;
        state[ST_AH_IM] = state[ST_A_IM] + 0.5 * dt * b_im;
        // kick amplitude K = A^{1/2} (space charge adds i sigma2 <e^{-i theta~}> afterwards)
        state[ST_K_RE] = state[ST_AH_RE];
        state[ST_K_IM] = state[ST_AH_IM];
        state[ST_M] = hypot(state[ST_AH_RE], state[ST_AH_IM]);
        state[ST_PHI] = atan2(state[ST_AH_RE], -state[ST_AH_IM]);
        return;
    }
    // DKD: A^{n+1} = A^{n+1/2} + h/2 b^{n+1}; RK4: the stages left A^{n+1} in ST_AH
    const double are = rk4 ? state[ST_AH_RE] : state[ST_AH_RE] + 0.5 * dt * b_re;
    const double aim = rk4 ? state[ST_AH_IM] : state[ST_AH_IM] + 0.5 * dt * b_im;
    state[ST_A_RE] = are;
    state[ST_A_IM] = aim;
    state[ST_AH_RE] = are + 0.5 * dt * b_re;
    state[ST_AH_IM] = aim + 0.5 * dt * b_im;
    state[ST_K_RE] = state[ST_AH_RE];
    state[ST_K_IM] = state[ST_AH_IM];
    // sine-term weights of the next push: alpha = -Im K, beta = Re K
    state[ST_M] = hypot(state[ST_AH_RE], state[ST_AH_IM]);
    state[ST_PHI] = atan2(state[ST_AH_RE], -state[ST_AH_IM]);
    const long step = (long)state[ST_STEP];
    if (hist && hist_cap > 0) {
        const long slot = step % hist_cap;
        hist[2 * slot] = are;
        hist[2 * slot + 1] = aim;
    }
    state[ST_STEP] = (double)(step + 1);
    state[ST_TAU] = (double)(step + 1) * dt;
}

}  // namespace vp
