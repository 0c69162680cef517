// finish.cuh -- the end of a stream-K segment of the plain (non-symmetric)
// product kernels: a target tile covered by one CTA is written directly; one
// split over several CTAs is finished by the last of them to arrive, which
// adds the partial rows in CTA order (deterministic, no floating-point
// atomics) and the diagonal term.
#pragma once

#include "pb_internal.cuh"

namespace pb {

// Finish a segment: either write y directly (one CTA covers the whole target
// tile) or publish partial rows and let the last arriving CTA reduce them.
template <int TT, int T, int BS>
__device__ __forceinline__ void finish_segment(const StreamKPlan &plan, int64_t a, int64_t c,
                                               const double (&acc1)[T], const double (&acc2)[T],
                                               const double *__restrict__ u, int64_t N, double diag1,
                                               double diag2, double *__restrict__ partials,
                                               unsigned int *__restrict__ counters, double *__restrict__ y) {
    const int64_t S = plan.source_tiles;
    const int64_t c0 = sk_cta_of(a * S, plan.work, plan.ctas);
    const int64_t c1 = sk_cta_of(a * S + S - 1, plan.work, plan.ctas);
    const int nseg = (int)(c1 - c0 + 1);
    const int tid = threadIdx.x;
    if (nseg == 1) {
#pragma unroll
        for (int t = 0; t < T; ++t) {
            int64_t i = a * TT + t * BS + tid;
            if (i < N) {
                y[i] = diag1 * u[i] - acc1[t];
                y[N + i] = diag2 * u[N + i] - acc2[t];
            }
        }
        return;
    }
    const int ord = (int)(c - c0);
    double *mine = partials + ((a * plan.max_segments + ord) * 2) * TT;
#pragma unroll
    for (int t = 0; t < T; ++t) {
        mine[t * BS + tid] = acc1[t];
        mine[TT + t * BS + tid] = acc2[t];
    }
    __threadfence();
    __syncthreads();
    __shared__ int s_last;
    if (tid == 0) {
        unsigned int prev = atomicAdd(&counters[a], 1u);
        s_last = (prev == (unsigned int)(nseg - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
#pragma unroll
    for (int t = 0; t < T; ++t) {
        int64_t i = a * TT + t * BS + tid;
        double s1 = 0.0, s2 = 0.0;
        for (int o = 0; o < nseg; ++o) {
            const double *pp = partials + ((a * plan.max_segments + o) * 2) * TT;
            s1 += __ldcg(pp + t * BS + tid);
            s2 += __ldcg(pp + TT + t * BS + tid);
        }
        if (i < N) {
            y[i] = diag1 * u[i] - s1;
            y[N + i] = diag2 * u[N + i] - s2;
        }
    }
    if (tid == 0) counters[a] = 0u;   // ready for the next launch
}

}  // namespace pb
