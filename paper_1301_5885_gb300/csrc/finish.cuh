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
// Target row t of the segment is row rb.row0 + t of both blocks of A u; it
// is written to y[t] (phi block) and y[rb.ld + t] (psi block), so the full
// product (rb = {0, N, N}) writes y[i] and y[N + i].
template <int TT, int T, int BS>
__device__ __forceinline__ void finish_segment(const StreamKPlan &plan, int64_t a, int64_t c,
                                               const double (&acc1)[T], const double (&acc2)[T],
                                               const double *__restrict__ u, int64_t N, RowBlock rb, double diag1,
                                               double diag2, double *__restrict__ partials,
                                               unsigned int *__restrict__ counters, double *__restrict__ y) {
    const double *__restrict__ uphi = u + rb.row0;
    const double *__restrict__ upsi = u + N + rb.row0;
    double *__restrict__ ypsi = y + rb.ld;
    const int64_t S = plan.source_tiles;
    const int64_t c0 = sk_cta_of(a * S, plan.work, plan.ctas);
    const int64_t c1 = sk_cta_of(a * S + S - 1, plan.work, plan.ctas);
    const int nseg = (int)(c1 - c0 + 1);
    const int tid = threadIdx.x;
    if (nseg == 1) {
#pragma unroll
        for (int t = 0; t < T; ++t) {
            int64_t i = a * TT + t * BS + tid;
            if (i < rb.nrows) {
                y[i] = diag1 * uphi[i] - acc1[t];
                ypsi[i] = diag2 * upsi[i] - acc2[t];
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
        if (i < rb.nrows) {
            y[i] = diag1 * uphi[i] - s1;
            ypsi[i] = diag2 * upsi[i] - s2;
        }
    }
    if (tid == 0) counters[a] = 0u;   // ready for the next launch
}

}  // namespace pb
