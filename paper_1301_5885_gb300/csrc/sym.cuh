// sym.cuh -- shared pieces of the symmetric products: the numbering of the
// upper triangle of square tile pairs and the kernel that finishes a product
// from its row sides and per-tile-pair column sides.
#pragma once

#include <stdint.h>

#include "pb_internal.cuh"

namespace pb {
namespace {

// first tile pair of row tile I (pairs are numbered row by row)
__host__ __device__ inline int64_t sym_row_start(int64_t I, int64_t tiles) { return I * tiles - I * (I - 1) / 2; }
// row tile of tile pair p
__host__ __device__ inline int64_t sym_row_of(int64_t p, int64_t tiles) {
    int64_t lo = 0, hi = tiles - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (sym_row_start(mid, tiles) <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}
// slot of off-diagonal tile pair (I, J), J > I, among the off-diagonal pairs
__host__ __device__ inline int64_t sym_offdiag_index(int64_t I, int64_t J, int64_t tiles) {
    return sym_row_start(I, tiles) + (J - I) - I - 1;
}

// y = diag u - (row side + column sides), each row summed in a fixed order:
// its row-side parts in CTA order, then the column sides of the tile pairs
// (I', R), I' = 0 .. R-1.  Block (R, c) finishes rows R B + 64 c .. + 63 of
// row tile R: its four groups of 64 threads sum the column sides of I' = g,
// g + 4, g + 8, ... (g the group), and group 0 adds the four group sums in
// order of g.
constexpr int kSymFinRows = 64;
constexpr int kSymFinThreads = 256;

template <int B, typename JT>
__global__ void __launch_bounds__(kSymFinThreads)
matvec_sym_finalize(const double *__restrict__ u, int64_t N, double diag1, double diag2, SymPlan plan,
                    const double *__restrict__ islots, const double *__restrict__ iside,
                    const JT *__restrict__ jpart, double *__restrict__ y, const int *__restrict__ skip) {
    constexpr int NG = kSymFinThreads / kSymFinRows;
    static_assert(B % kSymFinRows == 0, "row chunks");
    if (skip != nullptr && *((volatile const int *)skip)) return;
    __shared__ double s_part[NG][2][kSymFinRows];
    const int64_t Tt = plan.tiles;
    const int64_t R = blockIdx.x;
    const int g = threadIdx.x / kSymFinRows;
    const int k = blockIdx.y * kSymFinRows + (threadIdx.x % kSymFinRows);
    double a1 = 0.0, a2 = 0.0;
    for (int64_t Ip = g; Ip < R; Ip += NG) {
        const JT *jp = jpart + sym_offdiag_index(Ip, R, Tt) * 2 * B;
        a1 += (double)jp[k];
        a2 += (double)jp[B + k];
    }
    s_part[g][0][threadIdx.x % kSymFinRows] = a1;
    s_part[g][1][threadIdx.x % kSymFinRows] = a2;
    __syncthreads();
    if (g != 0) return;
    const int64_t i = R * B + k;
    if (i >= N) return;
    const int64_t c0 = sk_cta_of(sym_row_start(R, Tt), plan.work, plan.ctas);
    const int64_t c1 = sk_cta_of(sym_row_start(R + 1, Tt) - 1, plan.work, plan.ctas);
    double s1 = 0.0, s2 = 0.0;
    if (c0 == c1) {
        s1 = iside[R * 2 * B + k];
        s2 = iside[R * 2 * B + B + k];
    } else {
        for (int64_t cc = c0; cc <= c1; ++cc) {
            const int64_t first = sym_row_of(sk_begin(cc, plan.work, plan.ctas), Tt);
            const double *sl = islots + (2 * cc + (R == first ? 0 : 1)) * 2 * B;
            s1 += sl[k];
            s2 += sl[B + k];
        }
    }
#pragma unroll
    for (int gg = 0; gg < NG; ++gg) {
        s1 += s_part[gg][0][threadIdx.x];
        s2 += s_part[gg][1][threadIdx.x];
    }
    y[i] = diag1 * u[i] - s1;
    y[N + i] = diag2 * u[N + i] - s2;
}

}  // namespace
}  // namespace pb
