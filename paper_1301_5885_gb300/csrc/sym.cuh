// sym.cuh -- shared pieces of the symmetric products: the numbering of the
// upper triangle of square tile pairs and the kernel that finishes a product
// from its row sides and per-tile-pair column sides.
#pragma once

#include <stdint.h>

#include <vector>

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

// Banded form (the default for large N, see sym_band_cuts).  The product runs
// as bands of whole row tiles [R0, R1): the pair kernel evaluates the band's
// tile pairs (plan with work_begin = sym_row_start(R0)) and stores only the
// band's column sides; this kernel then finishes the band's rows and folds
// the band's column sides of the later row tiles into FP64 accumulators
// colacc (tiles x 2B).
// Block (R - R0, c), R in [R0, tiles), covers entries 64 c .. + 63 of tile R:
// its four groups sum the band's column sides (I', R), I' = R0 + g, R0 + g + 4,
// ... (I' < min(R, R1)), then
//   R <  R1: y = diag u - (row side + colacc[R] + group sums in order of g),
//            colacc[R] holding the earlier bands' column sides of R;
//   R >= R1: colacc[R] (+)= group sums in order of g (stored by the first band).
// Every row is summed in a fixed order, independent of the launch shape.
template <int B, typename JT>
__global__ void __launch_bounds__(kSymFinThreads)
matvec_sym_band_finish(const double *__restrict__ u, int64_t N, double diag1, double diag2, SymPlan plan,
                       int64_t R0, int64_t R1, const double *__restrict__ islots, const double *__restrict__ iside,
                       const JT *__restrict__ jpart, double *__restrict__ colacc, double *__restrict__ y,
                       const int *__restrict__ skip) {
    constexpr int NG = kSymFinThreads / kSymFinRows;
    static_assert(B % kSymFinRows == 0, "row chunks");
    if (skip != nullptr && *((volatile const int *)skip)) return;
    __shared__ double s_part[NG][2][kSymFinRows];
    const int64_t Tt = plan.tiles;
    const int64_t R = R0 + blockIdx.x;
    const int g = threadIdx.x / kSymFinRows, kl = threadIdx.x % kSymFinRows;
    const int k = blockIdx.y * kSymFinRows + kl;
    const int64_t Iend = R < R1 ? R : R1;
    double a1 = 0.0, a2 = 0.0;
    for (int64_t Ip = R0 + g; Ip < Iend; Ip += NG) {
        const JT *jp = jpart + (sym_offdiag_index(Ip, R, Tt) - plan.joff) * 2 * B;
        a1 += (double)jp[k];
        a2 += (double)jp[B + k];
    }
    s_part[g][0][kl] = a1;
    s_part[g][1][kl] = a2;
    __syncthreads();
    if (g != 0) return;
    double t1 = s_part[0][0][kl], t2 = s_part[0][1][kl];
#pragma unroll
    for (int gg = 1; gg < NG; ++gg) {
        t1 += s_part[gg][0][kl];
        t2 += s_part[gg][1][kl];
    }
    double *ca = colacc + R * 2 * B;
    if (R >= R1) {
        if (R0 == 0) {
            ca[k] = t1;
            ca[B + k] = t2;
        } else {
            ca[k] += t1;
            ca[B + k] += t2;
        }
        return;
    }
    const int64_t i = R * B + k;
    if (i >= N) return;
    const int64_t wb = plan.work_begin;
    const int64_t c0 = sk_cta_of(sym_row_start(R, Tt) - wb, plan.work, plan.ctas);
    const int64_t c1 = sk_cta_of(sym_row_start(R + 1, Tt) - 1 - wb, plan.work, plan.ctas);
    double s1 = 0.0, s2 = 0.0;
    if (c0 == c1) {
        s1 = iside[R * 2 * B + k];
        s2 = iside[R * 2 * B + B + k];
    } else {
        for (int64_t cc = c0; cc <= c1; ++cc) {
            const int64_t first = sym_row_of(wb + sk_begin(cc, plan.work, plan.ctas), Tt);
            const double *sl = islots + (2 * cc + (R == first ? 0 : 1)) * 2 * B;
            s1 += sl[k];
            s2 += sl[B + k];
        }
    }
    if (R0 > 0) {
        s1 += ca[k];
        s2 += ca[B + k];
    }
    s1 += t1;
    s2 += t2;
    y[i] = diag1 * u[i] - s1;
    y[N + i] = diag2 * u[N + i] - s2;
}

// Scratch of a symmetric product with tiles of B targets and column sides of
// elem bytes: row sides (tiles x 2B FP64), split-row slots (2 per CTA, 2B
// FP64 each), the column sides (of all off-diagonal tile pairs, or of the
// largest band, 2B elem each) and, when banded, the FP64 column accumulators
// (tiles x 2B).  A banded product keeps two sets of slots and column sides,
// so that consecutive bands can run at the same time.  Offsets in bytes.
struct SymLayout {
    int64_t islots, jpart, colacc, bytes;
    int64_t islots_stride, jpart_stride;   // bytes between the two sets (banded)
};
inline int64_t sym_r256(int64_t b) { return (b + 255) / 256 * 256; }
inline SymLayout sym_layout(const SymPlan &pl, int B, int elem, int64_t slots, bool banded) {
    const int nbuf = banded ? 2 : 1;
    SymLayout l;
    l.islots = sym_r256(pl.tiles * 2 * B * (int64_t)sizeof(double));
    l.islots_stride = sym_r256(pl.ctas * 4 * B * (int64_t)sizeof(double));
    l.jpart = l.islots + nbuf * l.islots_stride;
    l.jpart_stride = sym_r256(slots * 2 * B * (int64_t)elem);
    l.colacc = l.jpart + nbuf * l.jpart_stride;
    l.bytes = l.colacc + (banded ? sym_r256(pl.tiles * 2 * B * (int64_t)sizeof(double)) : 0);
    return l;
}

// off-diagonal column sides of the row tiles [R0, R1)
inline int64_t sym_band_slots(int64_t tiles, int64_t R0, int64_t R1) {
    return (sym_row_start(R1, tiles) - R1) - (sym_row_start(R0, tiles) - R0);
}

// the plan of band [R0, R1) of a full plan: its tile pairs, CTAs and offsets
inline SymPlan sym_band_plan(const SymPlan &full, int64_t R0, int64_t R1) {
    SymPlan b = full;
    b.work_begin = sym_row_start(R0, full.tiles);
    b.work = sym_row_start(R1, full.tiles) - b.work_begin;
    b.joff = b.work_begin - R0;
    b.ctas = full.ctas < b.work ? full.ctas : b.work;
    return b;
}

// Bands split off for speed (bands = 0): the pair kernel of one launch ends
// on a tail of CTAs finishing at different times, which the next band's
// launch on the other stream fills.  As many bands as give every CTA at
// least kBandMinPairs tile pairs each, at most kBandMaxAuto (measured on
// GB300: 81,920 triangles 1295 -> 1337 Gpairs/s at 6 bands, 2572 -> 2731
// with kappa = 0; 300,176 triangles 1317 -> 1396..1402 at 14 to 79 bands;
// at 79 bands (the cap's choice there) each band's column sides stay in L2
// and the product moves 27 MB through DRAM instead of 1.47 GB, with 44 MB of
// scratch; bands of 2 tile pairs per CTA lose again for kappa = 0).
constexpr int64_t kBandMinPairs = 5;
constexpr int64_t kBandMaxAuto = 72;

// Band cuts 0 = R_0 < R_1 < ... < R_m = tiles: whole row tiles holding about
// equal numbers of column sides, at most the room that the scratch bound
// limit leaves (bytes, 0: no bound; two sets of column sides) and at most
// total / n for n requested bands: bands = 0 for the automatic split above,
// 1 for none, n >= 2 for at least n.  Without a request of n >= 2 the product
// takes one band whenever bands would not need less scratch.  A row tile whose
// column sides alone exceed the room is a band of its own.
inline void sym_band_cuts(const SymPlan &pl, int B, int elem, int64_t limit, int bands,
                          std::vector<int64_t> *cuts) {
    const int64_t tiles = pl.tiles, total = sym_band_slots(tiles, 0, tiles);
    const int64_t unbanded = sym_layout(pl, B, elem, total, false).bytes;
    cuts->clear();
    cuts->push_back(0);
    int64_t room = total + 1;                     // no constraint
    if (limit > 0 && unbanded > limit) {
        const SymLayout fixed = sym_layout(pl, B, elem, 0, true);
        const int64_t r = (limit - fixed.bytes) / (2 * 2 * B * (int64_t)elem);
        room = r < 1 ? 1 : r;
    }
    int64_t want = bands >= 2 ? bands : 1;
    if (bands == 0) {
        want = (pl.work / (pl.ctas > 0 ? pl.ctas : 1)) / kBandMinPairs;
        if (want > kBandMaxAuto) want = kBandMaxAuto;
    }
    if (want >= 2) {
        const int64_t r = (total + want - 1) / want;
        if (r < room) room = r < 1 ? 1 : r;
    }
    if (total <= room) {
        cuts->push_back(tiles);
        return;
    }
    const int64_t nb = (total + room - 1) / room;
    const int64_t target = (total + nb - 1) / nb;
    for (int64_t R0 = 0; R0 < tiles;) {
        int64_t R1 = R0 + 1;
        while (R1 < tiles && sym_band_slots(tiles, R0, R1 + 1) <= target) ++R1;
        cuts->push_back(R1);
        R0 = R1;
    }
    if (bands < 2) {
        int64_t m = 0;
        for (size_t b = 0; b + 1 < cuts->size(); ++b) {
            const int64_t sl = sym_band_slots(tiles, (*cuts)[b], (*cuts)[b + 1]);
            if (sl > m) m = sl;
        }
        if (sym_layout(pl, B, elem, m, true).bytes >= unbanded) {
            cuts->resize(1);
            cuts->push_back(tiles);
        }
    }
}

// largest band of the cuts, in column sides
inline int64_t sym_max_band_slots(int64_t tiles, const std::vector<int64_t> &cuts) {
    int64_t m = 0;
    for (size_t b = 0; b + 1 < cuts.size(); ++b) {
        const int64_t s = sym_band_slots(tiles, cuts[b], cuts[b + 1]);
        if (s > m) m = s;
    }
    return m;
}

// Enqueue one symmetric product: pair(plan, islots, iside, jpart, evaluated,
// stream) launches the pair kernel over the plan's tile pairs, then the
// finishing kernel runs.  With more than one band, band b runs on st (b even)
// or aux (b odd) with set b % 2 of the slots and column sides: the pair
// kernel of band b + 1 overlaps the end of band b's (whose last CTAs leave
// SMs idle), the finishing kernels run in band order (each waits for the
// previous one: the column accumulators), and a set is reused by the same
// stream two bands later.  ev: three events; aux joins st at the end.  The
// product counter goes to the first band's pair kernel only.  Counts every
// launch but one (the caller counts the product's first).
template <int B, typename JT, typename Pair>
cudaError_t sym_enqueue(const SymPlan &sp, const std::vector<int64_t> &cuts, void *scratch, const double *u,
                        int64_t N, double diag1, double diag2, double *y, const int *skip,
                        unsigned long long *counter, cudaStream_t st, cudaStream_t aux, cudaEvent_t *ev,
                        Pair pair) {
    const bool banded = cuts.size() > 2;
    const SymLayout l = sym_layout(sp, B, (int)sizeof(JT), banded ? sym_max_band_slots(sp.tiles, cuts) : 0, banded);
    char *base = (char *)scratch;
    double *iside = (double *)base;
    if (!banded) {
        double *islots = (double *)(base + l.islots);
        JT *jpart = (JT *)(base + l.jpart);
        pair(sp, islots, iside, jpart, counter, st);
        matvec_sym_finalize<B, JT><<<dim3((unsigned)sp.tiles, B / kSymFinRows), kSymFinThreads, 0, st>>>(
            u, N, diag1, diag2, sp, islots, iside, jpart, y, skip);
        PB_LAUNCHED();
        return cudaSuccess;
    }
    double *colacc = (double *)(base + l.colacc);
    cudaError_t e = cudaEventRecord(ev[2], st);            // the product's inputs are ready on st
    if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev[2], 0);
    const size_t nb = cuts.size() - 1;
    for (size_t b = 0; b < nb && e == cudaSuccess; ++b) {
        const int64_t R0 = cuts[b], R1 = cuts[b + 1];
        const SymPlan bp = sym_band_plan(sp, R0, R1);
        cudaStream_t s = (b & 1) ? aux : st;
        double *islots = (double *)(base + l.islots + (int64_t)(b & 1) * l.islots_stride);
        JT *jpart = (JT *)(base + l.jpart + (int64_t)(b & 1) * l.jpart_stride);
        pair(bp, islots, iside, jpart, b == 0 ? counter : nullptr, s);
        if (b > 0) PB_LAUNCHED();
        if (b > 0) e = cudaStreamWaitEvent(s, ev[(b - 1) & 1], 0);
        if (e != cudaSuccess) break;
        matvec_sym_band_finish<B, JT><<<dim3((unsigned)(sp.tiles - R0), B / kSymFinRows), kSymFinThreads, 0, s>>>(
            u, N, diag1, diag2, bp, R0, R1, islots, iside, jpart, colacc, y, skip);
        PB_LAUNCHED();
        e = cudaEventRecord(ev[b & 1], s);
    }
    // the last finishing kernel follows every other launch of the product
    if (e == cudaSuccess && ((nb - 1) & 1)) e = cudaStreamWaitEvent(st, ev[(nb - 1) & 1], 0);
    if (e != cudaSuccess) {
        // join whatever reached the second stream before reporting the error
        if (cudaEventRecord(ev[2], aux) == cudaSuccess) cudaStreamWaitEvent(st, ev[2], 0);
    }
    return e;
}

}  // namespace
}  // namespace pb
