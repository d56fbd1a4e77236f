// Unit lengths of the tensor-core leaf from the digits a call actually holds.
//
// Delayed modular reduction (arXiv 2001.04109, Section 4.2) lets an exact
// accumulator run as long as no partial sum can leave its exact range; for
// the FP32 tensor-memory accumulators of the leaf that range is |x| ≤ 2^24.
// The host schedule (build_segments) bounds a unit by the largest digit
// magnitudes.  Here the bound comes from the operands: for one digit pair
// over a K range, every partial sum of Σ_k x_k·z_k, summed in any order, is
// at most Σ_k |x_k|·|z_k| ≤ sqrt(Σ_k x_k²)·sqrt(Σ_k z_k²) (Cauchy–Schwarz).
//
//  * The block maxima: for every digit plane of an arena and every block of
//    256 columns (4 k-blocks), the largest row sum of squares.  The kernels
//    that write the digit planes take them (put8 with a NormAcc: one warp
//    writes one row of a block, adds its lanes' sums and keeps the largest
//    per plane, merged into the table with atomicMax), so the planes are
//    not read again.
//  * k_unit_schedule: one CTA per K schedule walks its segments and sets
//    `first`: a segment continues the open unit when its link allows it and
//    the unit's bound, the sum of its segments' bounds, stays ≤ 2^24.  A
//    segment's bound is sqrt(N_i·N_j), N_t the sum of plane t's block maxima
//    over the blocks the segment touches (the largest over the arenas that
//    share the schedule), and never more than its worst-case bound
//    nkb·64·max|d_i|·max|d_j|.
#include <cuda_runtime.h>

#include <cmath>

#include "ffsyrk_internal.h"

namespace fsk {
namespace {

constexpr int SCHED_THREADS = 256;
constexpr int SCHED_CHUNK = 1024;  // segments whose bounds are staged in shared memory at a time

// One CTA per K schedule.  Every segment's bound needs a few dependent global
// loads, so the CTA's threads compute a chunk of bounds in parallel into
// shared memory; thread 0 then walks the chunk (the greedy merge is
// sequential) and writes the `first` flags, carrying the open unit's bound
// into the next chunk.
__global__ void __launch_bounds__(SCHED_THREADS) k_unit_schedule(const UnitJob *__restrict__ jobs,
                                                                 const NormTables t,
                                                                 const uint8_t *__restrict__ links,
                                                                 LeafSeg *segs,
                                                                 const __grid_constant__ DigitScheme ds) {
    __shared__ double bnd[SCHED_CHUNK];
    __shared__ uint8_t lnk[SCHED_CHUNK];
    const UnitJob J = jobs[blockIdx.x];
    const double limit = 16777216.0;  // 2^24
    double cur = 0.0;                 // thread 0: bound of the open unit
    for (int base = 0; base < J.nseg; base += SCHED_CHUNK) {
        const int cnt = min(SCHED_CHUNK, J.nseg - base);
        for (int s = threadIdx.x; s < cnt; s += SCHED_THREADS) {
            const LeafSeg sg = segs[J.seg0 + base + s];
            const int i = sg.ij >> 4, j = sg.ij & 15;
            const int b0 = sg.kb0 / 4, b1 = (sg.kb0 + (int)sg.nkb - 1) / 4;
            double ni = 0.0, nj = 0.0;
            for (int b = b0; b <= b1; ++b) {
                uint32_t mi = 0, mj = 0;
                for (int a = 0; a <= kMaxLevels; ++a) {
                    if (!((J.arenas >> a) & 1u)) continue;
                    if (b >= t.nb[a]) {  // no table entry: the largest a block can hold
                        mi = mj = 16777216u;
                        continue;
                    }
                    const uint32_t *T = t.base + t.off[a];
                    mi = max(mi, T[(int64_t)i * t.nb[a] + b]);
                    mj = max(mj, T[(int64_t)j * t.nb[a] + b]);
                }
                ni += mi;
                nj += mj;
            }
            const double worst = (double)sg.nkb * 64.0 * ds.max_digit[i] * ds.max_digit[j];
            // sqrt of an exact double product: relative error ~2^-52, covered by the margin
            const double b = i == j ? ni : sqrt(ni * nj) * (1.0 + 1e-12) + 1.0;
            bnd[s] = fmin(b, worst);
            lnk[s] = (base + s > 0) ? links[J.seg0 + base + s] : 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int s = 0; s < cnt; ++s) {
                const bool cont = lnk[s] != 0 && cur + bnd[s] <= limit;
                segs[J.seg0 + base + s].first = cont ? 0 : 1;
                cur = cont ? cur + bnd[s] : bnd[s];
            }
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_unit_schedule(const UnitJob *jobs_dev, int njobs, const NormTables &t,
                                 const uint8_t *links, LeafSeg *segs, const DigitScheme &ds,
                                 cudaStream_t st) {
    if (njobs == 0) return cudaSuccess;
    k_unit_schedule<<<njobs, SCHED_THREADS, 0, st>>>(jobs_dev, t, links, segs, ds);
    return cudaGetLastError();
}

}  // namespace fsk
