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
//  * k_plane_norms: for every digit plane of an arena and every block of
//    256 columns (4 k-blocks), the largest row sum of squares.  One warp per
//    row and block (32 lanes × 8 bf16 digits), 16 rows per warp, 128 rows
//    of one operand per CTA, the CTA's maxima merged with atomicMax.  A
//    streaming read of the D digit planes (the Karatsuba sum planes' sums
//    follow from the digits' squares and cross products).
//  * k_unit_schedule: one CTA per K schedule walks its segments and sets
//    `first`: a segment continues the open unit when its link allows it and
//    the unit's bound, the sum of its segments' bounds, stays ≤ 2^24.  A
//    segment's bound is sqrt(N_i·N_j), N_t the sum of plane t's block maxima
//    over the blocks the segment touches (the largest over the arenas that
//    share the schedule), and never more than its worst-case bound
//    nkb·64·max|d_i|·max|d_j|.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "ffsyrk_internal.h"

namespace fsk {
namespace {

constexpr int NORM_THREADS = 256;
constexpr int NORM_ROWS = 128;                            // rows per CTA
constexpr int NORM_ROWS_PER_WARP = NORM_ROWS / (NORM_THREADS / 32);

// Eight bf16 digits (integers of magnitude ≤ 256) of a 16-byte group.
__device__ __forceinline__ void unpack8(uint4 v, float (&d)[8]) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        d[2 * i] = __uint_as_float(w[i] << 16);
        d[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
}

// Per row and 256-column block the sums of squares of every plane, read
// from the D digit planes alone.  A Karatsuba sum plane's (X_i + X_j)² sums
// to q_i + q_j + 2·c_ij with c_ij = Σ x_i·x_j, so those planes (half of a
// Karatsuba operand's bytes) are never read.  Every quantity is an integer
// of magnitude ≤ 2^24 at every step (digits ≤ 256 in magnitude, 256
// columns; sums of two digits ≤ 256): exact in FP32.  Rows [h, rpad) of
// each plane are padding the pre-additions never write (and no stored
// result reads): skipped.  Grid: x = column block, y = (operand, 128-row
// block of its planes).
template <int D, bool KS>
__global__ void __launch_bounds__(NORM_THREADS, 5) k_plane_norms(const uint16_t *__restrict__ base,
                                                              int64_t kpad, int64_t rpad, int64_t h,
                                                              int planes, int64_t nry,
                                                              uint32_t *table, int32_t nb) {
    constexpr int NQ = KS ? D + D * (D - 1) / 2 : D;  // planes of an operand
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * kNormCols + lane * 8;
    const bool col_ok = c < kpad;  // kpad is a multiple of 64: whole 16-byte groups
    __shared__ uint32_t wmax[NORM_THREADS / 32][NQ];
    const int64_t nyb = (int64_t)gridDim.y;
    for (int64_t y = blockIdx.y; y < nry; y += nyb) {
        const int64_t op = y / (rpad / NORM_ROWS), r0 = (y % (rpad / NORM_ROWS)) * NORM_ROWS;
        const int64_t rw = r0 + (int64_t)warp * NORM_ROWS_PER_WARP;  // row inside a plane
        const uint16_t *ob = base + (op * planes * rpad) * kpad;
        uint32_t best[NQ];
#pragma unroll
        for (int t = 0; t < NQ; ++t) best[t] = 0;
#pragma unroll 2
        for (int i = 0; i < NORM_ROWS_PER_WARP; ++i) {
            const int64_t r = rw + i;
            float q[NQ];
#pragma unroll
            for (int t = 0; t < NQ; ++t) q[t] = 0.f;
            if (col_ok && r < h) {
                float d[D][8];
#pragma unroll
                for (int t = 0; t < D; ++t)
                    unpack8(__ldcs(reinterpret_cast<const uint4 *>(ob + ((int64_t)t * rpad + r) * kpad + c)), d[t]);
#pragma unroll
                for (int e = 0; e < 8; ++e) {
#pragma unroll
                    for (int t = 0; t < D; ++t) q[t] = fmaf(d[t][e], d[t][e], q[t]);
                    if constexpr (KS) {
                        int u = D;
#pragma unroll
                        for (int a = 0; a < D; ++a)
#pragma unroll
                            for (int b = a + 1; b < D; ++b, ++u) q[u] = fmaf(d[a][e], d[b][e], q[u]);
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < NQ; ++t)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) q[t] += __shfl_xor_sync(0xffffffffu, q[t], o);
            if constexpr (KS) {
                int u = D;
#pragma unroll
                for (int a = 0; a < D; ++a)
#pragma unroll
                    for (int b = a + 1; b < D; ++b, ++u) q[u] = q[a] + q[b] + 2.f * q[u];
            }
#pragma unroll
            for (int t = 0; t < NQ; ++t) {
                // a block of digits sums to at most 2^24 (anything else is taken as that)
                const uint32_t v = (q[t] >= 0.f && q[t] <= 16777216.f) ? (uint32_t)q[t] : 16777216u;
                best[t] = max(best[t], v);
            }
        }
        if (lane == 0)
#pragma unroll
            for (int t = 0; t < NQ; ++t) wmax[warp][t] = best[t];
        __syncthreads();
        if (threadIdx.x < NQ) {
            uint32_t m = 0;
#pragma unroll
            for (int w = 0; w < NORM_THREADS / 32; ++w) m = max(m, wmax[w][threadIdx.x]);
            if (m) atomicMax(table + (int64_t)threadIdx.x * nb + blockIdx.x, m);
        }
        __syncthreads();
    }
}

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

cudaError_t launch_plane_norms(const Arena &a, int64_t h, const NormTables &t, int j, int D, bool ks,
                               cudaStream_t st) {
    if (a.rows == 0 || a.kpad == 0) return cudaSuccess;
    if (a.kind != ARENA_BF16 && a.kind != ARENA_BF16_KS) return cudaErrorInvalidValue;
    if (a.rpad % NORM_ROWS != 0 || a.rows % (a.planes * a.rpad) != 0) return cudaErrorInvalidValue;
    const int nq = ks ? D + D * (D - 1) / 2 : D;
    if (nq != a.planes) return cudaErrorInvalidValue;
    const int64_t nb = (a.kpad + kNormCols - 1) / kNormCols;
    if (nb != t.nb[j]) return cudaErrorInvalidValue;
    const int64_t nry = (a.rows / (a.planes * a.rpad)) * (a.rpad / NORM_ROWS);
    dim3 grid((unsigned)nb, (unsigned)std::min<int64_t>(nry, 65535));
    const uint16_t *b = reinterpret_cast<const uint16_t *>(a.base);
    uint32_t *tb = t.base + t.off[j];
#define FSK_NORMS(DD, KK) \
    k_plane_norms<DD, KK><<<grid, NORM_THREADS, 0, st>>>(b, a.kpad, a.rpad, h, a.planes, nry, tb, (int32_t)nb)
    switch (D * 2 + (ks ? 1 : 0)) {
        case 2: FSK_NORMS(1, false); break;
        case 4: FSK_NORMS(2, false); break;
        case 5: FSK_NORMS(2, true); break;
        case 6: FSK_NORMS(3, false); break;
        case 7: FSK_NORMS(3, true); break;
        default: return cudaErrorInvalidValue;
    }
#undef FSK_NORMS
    return cudaGetLastError();
}

cudaError_t launch_unit_schedule(const UnitJob *jobs_dev, int njobs, const NormTables &t,
                                 const uint8_t *links, LeafSeg *segs, const DigitScheme &ds,
                                 cudaStream_t st) {
    if (njobs == 0) return cudaSuccess;
    k_unit_schedule<<<njobs, SCHED_THREADS, 0, st>>>(jobs_dev, t, links, segs, ds);
    return cudaGetLastError();
}

}  // namespace fsk
