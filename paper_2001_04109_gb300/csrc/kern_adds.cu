// Block additions of Algorithm 2 (arXiv 2001.04109, Section 3) on the GPU.
//
//  * prep: the 4 pre-additions S1 = (A21 − A11)·Y, S2 = A22 − A21·Y,
//    S3 = S1 − A22, S4 = S3 + A12 of every node of one recursion depth, fused
//    with the signed base-256 digit split that feeds the leaf products.
//  * digitize: the digit split alone, for the classical path's operands.
//  * post: the post-additions Low(U1) = Low(P1 + P5), Low(U3) = Low(P1 + P2),
//    Up(U1) = Low(U1)ᵀ, U2 = U1 + P4, U4 = U2 + P3, Low(U5) = Low(U2 + P4ᵀ),
//    written straight into the node's result [[U3, ·], [U4, U5]].
// All are HBM-bound streaming kernels, coalesced along rows; the two
// transposed reads of the post-additions are staged through shared memory.
// The prep and digit kernels are instantiated per digit count, operand type
// and Y form, so the per-element work is straight-line integer code.
#include <cuda_bf16.h>

#include <algorithm>

#include "ffsyrk_internal.h"

namespace fsk {
namespace {

__device__ __forceinline__ uint32_t red(uint32_t x, const ModP &m) {
    // x < 2^32: q under-estimates x/p by at most one, so r ∈ [0, 2p).
    uint32_t q = __umulhi(x, m.barrett);
    uint32_t r = x - q * m.p;
    return r >= m.p ? r - m.p : r;
}
__device__ __forceinline__ uint32_t addm(uint32_t a, uint32_t b, uint32_t p) {
    uint32_t r = a + b;
    return r >= p ? r - p : r;
}
__device__ __forceinline__ uint32_t subm(uint32_t a, uint32_t b, uint32_t p) {
    uint32_t r = a + (p - b);
    return r >= p ? r - p : r;
}
// x·w mod p for x < 2^32, w < p (Shoup: q = ⌊x·w_sh / 2^32⌋, r ∈ [0, 2p)).
__device__ __forceinline__ uint32_t mulc(uint32_t x, MulConst c, uint32_t p) {
    uint32_t q = __umulhi(x, c.w_sh);
    uint32_t r = x * c.w - q * p;
    return r >= p ? r - p : r;
}

__device__ __forceinline__ uint32_t ld_view(const MatView &v, int64_t r, int64_t c) {
    return (r < v.vr && c < v.vc) ? __ldg(v.ptr + r * v.ld + c) : 0u;
}

// Float bits of the small integer d (|d| < 2^22) without a conversion
// instruction: 1.5·2^23 + d is exact in FP32, so subtracting 1.5·2^23 leaves
// exactly d.  For |d| ≤ 256 the low 16 bits are zero, i.e. the high half is
// the exact bf16 encoding of d.
__device__ __forceinline__ uint32_t small_int_f32_bits(int d) {
    return __float_as_uint(__int_as_float(0x4B400000 + d) - 12582912.0f);
}
__device__ __forceinline__ int sbyte(int s) {
    int d;
    asm("bfe.s32 %0, %1, 0, 8;" : "=r"(d) : "r"(s));
    return d;
}

// Store the residue pair (v0, v1) at (row r, column c) of an operand.
template <int D, bool U32>
__device__ __forceinline__ void put_pair(const OperandDst &d, int64_t r, int64_t c, uint32_t v0,
                                         uint32_t v1, uint32_t half, uint32_t p) {
    if (d.arena == nullptr) return;
    if (U32) {
        *reinterpret_cast<uint2 *>(static_cast<uint32_t *>(d.arena) + (d.row0 + r) * d.kpad + c) =
            make_uint2(v0, v1);
        return;
    }
    int s0 = v0 > half ? (int)v0 - (int)p : (int)v0;  // symmetric residue
    int s1 = v1 > half ? (int)v1 - (int)p : (int)v1;
    uint32_t *base = static_cast<uint32_t *>(d.arena);  // bf16 pairs
#pragma unroll
    for (int t = 0; t < D; ++t) {
        int d0, d1;
        if (t == D - 1) {
            d0 = s0;
            d1 = s1;
        } else {
            d0 = sbyte(s0);
            d1 = sbyte(s1);
            s0 = (s0 - d0) >> 8;
            s1 = (s1 - d1) >> 8;
        }
        const uint32_t packed =
            __byte_perm(small_int_f32_bits(d0), small_int_f32_bits(d1), 0x7632);
        base[((d.row0 + t * d.rpad + r) * d.kpad + c) >> 1] = packed;
    }
}

template <int YF>
__device__ __forceinline__ void ymul(const YConst &y, uint32_t t0, uint32_t t1, uint32_t &o0,
                                     uint32_t &o1, uint32_t p) {
    if (YF == 0) {
        o0 = mulc(t0, y.a, p);
        o1 = mulc(t1, y.a, p);
    } else {
        // row vector times I ⊗ [[a, b], [−b, a]]: (t0·a − t1·b, t0·b + t1·a)
        o0 = subm(mulc(t0, y.a, p), mulc(t1, y.b, p), p);
        o1 = addm(mulc(t0, y.b, p), mulc(t1, y.a, p), p);
    }
}

constexpr int PREP_THREADS = 128;  // column pairs per block
constexpr int PREP_ROWS = 4;       // rows per thread (independent loads in flight)

// Columns [w, kpad) of every written operand are zero (K padding of the
// leaf products); rows [h, rpad) are never read into a stored result.
// Grid: x = column-pair blocks, y = row blocks (strided), z = node.
// RED: reduce the loaded values mod p (only the caller's A can hold values ≥ p).
template <int D, bool U32, int YF, bool RED>
__global__ void __launch_bounds__(PREP_THREADS) k_prep(const PrepNode *__restrict__ nodes,
                                                       int64_t h, int64_t w, int64_t kpad, ModP m,
                                                       YConst y) {
    const int64_t c = 2 * ((int64_t)blockIdx.x * PREP_THREADS + threadIdx.x);
    if (c >= kpad) return;
    const PrepNode &nd = nodes[blockIdx.z];
    const uint32_t p = m.p, half = m.half;
    const bool inside = c < w;
    const int64_t nrb = (h + PREP_ROWS - 1) / PREP_ROWS;
    for (int64_t rb = blockIdx.y; rb < nrb; rb += gridDim.y) {
        uint32_t a[PREP_ROWS][4][2];  // quadrant 0..3 = A11, A12, A21, A22
#pragma unroll
        for (int i = 0; i < PREP_ROWS; ++i) {
            const int64_t r = rb * PREP_ROWS + i;
            const bool ok = inside && r < h;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                a[i][0][e] = ok ? ld_view(nd.X, r, c + e) : 0u;
                a[i][1][e] = ok ? ld_view(nd.X, r, w + c + e) : 0u;
                a[i][2][e] = ok ? ld_view(nd.X, h + r, c + e) : 0u;
                a[i][3][e] = ok ? ld_view(nd.X, h + r, w + c + e) : 0u;
            }
        }
#pragma unroll
        for (int i = 0; i < PREP_ROWS; ++i) {
            const int64_t r = rb * PREP_ROWS + i;
            if (r >= h) break;
            uint32_t x11[2], x12[2], x21[2], x22[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                x11[e] = RED ? red(a[i][0][e], m) : a[i][0][e];
                x12[e] = RED ? red(a[i][1][e], m) : a[i][1][e];
                x21[e] = RED ? red(a[i][2][e], m) : a[i][2][e];
                x22[e] = RED ? red(a[i][3][e], m) : a[i][3][e];
            }
            uint32_t t0 = subm(x21[0], x11[0], p), t1 = subm(x21[1], x11[1], p);
            uint32_t s1[2], s2[2], s3[2], s4[2], u[2];
            ymul<YF>(y, t0, t1, s1[0], s1[1], p);       // S1 = (A21 − A11)·Y
            ymul<YF>(y, x21[0], x21[1], u[0], u[1], p);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                s2[e] = subm(x22[e], u[e], p);          // S2 = A22 − A21·Y
                s3[e] = subm(s1[e], x22[e], p);         // S3 = S1 − A22
                s4[e] = addm(s3[e], x12[e], p);         // S4 = S3 + A12
            }
            put_pair<D, U32>(nd.gemm[0], r, c, x22[0], x22[1], half, p);
            put_pair<D, U32>(nd.gemm[1], r, c, s4[0], s4[1], half, p);
            put_pair<D, U32>(nd.gemm[2], r, c, s1[0], s1[1], half, p);
            put_pair<D, U32>(nd.gemm[3], r, c, s2[0], s2[1], half, p);
            put_pair<D, U32>(nd.leaf[0], r, c, x11[0], x11[1], half, p);
            put_pair<D, U32>(nd.leaf[1], r, c, x12[0], x12[1], half, p);
            put_pair<D, U32>(nd.leaf[2], r, c, s3[0], s3[1], half, p);
            if (nd.s3 != nullptr && inside)
                *reinterpret_cast<uint2 *>(nd.s3 + r * nd.s3_ld + c) = make_uint2(s3[0], s3[1]);
        }
    }
}

// Digit split of whole matrices (the classical path's operands): rows
// [0, rows) × columns [0, kpad) of each destination, zero beyond the view.
// Grid: x = column-pair blocks, y = row blocks (strided), z = matrix.
constexpr int DIG_ROWS = 8;
template <int D, bool U32>
__global__ void __launch_bounds__(PREP_THREADS) k_digitize(const DigitizeJob *__restrict__ jobs,
                                                           ModP m) {
    const DigitizeJob &jb = jobs[blockIdx.z];
    const int64_t c = 2 * ((int64_t)blockIdx.x * PREP_THREADS + threadIdx.x);
    if (c >= jb.dst.kpad) return;
    const int64_t nrb = (jb.rows + DIG_ROWS - 1) / DIG_ROWS;
    for (int64_t rb = blockIdx.y; rb < nrb; rb += gridDim.y) {
        uint32_t v[DIG_ROWS][2];
#pragma unroll
        for (int i = 0; i < DIG_ROWS; ++i) {
            const int64_t r = rb * DIG_ROWS + i;
            v[i][0] = r < jb.rows ? ld_view(jb.X, r, c) : 0u;
            v[i][1] = r < jb.rows ? ld_view(jb.X, r, c + 1) : 0u;
        }
#pragma unroll
        for (int i = 0; i < DIG_ROWS; ++i) {
            const int64_t r = rb * DIG_ROWS + i;
            if (r >= jb.rows) break;
            put_pair<D, U32>(jb.dst, r, c, red(v[i][0], m), red(v[i][1], m), m.half, m.p);
        }
    }
}

// The same digit split over a flattened block list: block b belongs to the
// job t with block0[t] ≤ b < block0[t+1] (binary search), then to one row
// block and one column block of that job.
template <int D, bool U32>
__global__ void __launch_bounds__(PREP_THREADS) k_digitize_flat(const DigitizeJob *__restrict__ jobs,
                                                                int njobs, ModP m) {
    const int64_t b = blockIdx.x + (int64_t)blockIdx.y * gridDim.x;
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].block0 <= b) lo = mid; else hi = mid - 1;
    }
    const DigitizeJob &jb = jobs[lo];
    const int64_t gx = (jb.dst.kpad / 2 + PREP_THREADS - 1) / PREP_THREADS;
    const int64_t local = b - jb.block0;
    const int64_t rb = local / gx, cb = local - rb * gx;
    if (rb * DIG_ROWS >= jb.rows) return;
    const int64_t c = 2 * (cb * PREP_THREADS + threadIdx.x);
    if (c >= jb.dst.kpad) return;
    uint32_t v[DIG_ROWS][2];
#pragma unroll
    for (int i = 0; i < DIG_ROWS; ++i) {
        const int64_t r = rb * DIG_ROWS + i;
        v[i][0] = r < jb.rows ? ld_view(jb.X, r, c) : 0u;
        v[i][1] = r < jb.rows ? ld_view(jb.X, r, c + 1) : 0u;
    }
#pragma unroll
    for (int i = 0; i < DIG_ROWS; ++i) {
        const int64_t r = rb * DIG_ROWS + i;
        if (r >= jb.rows) break;
        put_pair<D, U32>(jb.dst, r, c, red(v[i][0], m), red(v[i][1], m), m.half, m.p);
    }
}

constexpr int PT = 32;  // post-addition tile: 32×32, 256 threads, 4 rows each

// Grid: x = tile column J, y = tile row I, z = 3·node + quadrant, where the
// quadrants of the node's 2h×2h result are 0: C11 = Low(U3), 1: C21 = U4,
// 2: C22 = Low(U5).  Tiles above the diagonal of quadrants 0 and 2 exit.
// Every quadrant first issues all of its loads, then combines.
__global__ void __launch_bounds__(256) k_post(const PostNode *__restrict__ nodes, int64_t h,
                                              ModP m) {
    __shared__ uint32_t sa[PT][PT + 1];
    __shared__ uint32_t so[PT][PT + 1];
    const PostNode &nd = nodes[blockIdx.z / 3];
    const int quad = blockIdx.z % 3;
    const int64_t I = blockIdx.y, J = blockIdx.x;
    if (quad != 1 && J > I) return;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const uint32_t p = m.p;
    constexpr int NR = PT / 8;
    const int64_t j = J * PT + tx;
    uint32_t vals[NR];
    if (quad == 0) {
        uint32_t x[NR], z[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            const int64_t i = I * PT + ty + 8 * q;
            const bool ok = i < h && j < h && j <= i;
            x[q] = ok ? __ldg(nd.P1 + i * nd.ldr + j) : 0u;
            z[q] = ok ? __ldg(nd.P2 + i * nd.ldr + j) : 0u;
        }
#pragma unroll
        for (int q = 0; q < NR; ++q) vals[q] = addm(x[q], z[q], p);  // Low(U3) = Low(P1 + P2)
    } else if (quad == 1) {
        // Up(U1) = Low(U1)ᵀ: tile (J, I) of P1 + P5 through shared memory
        if (I <= J) {
            uint32_t t1[NR], t5[NR];
#pragma unroll
            for (int q = 0; q < NR; ++q) {
                const int64_t rr = J * PT + ty + 8 * q, cc = I * PT + tx;
                const bool ok = rr < h && cc < h;
                t1[q] = ok ? __ldg(nd.P1 + rr * nd.ldr + cc) : 0u;
                t5[q] = ok ? __ldg(nd.P5 + rr * nd.ldr + cc) : 0u;
            }
#pragma unroll
            for (int q = 0; q < NR; ++q) sa[ty + 8 * q][tx] = t1[q] + t5[q];
            __syncthreads();
        }
        uint32_t u1[NR], g3[NR], g4[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            const int ly = ty + 8 * q;
            const int64_t i = I * PT + ly;
            const bool ok = i < h && j < h;
            const bool lowr = ok && i >= j;
            const uint32_t a1 = lowr ? __ldg(nd.P1 + i * nd.ldr + j) : 0u;
            const uint32_t a5 = lowr ? __ldg(nd.P5 + i * nd.ldr + j) : 0u;
            u1[q] = lowr ? a1 + a5 : (ok ? sa[tx][ly] : 0u);
            g3[q] = ok ? __ldg(nd.P3 + i * nd.ldg + j) : 0u;
            g4[q] = ok ? __ldg(nd.P4 + i * nd.ldg + j) : 0u;
        }
#pragma unroll
        for (int q = 0; q < NR; ++q) vals[q] = red(u1[q] + g4[q] + g3[q], m);  // U4 = U1 + P4 + P3
    } else {
        // P4ᵀ: tile (J, I) of P4 through shared memory
        {
            uint32_t t4[NR];
#pragma unroll
            for (int q = 0; q < NR; ++q) {
                const int64_t rr = J * PT + ty + 8 * q, cc = I * PT + tx;
                t4[q] = (rr < h && cc < h) ? __ldg(nd.P4 + rr * nd.ldg + cc) : 0u;
            }
#pragma unroll
            for (int q = 0; q < NR; ++q) sa[ty + 8 * q][tx] = t4[q];
        }
        uint32_t a1[NR], a5[NR], g4[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            const int64_t i = I * PT + ty + 8 * q;
            const bool ok = i < h && j < h && j <= i;
            a1[q] = ok ? __ldg(nd.P1 + i * nd.ldr + j) : 0u;
            a5[q] = ok ? __ldg(nd.P5 + i * nd.ldr + j) : 0u;
            g4[q] = ok ? __ldg(nd.P4 + i * nd.ldg + j) : 0u;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            const int ly = ty + 8 * q;
            vals[q] = red(a1[q] + a5[q] + g4[q] + sa[tx][ly], m);  // Low(U5) = Low(U1 + P4 + P4ᵀ)
        }
    }
    const int64_t r0 = (quad == 0 ? 0 : h) + I * PT, c0 = (quad == 2 ? h : 0) + J * PT;
    if (!nd.upper) {
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            const int ly = ty + 8 * q;
            const int64_t R = r0 + ly, Cc = c0 + tx;
            const bool inside = (I * PT + ly < h) && (J * PT + tx < h);
            if (inside && R < nd.vn && Cc < nd.vn && Cc <= R) nd.out[R * nd.ldo + Cc] = vals[q];
        }
    } else {
#pragma unroll
        for (int q = 0; q < NR; ++q) so[ty + 8 * q][tx] = vals[q];
        __syncthreads();
        // element (R, Cc) of the lower result goes to out[Cc][R]
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            const int lc = ty + 8 * q;  // column within the tile
            const int64_t R = r0 + tx, Cc = c0 + lc;
            const bool inside = (I * PT + tx < h) && (J * PT + lc < h);
            if (inside && R < nd.vn && Cc < nd.vn && Cc <= R) nd.out[Cc * nd.ldo + R] = so[tx][lc];
        }
    }
}

// Zero row r0 + blockIdx.y of the selected triangle of C.
__global__ void k_zero_tri(uint32_t *C, int64_t n, int64_t ldc, int upper, int64_t r0) {
    const int64_t r = r0 + blockIdx.y;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x)
        if (upper ? c >= r : c <= r) C[r * ldc + c] = 0;
}

template <int D, bool U32, int YF, bool RED>
cudaError_t launch_prep_t(dim3 grid, cudaStream_t st, const PrepNode *nodes, int64_t h, int64_t w,
                          int64_t kpad, ModP mp, YConst y) {
    k_prep<D, U32, YF, RED><<<grid, PREP_THREADS, 0, st>>>(nodes, h, w, kpad, mp, y);
    return cudaGetLastError();
}

template <int D, bool U32>
cudaError_t launch_prep_d(dim3 grid, cudaStream_t st, const PrepNode *nodes, int64_t h, int64_t w,
                          int64_t kpad, ModP mp, YConst y, bool reduce) {
    if (y.form == 0)
        return reduce ? launch_prep_t<D, U32, 0, true>(grid, st, nodes, h, w, kpad, mp, y)
                      : launch_prep_t<D, U32, 0, false>(grid, st, nodes, h, w, kpad, mp, y);
    return reduce ? launch_prep_t<D, U32, 1, true>(grid, st, nodes, h, w, kpad, mp, y)
                  : launch_prep_t<D, U32, 1, false>(grid, st, nodes, h, w, kpad, mp, y);
}

}  // namespace

cudaError_t launch_prep(const PrepNode *nodes_dev, int nnodes, int64_t h, int64_t w,
                        int64_t kpad, ModP mp, YConst y, DigitScheme ds, int arena_kind,
                        bool reduce_input, cudaStream_t st) {
    if (h == 0 || kpad == 0 || nnodes == 0) return cudaSuccess;
    const int64_t gx = (kpad / 2 + PREP_THREADS - 1) / PREP_THREADS;
    const int64_t gy = std::min<int64_t>((h + PREP_ROWS - 1) / PREP_ROWS, 65535);
    dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)nnodes);
    if (arena_kind == ARENA_U32)
        return launch_prep_d<1, true>(grid, st, nodes_dev, h, w, kpad, mp, y, reduce_input);
    switch (ds.D) {
        case 1: return launch_prep_d<1, false>(grid, st, nodes_dev, h, w, kpad, mp, y, reduce_input);
        case 2: return launch_prep_d<2, false>(grid, st, nodes_dev, h, w, kpad, mp, y, reduce_input);
        case 3: return launch_prep_d<3, false>(grid, st, nodes_dev, h, w, kpad, mp, y, reduce_input);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_digitize(const DigitizeJob *jobs_dev, int njobs, int64_t max_rows,
                            int64_t max_kpad, ModP mp, DigitScheme ds, int arena_kind,
                            cudaStream_t st) {
    if (njobs == 0 || max_rows == 0 || max_kpad == 0) return cudaSuccess;
    const int64_t gx = (max_kpad / 2 + PREP_THREADS - 1) / PREP_THREADS;
    const int64_t gy = std::min<int64_t>((max_rows + DIG_ROWS - 1) / DIG_ROWS, 65535);
    dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)njobs);
    if (arena_kind == ARENA_U32) {
        k_digitize<1, true><<<grid, PREP_THREADS, 0, st>>>(jobs_dev, mp);
    } else {
        switch (ds.D) {
            case 1: k_digitize<1, false><<<grid, PREP_THREADS, 0, st>>>(jobs_dev, mp); break;
            case 2: k_digitize<2, false><<<grid, PREP_THREADS, 0, st>>>(jobs_dev, mp); break;
            case 3: k_digitize<3, false><<<grid, PREP_THREADS, 0, st>>>(jobs_dev, mp); break;
            default: return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

int64_t digitize_flat_blocks(int64_t rows, int64_t kpad) {
    return ((rows + DIG_ROWS - 1) / DIG_ROWS) * ((kpad / 2 + PREP_THREADS - 1) / PREP_THREADS);
}

cudaError_t launch_digitize_flat(const DigitizeJob *jobs_dev, int njobs, int64_t total_blocks,
                                 ModP mp, DigitScheme ds, int arena_kind, cudaStream_t st) {
    if (njobs == 0 || total_blocks == 0) return cudaSuccess;
    const int64_t gx = std::min<int64_t>(total_blocks, 65535);
    const int64_t gy = (total_blocks + gx - 1) / gx;
    if (gy > 65535) return cudaErrorInvalidValue;
    dim3 grid((unsigned)gx, (unsigned)gy);
    // blocks past the last job's range find its job and return on the row check
    if (arena_kind == ARENA_U32) {
        k_digitize_flat<1, true><<<grid, PREP_THREADS, 0, st>>>(jobs_dev, njobs, mp);
    } else {
        switch (ds.D) {
            case 1: k_digitize_flat<1, false><<<grid, PREP_THREADS, 0, st>>>(jobs_dev, njobs, mp); break;
            case 2: k_digitize_flat<2, false><<<grid, PREP_THREADS, 0, st>>>(jobs_dev, njobs, mp); break;
            case 3: k_digitize_flat<3, false><<<grid, PREP_THREADS, 0, st>>>(jobs_dev, njobs, mp); break;
            default: return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_post(const PostNode *nodes_dev, int nnodes, int64_t h, ModP mp,
                        cudaStream_t st) {
    if (h == 0 || nnodes == 0) return cudaSuccess;
    const int64_t T = (h + PT - 1) / PT;
    if (T > 65535 || 3 * (int64_t)nnodes > 65535) return cudaErrorInvalidValue;
    dim3 grid((unsigned)T, (unsigned)T, (unsigned)(3 * nnodes));
    k_post<<<grid, 256, 0, st>>>(nodes_dev, h, mp);
    return cudaGetLastError();
}

cudaError_t launch_zero_tri(uint32_t *C, int64_t n, int64_t ldc, int upper, cudaStream_t st) {
    for (int64_t r0 = 0; r0 < n; r0 += 65535) {
        const int64_t rows = std::min<int64_t>(65535, n - r0);
        dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 1024), (unsigned)rows);
        k_zero_tri<<<grid, 256, 0, st>>>(C, n, ldc, upper, r0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace fsk
