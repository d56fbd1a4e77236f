// Block additions of Algorithm 2 (arXiv 2001.04109, Section 3) on the GPU.
//
//  * prep: the 4 pre-additions S1 = (A21 − A11)·Y, S2 = A22 − A21·Y,
//    S3 = S1 − A22, S4 = S3 + A12 of every node of one recursion depth, fused
//    with the signed base-256 digit split that feeds the leaf products.
//  * post: the post-additions Low(U1) = Low(P1 + P5), Low(U3) = Low(P1 + P2),
//    Up(U1) = Low(U1)ᵀ, U2 = U1 + P4, U4 = U2 + P3, Low(U5) = Low(U2 + P4ᵀ),
//    written straight into the node's result [[U3, ·], [U4, U5]].
// Both are HBM-bound streaming kernels: coalesced along rows, with the two
// transposed reads of the post-additions staged through shared memory.
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

// Write the residue pair (v0, v1) at (r, 2·cp) of an operand destination.
__device__ __forceinline__ void put_pair(const OperandDst &d, int64_t r, int64_t c, uint32_t v0,
                                         uint32_t v1, const ModP &m, const DigitScheme &ds,
                                         int kind) {
    if (d.arena == nullptr) return;
    if (kind == ARENA_U32) {
        uint2 *dst = reinterpret_cast<uint2 *>(static_cast<uint32_t *>(d.arena) +
                                               (d.row0 + r) * d.kpad + c);
        *dst = make_uint2(v0, v1);
        return;
    }
    int s0 = v0 > m.half ? (int)v0 - (int)m.p : (int)v0;
    int s1 = v1 > m.half ? (int)v1 - (int)m.p : (int)v1;
    __nv_bfloat16 *base = static_cast<__nv_bfloat16 *>(d.arena);
#pragma unroll
    for (int t = 0; t < kMaxDigits; ++t) {
        if (t >= ds.D) break;
        int d0, d1;
        if (t == ds.D - 1) {
            d0 = s0;
            d1 = s1;
        } else {
            d0 = (int)(int8_t)(s0 & 0xFF);
            d1 = (int)(int8_t)(s1 & 0xFF);
            s0 = (s0 - d0) >> 8;
            s1 = (s1 - d1) >> 8;
        }
        __nv_bfloat162 pr;
        pr.x = __int2bfloat16_rn(d0);
        pr.y = __int2bfloat16_rn(d1);
        *reinterpret_cast<__nv_bfloat162 *>(base + (d.row0 + t * d.rpad + r) * d.kpad + c) = pr;
    }
}

__device__ __forceinline__ void ymul(const YConst &y, uint32_t t0, uint32_t t1, uint32_t &o0,
                                     uint32_t &o1, uint32_t p) {
    if (y.form == 0) {
        o0 = mulc(t0, y.a, p);
        o1 = mulc(t1, y.a, p);
    } else {
        // row vector times I ⊗ [[a, b], [−b, a]]: (t0·a − t1·b, t0·b + t1·a)
        o0 = subm(mulc(t0, y.a, p), mulc(t1, y.b, p), p);
        o1 = addm(mulc(t0, y.b, p), mulc(t1, y.a, p), p);
    }
}

// Columns [w, kpad) of every written operand are zero (K padding of the
// leaf products); rows [h, rpad) are never read into a stored result.
__global__ void __launch_bounds__(256) k_prep(const PrepNode *__restrict__ nodes, int nnodes,
                                              int64_t h, int64_t w, int64_t kpad, ModP m,
                                              YConst y, DigitScheme ds, int kind) {
    const int64_t wp = kpad / 2;  // column pairs written per operand row
    const int64_t per_node = h * wp;
    const int64_t total = per_node * nnodes;
    const uint32_t p = m.p;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int node = (int)(idx / per_node);
        const int64_t rem = idx - node * per_node;
        const int64_t r = rem / wp;
        const int64_t c = (rem - r * wp) * 2;
        const PrepNode &nd = nodes[node];
        const bool inside = c < w;
        uint32_t a11[2] = {0, 0}, a12[2] = {0, 0}, a21[2] = {0, 0}, a22[2] = {0, 0};
        if (inside) {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                a11[e] = red(ld_view(nd.X, r, c + e), m);
                a12[e] = red(ld_view(nd.X, r, w + c + e), m);
                a21[e] = red(ld_view(nd.X, h + r, c + e), m);
                a22[e] = red(ld_view(nd.X, h + r, w + c + e), m);
            }
        }
        uint32_t t0 = subm(a21[0], a11[0], p), t1 = subm(a21[1], a11[1], p);
        uint32_t s1[2], s2[2], s3[2], s4[2], u[2];
        ymul(y, t0, t1, s1[0], s1[1], p);          // S1 = (A21 − A11)·Y
        ymul(y, a21[0], a21[1], u[0], u[1], p);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            s2[e] = subm(a22[e], u[e], p);          // S2 = A22 − A21·Y
            s3[e] = subm(s1[e], a22[e], p);         // S3 = S1 − A22
            s4[e] = addm(s3[e], a12[e], p);         // S4 = S3 + A12
        }
        put_pair(nd.gemm[0], r, c, a22[0], a22[1], m, ds, kind);
        put_pair(nd.gemm[1], r, c, s4[0], s4[1], m, ds, kind);
        put_pair(nd.gemm[2], r, c, s1[0], s1[1], m, ds, kind);
        put_pair(nd.gemm[3], r, c, s2[0], s2[1], m, ds, kind);
        put_pair(nd.leaf[0], r, c, a11[0], a11[1], m, ds, kind);
        put_pair(nd.leaf[1], r, c, a12[0], a12[1], m, ds, kind);
        put_pair(nd.leaf[2], r, c, s3[0], s3[1], m, ds, kind);
        if (nd.s3 != nullptr && inside)
            *reinterpret_cast<uint2 *>(nd.s3 + r * nd.s3_ld + c) = make_uint2(s3[0], s3[1]);
    }
}

// Digit split of a whole matrix (the classical path's only operand).
// Digit split of whole matrices (the classical path's operands): rows
// [0, rows) × columns [0, kpad) of each destination, zero beyond the view.
// blockIdx.y selects the matrix.
__global__ void __launch_bounds__(256) k_digitize(const DigitizeJob *__restrict__ jobs, ModP m,
                                                  DigitScheme ds, int kind) {
    const DigitizeJob jb = jobs[blockIdx.y];
    const int64_t cp = jb.dst.kpad / 2;
    const int64_t total = jb.rows * cp;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = idx / cp;
        const int64_t c = (idx - r * cp) * 2;
        uint32_t v0 = red(ld_view(jb.X, r, c), m);
        uint32_t v1 = red(ld_view(jb.X, r, c + 1), m);
        put_pair(jb.dst, r, c, v0, v1, m, ds, kind);
    }
}

// Lower-triangular tile index → (I, J), I ≥ J.
__device__ __forceinline__ void tri_tile(int64_t idx, int64_t &I, int64_t &J) {
    int64_t i = (int64_t)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
    while (i * (i + 1) / 2 > idx) --i;
    while ((i + 1) * (i + 2) / 2 <= idx) ++i;
    I = i;
    J = idx - i * (i + 1) / 2;
}

constexpr int PT = 32;  // post-addition tile

__global__ void __launch_bounds__(256) k_post(const PostNode *__restrict__ nodes, int64_t h,
                                              ModP m) {
    __shared__ uint32_t sa[PT][PT + 1];
    __shared__ uint32_t sb[PT][PT + 1];
    __shared__ uint32_t so[PT][PT + 1];
    const PostNode &nd = nodes[blockIdx.y];
    const int64_t T = (h + PT - 1) / PT;
    const int64_t ntri = T * (T + 1) / 2;
    int64_t t = blockIdx.x;
    int quad;  // 0: C11 = Low(U3); 1: C21 = U4; 2: C22 = Low(U5)
    int64_t I, J;
    if (t < ntri) {
        quad = 0;
        tri_tile(t, I, J);
    } else if (t < ntri + T * T) {
        quad = 1;
        t -= ntri;
        I = t / T;
        J = t - I * T;
    } else {
        quad = 2;
        t -= ntri + T * T;
        if (t >= ntri) return;
        tri_tile(t, I, J);
    }
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const uint32_t p = m.p;
    // transposed sources: tile (J, I) of P1 + P5 (quad 1) or of P4 (quad 2)
    const bool need_t = (quad == 1 && I <= J) || (quad == 2);
    if (need_t) {
        for (int q = 0; q < PT; q += 8) {
            int64_t rr = J * PT + ty + q, cc = I * PT + tx;
            uint32_t va = 0, vb = 0;
            if (rr < h && cc < h) {
                if (quad == 1) {
                    va = __ldg(nd.P1 + rr * nd.ldr + cc);
                    vb = __ldg(nd.P5 + rr * nd.ldr + cc);
                } else {
                    va = __ldg(nd.P4 + rr * nd.ldg + cc);
                }
            }
            sa[ty + q][tx] = va;
            sb[ty + q][tx] = vb;
        }
        __syncthreads();
    }
    int64_t r0, c0;  // output tile origin in the node's 2h×2h result
    if (quad == 0) {
        r0 = I * PT;
        c0 = J * PT;
    } else if (quad == 1) {
        r0 = h + I * PT;
        c0 = J * PT;
    } else {
        r0 = h + I * PT;
        c0 = h + J * PT;
    }
    for (int q = 0; q < PT; q += 8) {
        const int ly = ty + q;
        const int64_t i = I * PT + ly, j = J * PT + tx;
        uint32_t val = 0;
        if (i < h && j < h) {
            if (quad == 0) {
                if (j <= i) val = addm(__ldg(nd.P1 + i * nd.ldr + j), __ldg(nd.P2 + i * nd.ldr + j), p);
            } else if (quad == 1) {
                uint32_t u1;
                if (i >= j)
                    u1 = __ldg(nd.P1 + i * nd.ldr + j) + __ldg(nd.P5 + i * nd.ldr + j);
                else
                    u1 = sa[tx][ly] + sb[tx][ly];  // Up(U1) = Low(U1)ᵀ
                val = red(u1 + __ldg(nd.P4 + i * nd.ldg + j) + __ldg(nd.P3 + i * nd.ldg + j), m);
            } else if (j <= i) {
                val = red(__ldg(nd.P1 + i * nd.ldr + j) + __ldg(nd.P5 + i * nd.ldr + j) +
                              __ldg(nd.P4 + i * nd.ldg + j) + sa[tx][ly],
                          m);
            }
        }
        so[ly][tx] = val;
    }
    if (!nd.upper) {
        for (int q = 0; q < PT; q += 8) {
            const int ly = ty + q;
            const int64_t R = r0 + ly, Cc = c0 + tx;
            const bool inside = (I * PT + ly < h) && (J * PT + tx < h);
            if (inside && R < nd.vn && Cc < nd.vn && Cc <= R) nd.out[R * nd.ldo + Cc] = so[ly][tx];
        }
    } else {
        __syncthreads();
        // element (R, Cc) of the lower result goes to out[Cc][R]
        for (int q = 0; q < PT; q += 8) {
            const int lc = ty + q;  // column within the tile
            const int64_t R = r0 + tx, Cc = c0 + lc;
            const bool inside = (I * PT + tx < h) && (J * PT + lc < h);
            if (inside && R < nd.vn && Cc < nd.vn && Cc <= R) nd.out[Cc * nd.ldo + R] = so[tx][lc];
        }
    }
}

__global__ void k_zero_tri(uint32_t *C, int64_t n, int64_t ldc, int upper) {
    const int64_t total = n * n;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = idx / n, c = idx - r * n;
        if (upper ? c >= r : c <= r) C[r * ldc + c] = 0;
    }
}

int grid_for(int64_t work, int threads) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (work + threads - 1) / threads;
    int64_t cap = (int64_t)sms * 16;  // grid-stride beyond 16 blocks per SM
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

}  // namespace

cudaError_t launch_prep(const PrepNode *nodes_dev, int nnodes, int64_t h, int64_t w,
                        int64_t kpad, ModP mp, YConst y, DigitScheme ds, int arena_kind,
                        cudaStream_t st) {
    int64_t work = h * (kpad / 2) * nnodes;
    if (work == 0) return cudaSuccess;
    k_prep<<<grid_for(work, 256), 256, 0, st>>>(nodes_dev, nnodes, h, w, kpad, mp, y, ds,
                                                arena_kind);
    return cudaGetLastError();
}

cudaError_t launch_digitize(const DigitizeJob *jobs_dev, int njobs, int64_t max_work, ModP mp,
                            DigitScheme ds, int arena_kind, cudaStream_t st) {
    if (njobs == 0 || max_work == 0) return cudaSuccess;
    int gx = grid_for(max_work, 256);
    if (njobs > 1) gx = (int)std::min<int64_t>(gx, std::max<int64_t>(1, (max_work + 1023) / 1024));
    dim3 grid((unsigned)gx, (unsigned)njobs);
    k_digitize<<<grid, 256, 0, st>>>(jobs_dev, mp, ds, arena_kind);
    return cudaGetLastError();
}

cudaError_t launch_post(const PostNode *nodes_dev, int nnodes, int64_t h, ModP mp,
                        cudaStream_t st) {
    if (h == 0 || nnodes == 0) return cudaSuccess;
    int64_t T = (h + PT - 1) / PT;
    int64_t tiles = 2 * T * T + T;  // two triangles + one square
    dim3 grid((unsigned)tiles, (unsigned)nnodes);
    k_post<<<grid, 256, 0, st>>>(nodes_dev, h, mp);
    return cudaGetLastError();
}

cudaError_t launch_zero_tri(uint32_t *C, int64_t n, int64_t ldc, int upper, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_zero_tri<<<grid_for(n * n, 256), 256, 0, st>>>(C, n, ldc, upper);
    return cudaGetLastError();
}

}  // namespace fsk
