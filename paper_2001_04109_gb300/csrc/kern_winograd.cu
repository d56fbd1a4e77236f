// Block additions of Algorithm 1 (arXiv 2001.04109, Section 2: the Winograd
// variant of Strassen's product, C = W(A, B)) for the general products
// P3 = X22·S4ᵀ and P4 = S1·S2ᵀ of Algorithm 2, as the paper's fsyrk does
// (Section 4.2, the G-i variants).
//
// A general product here is L·Rᵀ with L and R row-major (the leaf's
// operand form), i.e. W(A, B) with A = L and B = Rᵀ, so B's blocks are
// b11 = R11ᵀ, b12 = R21ᵀ, b21 = R12ᵀ, b22 = R22ᵀ.  One level splits L and R
// into 2×2 blocks and produces, for p_m = L_m·R_mᵀ (m = 1..7):
//
//   left  L_m: a11, a12, a22, s1 = a11 − a21, s3 = s2 − a11,
//              s4 = a12 − s3, s2 = a21 + a22;
//   right R_m: R11, R12, R12 − T3, T1, T3, R22, T2 with
//              T1 = R22 − R21 (t1ᵀ), T2 = R21 − R11 (t2ᵀ), T3 = R11 + T1 (t3ᵀ),
//              R12 − T3 = t4ᵀ;
//
// and the post-additions c1 = p1 + p5, c2 = c1 + p4, c3 = p1 + p2,
// c4 = c2 + p3, c5 = c2 + p7, c6 = c1 + p7, c7 = c6 + p6 give
// C = [[c3, c7], [c4, c5]].  Both kernels stream: every input is read once,
// every output written once, 16-byte accesses along rows.
#include <algorithm>

#include "ffsyrk_internal.h"
#include "operand_digits.cuh"

namespace fsk {
namespace {

constexpr int SWP_THREADS = 128;
constexpr int SWP_COLS = 8;  // columns per thread (two 16-byte loads per block row)
constexpr int SWQ_THREADS = 256;

__device__ __forceinline__ uint32_t addp(uint32_t a, uint32_t b, uint32_t p) {
    const uint32_t r = a + b;
    return r >= p ? r - p : r;
}
__device__ __forceinline__ uint32_t subp(uint32_t a, uint32_t b, uint32_t p) {
    const uint32_t r = a + (p - b);
    return r >= p ? r - p : r;
}
__device__ __forceinline__ void allow_dependents_sw() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// row r, columns c..c+7 of a uint32 block whose row stride is a multiple of
// 4; `n4` of the two 4-column halves lie inside the block (0, 1 or 2)
__device__ __forceinline__ void ld8(const uint32_t *base, int64_t ld, int64_t r, int64_t c, int n4,
                                    uint32_t (&v)[8]) {
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
        if (hf < n4) {
            const uint4 a = __ldg(reinterpret_cast<const uint4 *>(base + r * ld + c + 4 * hf));
            v[4 * hf] = a.x;
            v[4 * hf + 1] = a.y;
            v[4 * hf + 2] = a.z;
            v[4 * hf + 3] = a.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) v[4 * hf + e] = 0u;
        }
    }
}

// One level of pre-additions: job z splits its hh·2 × ww·2 uint32 operand
// into 2×2 blocks and writes the 7 operands of p1..p7 (left side or right
// side), each hh × kpad with zeros in columns ≥ ww.
template <int D, int OK>
__global__ void __launch_bounds__(SWP_THREADS) k_sw_pre(const SwPreJob *__restrict__ jobs,
                                                        int64_t hh, int64_t ww, int64_t kpad,
                                                        ModP m) {
    allow_dependents_sw();
    const int64_t c = SWP_COLS * ((int64_t)blockIdx.x * SWP_THREADS + threadIdx.x);
    if (c >= kpad) return;
    const SwPreJob &jb = jobs[blockIdx.z];
    const int64_t c0 = c - SWP_COLS * (threadIdx.x & 31);  // the warp's first column
    NormAcc acc;
    acc.mask = norm_lanes(c0, kpad);
    const uint32_t p = m.p;
    // ww is a multiple of 4: each 4-column half lies wholly inside or outside
    const int n4 = c >= ww ? 0 : (c + 4 >= ww ? 1 : 2);
    for (int64_t r = blockIdx.y; r < hh; r += gridDim.y) {
        uint32_t x11[8], x12[8], x21[8], x22[8];
        ld8(jb.X, jb.ldx, r, c, n4, x11);
        ld8(jb.X, jb.ldx, r, ww + c, n4, x12);
        ld8(jb.X, jb.ldx, hh + r, c, n4, x21);
        ld8(jb.X, jb.ldx, hh + r, ww + c, n4, x22);
        uint32_t o[3][8];
        if (jb.side == 0) {
            // left operands: a11, a12, a22 as they are; s1, s3, s4, s2
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const uint32_t s2 = addp(x21[e], x22[e], p);
                const uint32_t s3 = subp(s2, x11[e], p);
                o[0][e] = subp(x11[e], x21[e], p);  // s1
                o[1][e] = s3;
                o[2][e] = subp(x12[e], s3, p);      // s4
                x21[e] = s2;                        // x21 is not an output: reuse for s2
            }
            put8<D, OK>(jb.dst[0], r, c, x11, m, &acc);
            put8<D, OK>(jb.dst[1], r, c, x12, m, &acc);
            put8<D, OK>(jb.dst[2], r, c, x22, m, &acc);
            put8<D, OK>(jb.dst[3], r, c, o[0], m, &acc);
            put8<D, OK>(jb.dst[4], r, c, o[1], m, &acc);
            put8<D, OK>(jb.dst[5], r, c, o[2], m, &acc);
            put8<D, OK>(jb.dst[6], r, c, x21, m, &acc);
        } else {
            // right operands: R11, R12, R12 − T3, T1, T3, R22, T2
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const uint32_t t1 = subp(x22[e], x21[e], p);
                const uint32_t t2 = subp(x21[e], x11[e], p);
                const uint32_t t3 = addp(x11[e], t1, p);
                o[0][e] = subp(x12[e], t3, p);  // t4ᵀ
                o[1][e] = t1;
                o[2][e] = t3;
                x21[e] = t2;  // x21 is not an output: reuse for T2
            }
            put8<D, OK>(jb.dst[0], r, c, x11, m, &acc);
            put8<D, OK>(jb.dst[1], r, c, x12, m, &acc);
            put8<D, OK>(jb.dst[2], r, c, o[0], m, &acc);
            put8<D, OK>(jb.dst[3], r, c, o[1], m, &acc);
            put8<D, OK>(jb.dst[4], r, c, o[2], m, &acc);
            put8<D, OK>(jb.dst[5], r, c, x22, m, &acc);
            put8<D, OK>(jb.dst[6], r, c, x21, m, &acc);
        }
    }
    norm_flush(acc, OK == ARENA_BF16_KS ? D + D * (D - 1) / 2 : D, c0);
}

// One level of post-additions: job z combines its 7 hh × hh products into
// the 2hh × 2hh result [[c3, c7], [c4, c5]].  Four columns per thread.
__global__ void __launch_bounds__(SWQ_THREADS) k_sw_post(const SwPostJob *__restrict__ jobs,
                                                         int64_t hh, ModP m) {
    const int64_t c = 4 * ((int64_t)blockIdx.x * SWQ_THREADS + threadIdx.x);
    if (c >= hh) return;
    const SwPostJob &jb = jobs[blockIdx.z];
    const uint32_t p = m.p;
    const int64_t ldc = 2 * hh;
    for (int64_t r = blockIdx.y; r < hh; r += gridDim.y) {
        uint32_t v[7][4];
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            const uint4 a = __ldg(reinterpret_cast<const uint4 *>(jb.P[q] + r * hh + c));
            v[q][0] = a.x;
            v[q][1] = a.y;
            v[q][2] = a.z;
            v[q][3] = a.w;
        }
        uint32_t c3[4], c4[4], c5[4], c7[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const uint32_t c1 = addp(v[0][e], v[4][e], p);  // p1 + p5
            const uint32_t c2 = addp(c1, v[3][e], p);       // c1 + p4
            c3[e] = addp(v[0][e], v[1][e], p);              // p1 + p2
            c4[e] = addp(c2, v[2][e], p);                   // c2 + p3
            c5[e] = addp(c2, v[6][e], p);                   // c2 + p7
            const uint32_t c6 = addp(c1, v[6][e], p);       // c1 + p7
            c7[e] = addp(c6, v[5][e], p);                   // c6 + p6
        }
        uint32_t *row0 = jb.C + r * ldc + c, *row1 = jb.C + (hh + r) * ldc + c;
        *reinterpret_cast<uint4 *>(row0) = make_uint4(c3[0], c3[1], c3[2], c3[3]);
        *reinterpret_cast<uint4 *>(row0 + hh) = make_uint4(c7[0], c7[1], c7[2], c7[3]);
        *reinterpret_cast<uint4 *>(row1) = make_uint4(c4[0], c4[1], c4[2], c4[3]);
        *reinterpret_cast<uint4 *>(row1 + hh) = make_uint4(c5[0], c5[1], c5[2], c5[3]);
    }
}

template <int D, int OK>
cudaError_t launch_pre_t(dim3 grid, cudaStream_t st, const SwPreJob *jobs, int64_t hh, int64_t ww,
                         int64_t kpad, ModP mp) {
    k_sw_pre<D, OK><<<grid, SWP_THREADS, 0, st>>>(jobs, hh, ww, kpad, mp);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sw_pre(const SwPreJob *jobs_dev, int njobs, int64_t hh, int64_t ww,
                          int64_t kpad, ModP mp, DigitScheme ds, int out_kind, cudaStream_t st) {
    if (njobs == 0 || hh == 0 || kpad == 0) return cudaSuccess;
    const int64_t gx = (kpad / SWP_COLS + SWP_THREADS - 1) / SWP_THREADS;
    const int64_t gy = std::min<int64_t>(hh, std::max<int64_t>(1, 152 * 24 / (gx * njobs)));
    dim3 grid((unsigned)gx, (unsigned)std::max<int64_t>(gy, 1), (unsigned)njobs);
    if (out_kind == ARENA_U32) return launch_pre_t<1, ARENA_U32>(grid, st, jobs_dev, hh, ww, kpad, mp);
    if (out_kind == ARENA_BF16_KS) {
        switch (ds.D) {
            case 2: return launch_pre_t<2, ARENA_BF16_KS>(grid, st, jobs_dev, hh, ww, kpad, mp);
            case 3: return launch_pre_t<3, ARENA_BF16_KS>(grid, st, jobs_dev, hh, ww, kpad, mp);
        }
        return cudaErrorInvalidValue;
    }
    if (out_kind == ARENA_I8) {
        switch (ds.D) {
            case 1: return launch_pre_t<1, ARENA_I8>(grid, st, jobs_dev, hh, ww, kpad, mp);
            case 2: return launch_pre_t<2, ARENA_I8>(grid, st, jobs_dev, hh, ww, kpad, mp);
            case 3: return launch_pre_t<3, ARENA_I8>(grid, st, jobs_dev, hh, ww, kpad, mp);
        }
        return cudaErrorInvalidValue;
    }
    switch (ds.D) {
        case 1: return launch_pre_t<1, ARENA_BF16>(grid, st, jobs_dev, hh, ww, kpad, mp);
        case 2: return launch_pre_t<2, ARENA_BF16>(grid, st, jobs_dev, hh, ww, kpad, mp);
        case 3: return launch_pre_t<3, ARENA_BF16>(grid, st, jobs_dev, hh, ww, kpad, mp);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_sw_post(const SwPostJob *jobs_dev, int njobs, int64_t hh, ModP mp,
                           cudaStream_t st) {
    if (njobs == 0 || hh == 0) return cudaSuccess;
    const int64_t gx = (hh / 4 + SWQ_THREADS - 1) / SWQ_THREADS;
    const int64_t gy = std::min<int64_t>(hh, std::max<int64_t>(1, 152 * 16 / (gx * njobs)));
    dim3 grid((unsigned)gx, (unsigned)std::max<int64_t>(gy, 1), (unsigned)njobs);
    k_sw_post<<<grid, SWQ_THREADS, 0, st>>>(jobs_dev, hh, mp);
    return cudaGetLastError();
}

}  // namespace fsk
