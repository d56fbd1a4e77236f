// Throughput probes of the arithmetic pipes the leaves can use: the
// denominators of their rooflines where no measured peak is on file.
//
//   kind 0: mma.sync.m16n8k32 s8 × s8 → s32     (warp-level INT8 tensor path)
//   kind 1: mma.sync.m16n8k32 u8 × s8 → s32
//   kind 2: mma.sync.m16n8k32 u8 × u8 → s32
//   kind 3: mad.wide.u32 (32 × 32 → 64-bit multiply-add, CUDA cores)
//   kind 4: mma.sync.m16n8k16 bf16 × bf16 → f32  (the same warp-level path in bf16)
//
// Every thread runs `iters` rounds of 8 independent multiply-add chains on
// register operands (no memory traffic), then folds its accumulators into
// one word that is xor-ed into *sink so that nothing is optimised away.  The
// host times the launch; multiply-adds per launch are returned by
// probe_macs().
#include <cuda_runtime.h>
#include <stdint.h>

#include "ffsyrk_internal.h"

namespace fsk {
namespace {

constexpr int kChains = 8;

template <int KIND>
__global__ void __launch_bounds__(256) k_probe(int64_t iters, uint32_t seed, unsigned int *sink) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t a0 = seed ^ (t * 0x9E3779B9u), a1 = a0 * 3u + 1u, a2 = a0 ^ 0x5A5A5A5Au, a3 = a0 + 7u;
    uint32_t b0 = a0 * 5u, b1 = a1 ^ 0x3C3C3C3Cu;
    uint32_t fold = 0;
    if constexpr (KIND <= 2) {
        int32_t acc[kChains][4];
#pragma unroll
        for (int c = 0; c < kChains; ++c)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[c][r] = 0;
        for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                if constexpr (KIND == 0)
                    asm volatile(
                        "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                        "{%8,%9}, {%0,%1,%2,%3};"
                        : "+r"(acc[c][0]), "+r"(acc[c][1]), "+r"(acc[c][2]), "+r"(acc[c][3])
                        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
                else if constexpr (KIND == 1)
                    asm volatile(
                        "mma.sync.aligned.m16n8k32.row.col.s32.u8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                        "{%8,%9}, {%0,%1,%2,%3};"
                        : "+r"(acc[c][0]), "+r"(acc[c][1]), "+r"(acc[c][2]), "+r"(acc[c][3])
                        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
                else
                    asm volatile(
                        "mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                        "{%8,%9}, {%0,%1,%2,%3};"
                        : "+r"(acc[c][0]), "+r"(acc[c][1]), "+r"(acc[c][2]), "+r"(acc[c][3])
                        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
            }
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            fold ^= (uint32_t)(acc[c][0] + acc[c][1] + acc[c][2] + acc[c][3]);
    } else if constexpr (KIND == 3) {
        uint64_t acc[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = c;
        const uint32_t x = a0 | 1u, y = b0 | 3u;
        for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int c = 0; c < kChains; ++c)
                asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc[c]) : "r"(x + c), "r"(y));
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c) fold ^= (uint32_t)(acc[c] ^ (acc[c] >> 32));
    } else {
        float acc[kChains][4];
#pragma unroll
        for (int c = 0; c < kChains; ++c)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[c][r] = 0.f;
        // small bf16 integers so the sums stay finite
        const uint32_t one = 0x3F803F80u;
        for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int c = 0; c < kChains; ++c)
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                    "{%8,%9}, {%0,%1,%2,%3};"
                    : "+f"(acc[c][0]), "+f"(acc[c][1]), "+f"(acc[c][2]), "+f"(acc[c][3])
                    : "r"(one), "r"(one), "r"(one), "r"(one), "r"(one), "r"(one));
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            fold ^= __float_as_uint(acc[c][0] + acc[c][1] + acc[c][2] + acc[c][3]);
    }
    if (fold == 0x12345678u) atomicXor(sink, fold);  // practically never; keeps the work live
}

}  // namespace

// Multiply-adds of one probe launch of `blocks` × 256 threads, `iters` rounds.
double probe_macs(int kind, int64_t iters, int blocks) {
    const double warps = (double)blocks * 256 / 32;
    switch (kind) {
        case 0: case 1: case 2: return warps * iters * kChains * 16.0 * 8 * 32;  // m16n8k32 per warp
        case 3: return (double)blocks * 256 * iters * kChains;                  // one per thread
        case 4: return warps * iters * kChains * 16.0 * 8 * 16;                 // m16n8k16 per warp
        default: return 0;
    }
}

cudaError_t launch_probe(int kind, int64_t iters, int blocks, unsigned int *sink, cudaStream_t st) {
    const uint32_t seed = 0x2001u;
    switch (kind) {
        case 0: k_probe<0><<<blocks, 256, 0, st>>>(iters, seed, sink); break;
        case 1: k_probe<1><<<blocks, 256, 0, st>>>(iters, seed, sink); break;
        case 2: k_probe<2><<<blocks, 256, 0, st>>>(iters, seed, sink); break;
        case 3: k_probe<3><<<blocks, 256, 0, st>>>(iters, seed, sink); break;
        case 4: k_probe<4><<<blocks, 256, 0, st>>>(iters, seed, sink); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace fsk
