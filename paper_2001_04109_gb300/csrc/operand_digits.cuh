// Signed digit split of residues into the tensor-core leaf's operand planes
// (arXiv 2001.04109, Section 4.2's delayed reduction, carried out here with
// exact small-integer digits in bf16).  Shared by every kernel that writes
// leaf operands, so that all of them encode digits the same way.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "ffsyrk_internal.h"

namespace fsk {

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
// Low signed digit of s in the scheme's base, leaving the rest in s.  Byte
// digits (base 256) are the low byte read as signed; for a balanced base b
// (two digits, |s| ≤ (p−1)/2 < 2^16, |s/b| < 182) the quotient is rounded to
// nearest: the float quotient s·(1/b) is off by less than 182·2^-23 < 2^-15,
// far less than the distance 1/b from a tie to any other value, so
// |digit| ≤ b/2 holds.
__device__ __forceinline__ int low_digit(int &s, const ModP &m) {
    if (m.dbase == 256u) {
        const int d = sbyte(s);
        s = (s - d) >> 8;
        return d;
    }
    const int q = __float2int_rn(__int2float_rn(s) * m.dinv);
    const int d = s - (int)m.dbase * q;
    s = q;
    return d;
}

// Byte t of the two's-complement symmetric residues s[0..3], packed in one
// word: the INT8 leaf's digit t (unsigned below the top digit, signed at
// the top; the digit count is chosen so that the top byte holds the sign).
template <int N>
__device__ __forceinline__ uint32_t byte_plane(const int (&sv)[N], int e0, int t) {
    uint32_t w = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) w |= ((uint32_t)(sv[e0 + e] >> (8 * t)) & 255u) << (8 * e);
    return w;
}

// A warp's share of the norm tables (see OperandDst::norm): the 32 lanes
// of a warp write 256 consecutive columns of one row (8 each), which is one
// block of the table.  Per row and operand the lanes' sums of squares of
// every plane are added across the warp; lane t keeps the running maximum
// of plane t.  `mask`: the lanes that took part (columns below kpad).
struct NormAcc {
    uint32_t mask = 0;
    uint32_t best = 0;       // lane t: plane t's largest row sum so far
    uint32_t *table = nullptr;
    int32_t nb = 0;
};
// The lanes of the warp whose first column is c0 that hold columns below kpad.
__device__ __forceinline__ uint32_t norm_lanes(int64_t c0, int64_t kpad) {
    const int64_t n = (kpad - c0 + 7) / 8;
    return n >= 32 ? 0xffffffffu : n <= 0 ? 0u : ((1u << n) - 1u);
}
// Lanes t < planes add their maximum into the table (block = c0 / 256).
// Every warp of every block that wrote this column block flushes into the
// same entries, so a kernel calls this once per thread at its end and its
// launcher keeps the number of blocks per column block small.
__device__ __forceinline__ void norm_flush(const NormAcc &acc, int planes, int64_t c0) {
    const int lane = threadIdx.x & 31;
    if (acc.table != nullptr && lane < planes && acc.best != 0)
        atomicMax(acc.table + (int64_t)lane * acc.nb + c0 / 256, acc.best);
}

// Store eight residues at (row r, columns c..c+7) of an operand: one
// 16-byte store per digit plane (bf16), two (uint32), or one 8-byte store
// per byte plane (INT8 leaf).  With `acc` and a destination that has a norm
// table, the warp also takes its row's sums of squares of every plane
// (integers ≤ 2^24: 256 columns of digits ≤ 256 in magnitude); every lane of
// acc.mask must make the same calls.
template <int D, int OK>
__device__ __forceinline__ void put8(const OperandDst &d, int64_t r, int64_t c, const uint32_t (&v)[8],
                                     const ModP &m, NormAcc *acc = nullptr) {
    if (d.arena == nullptr) return;
    if constexpr (OK == ARENA_U32) {
        uint4 *dst = reinterpret_cast<uint4 *>(static_cast<uint32_t *>(d.arena) + (d.row0 + r) * d.kpad + c);
        dst[0] = make_uint4(v[0], v[1], v[2], v[3]);
        dst[1] = make_uint4(v[4], v[5], v[6], v[7]);
    } else if constexpr (OK == ARENA_I8) {
        int sv[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) sv[e] = v[e] > m.half ? (int)v[e] - (int)m.p : (int)v[e];
        unsigned char *base = static_cast<unsigned char *>(d.arena);
#pragma unroll
        for (int t = 0; t < D; ++t)
            *reinterpret_cast<uint2 *>(base + (d.row0 + t * d.rpad + r) * d.kpad + c) =
                make_uint2(byte_plane(sv, 0, t), byte_plane(sv, 4, t));
    } else {
        // bf16 digit planes; with ARENA_BF16_KS also the Karatsuba sum planes
        // (0,1), (0,2), (1,2) after the D digits (every sum is ≤ 256 in
        // magnitude, so still an exact bf16 integer)
        int sv[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) sv[e] = v[e] > m.half ? (int)v[e] - (int)m.p : (int)v[e];
        // Every entry of a plane is an exact small integer in FP32 (|x| ≤ 256), so
        // the planes are formed, summed (Karatsuba planes) and squared (norms)
        // two entries at a time in packed FP32, all exactly: a sum of squares
        // stays below 2^24.  The bf16 encoding is the high half of the FP32 bits.
        uint32_t *base = static_cast<uint32_t *>(d.arena);
        const bool norms = acc != nullptr && d.norm != nullptr;
        const int lane = threadIdx.x & 31;
        // the float bits of 2^23 + q, summed over the acc->mask lanes, carry
        // popc(mask)·0x4B000000 beside Σq (mod 2^32; Σq ≤ 2^24)
        const uint32_t bias = norms ? (uint32_t)__popc(acc->mask) * 0x4B000000u : 0u;
        uint32_t mine = 0;  // this lane's plane's row sum (lane t: plane t)
        auto store_plane = [&](int t, const float2 (&x)[4]) {
            uint32_t w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) w[k] = __byte_perm(__float_as_uint(x[k].x), __float_as_uint(x[k].y), 0x7632);
            *reinterpret_cast<uint4 *>(base + (((d.row0 + t * d.rpad + r) * d.kpad + c) >> 1)) =
                make_uint4(w[0], w[1], w[2], w[3]);
            if (!norms) return;
            float2 q = make_float2(8388608.0f, 0.0f);  // 2^23: the sum's float bits are 0x4B000000 + q
#pragma unroll
            for (int k = 0; k < 4; ++k) q = __ffma2_rn(x[k], x[k], q);
            const uint32_t tot = __reduce_add_sync(acc->mask, __float_as_uint(__fadd_rn(q.x, q.y))) - bias;
            mine = lane == t ? tot : mine;
        };
        // The digits, in packed FP32 too, from s (|s| ≤ (p − 1)/2 < 2^23, exact in
        // FP32).  A low digit and the quotient that carries on are the same as
        // low_digit's: with byte digits the quotient is floor((s + 128)/256)
        // (s + 128 and its product with 2^-8 are exact, and adding 1.5·2^23
        // rounding down floors it), so s − 256·q is s's low byte read as
        // signed; with a balanced base b it is the float quotient s·(1/b)
        // rounded to nearest (adding 1.5·2^23, then taking it off, rounds any
        // |x| < 2^22 to an integer, ties to even).  s − b·q is exact: b·q and s
        // are integers below 2^24.
        const float2 M = make_float2(12582912.0f, 12582912.0f), negM = make_float2(-12582912.0f, -12582912.0f);
        float2 sf[4];
        if (m.p < (1u << 23)) {
            // |s| < 2^22: 1.5·2^23 + s is exact, so subtracting 1.5·2^23 leaves s
#pragma unroll
            for (int k = 0; k < 4; ++k)
                sf[k] = __fadd2_rn(make_float2(__int_as_float(0x4B400000 + sv[2 * k]),
                                               __int_as_float(0x4B400000 + sv[2 * k + 1])),
                                   negM);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) sf[k] = make_float2(__int2float_rn(sv[2 * k]), __int2float_rn(sv[2 * k + 1]));
        }
        float2 fd[D][4];
        if (m.dbase == 256u) {
            const float2 half = make_float2(128.0f, 128.0f), inv = make_float2(0.00390625f, 0.00390625f);
            const float2 negb = make_float2(-256.0f, -256.0f);
#pragma unroll
            for (int t = 0; t < D - 1; ++t)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 q = __fadd2_rn(__ffma2_rd(__fadd2_rn(sf[k], half), inv, M), negM);
                    fd[t][k] = __ffma2_rn(negb, q, sf[k]);
                    sf[k] = q;
                }
        } else {
            const float2 inv = make_float2(m.dinv, m.dinv);
            const float2 negb = make_float2(-(float)m.dbase, -(float)m.dbase);
#pragma unroll
            for (int t = 0; t < D - 1; ++t)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 q = __fadd2_rn(__fadd2_rn(__fmul2_rn(sf[k], inv), M), negM);
                    fd[t][k] = __ffma2_rn(negb, q, sf[k]);
                    sf[k] = q;
                }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) fd[D - 1][k] = sf[k];
#pragma unroll
        for (int t = 0; t < D; ++t) store_plane(t, fd[t]);
        if constexpr (OK == ARENA_BF16_KS) {
            int t = D;
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int j = i + 1; j < D; ++j, ++t) {
                    float2 sm[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) sm[k] = __fadd2_rn(fd[i][k], fd[j][k]);
                    store_plane(t, sm);
                }
        }
        if (norms) {
            acc->best = max(acc->best, mine);
            acc->table = d.norm;
            acc->nb = d.nb;
        }
    }
}

}  // namespace fsk
