// Device helpers shared by the tensor-core leaf kernels: PTX wrappers for
// mbarriers, TMA, tcgen05 (MMA, commit, fences, tensor-memory loads), bounded
// waits, and the (K-span, digit pair, K-chunk) iterator.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "ffsyrk_internal.h"

namespace fsk {
namespace tc {

constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;
constexpr unsigned int ERR_WAIT = 1u;

__device__ __forceinline__ uint32_t su32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// One try with a suspend-time hint: the thread sleeps until the phase
// completes or SUSPEND_HINT_NS pass.  Waiters that poll instead (try_wait
// without a hint, or test_wait) keep the shared-memory pipe busy and slow
// the tensor core's operand reads: measured on GB300, a 128×256×16 MMA
// stream fed through a 4-stage ring ran at 85 % of its peak with polling
// waiters and at 98 % with sleeping ones.
constexpr uint32_t SUSPEND_HINT_NS = 1000000u;
__device__ __forceinline__ bool mbar_sleep_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity), "r"(SUSPEND_HINT_NS)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of `bar` with the given parity.  Returns false
// (after recording the error) if it ran out or another role gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          unsigned int *err) {
    if (mbar_sleep_try(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (true) {
        if (*abort_flag) return false;
        if (mbar_sleep_try(bar, parity)) return true;
        if (gtimer() - t0 > WAIT_LIMIT_NS) {
            *abort_flag = 1;
            if (err) atomicOr(err, ERR_WAIT);
            return false;
        }
    }
}
// Bounded wait used while shutting down: ignores the abort flag so that
// copies and MMAs already in flight can finish before the CTA exits.
__device__ __forceinline__ void mbar_drain(uint64_t *bar, uint32_t parity) {
    const uint64_t t0 = gtimer();
    while (!mbar_try(bar, parity))
        if (gtimer() - t0 > WAIT_LIMIT_NS / 4) return;
}

__device__ __forceinline__ void tma_load(void *dst, const void *tmap, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(su32(dst)),
        "l"(tmap), "r"(su32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Warm L2 with the box a later tma_load at (x, y) will copy; no completion
// signal, no shared memory.  Out-of-range boxes are ignored like loads are.
__device__ __forceinline__ void tma_prefetch_l2(const void *tmap, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(tmap), "r"(x),
                 "r"(y)
                 : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;              // leading byte offset (unused with swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
    d |= (uint64_t)1 << 46;              // version
    d |= (uint64_t)2 << 61;              // SWIZZLE_128B
    return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     su32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// 32 lanes × 16 consecutive 32-bit columns: thread t of the warp gets lane
// (base lane + t), columns [col, col + 16).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// The same wait with the loaded registers as its operands, so that no use of
// them can be scheduled before it (a load's registers are written when the
// wait completes, not when tcgen05.ld issues).
__device__ __forceinline__ void tmem_wait_ld_tied(uint32_t (&v)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]),
                   "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]),
                   "+r"(v[14]), "+r"(v[15])
                 :
                 : "memory");
}

// 16-column chunks [lo, hi) of an epilogue warp's 32 rows × (nch·16) columns
// that hold stored entries: rows below `rows`, columns below `cols`, and for
// a triangular product only chunks that reach the stored side of the
// diagonal.  Warp-uniform; chunks outside are neither loaded nor reduced.
__device__ __forceinline__ void live_chunks(const LeafProd &pr, int64_t rbase, int64_t cbase,
                                            int nch, int &lo, int &hi) {
    lo = 0;
    hi = 0;
    if (rbase >= pr.rows || cbase >= pr.cols) return;
    int64_t cmax = pr.cols;                                       // exclusive
    if (pr.tri == 1 && rbase + 32 < cmax) cmax = rbase + 32;      // c ≤ r
    int64_t h = (cmax - cbase + 15) / 16;
    hi = (int)(h < 0 ? 0 : (h > nch ? nch : h));
    if (pr.tri == 2 && rbase > cbase) {                           // c ≥ r
        int64_t l = (rbase - cbase) / 16;
        lo = (int)(l > nch ? nch : l);
    }
}

// Running sums of the epilogue are reduced lazily: Barrett with
// floor(2^32 / p) brings any uint32 sum into [0, 2p).
__device__ __forceinline__ uint32_t reduce_2p(uint32_t x, uint32_t p, uint32_t barrett) {
    return x - __umulhi(x, barrett) * p;
}
__device__ __forceinline__ uint32_t final_mod(uint32_t x, uint32_t p) { return x >= p ? x - p : x; }

// One epilogue thread's N residues (sums below 2p) to a row at dst, where
// dst + E0 is the first 16-byte aligned address: E0 leading scalar stores,
// 16-byte stores, then the remaining scalars.
template <int E0, int N>
__device__ __forceinline__ void store_row(uint32_t *dst, const uint32_t (&acc)[N], uint32_t p) {
#pragma unroll
    for (int e = 0; e < E0; ++e) dst[e] = final_mod(acc[e], p);
    constexpr int NV = (N - E0) / 4;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const int e = E0 + 4 * v;
        *reinterpret_cast<uint4 *>(dst + e) = make_uint4(final_mod(acc[e], p), final_mod(acc[e + 1], p),
                                                         final_mod(acc[e + 2], p), final_mod(acc[e + 3], p));
    }
#pragma unroll
    for (int e = E0 + 4 * NV; e < N; ++e) dst[e] = final_mod(acc[e], p);
}

// The same with the output update C ← α·R + β·C_old (OutScale mode 1), for
// a 16-byte aligned row.
template <int E0, int N>
__device__ __forceinline__ void store_row_scaled(uint32_t *dst, const uint32_t (&acc)[N], uint32_t p,
                                                 const OutScale &sc) {
    static_assert(E0 == 0 && N % 4 == 0, "aligned rows of whole 16-byte groups");
#pragma unroll
    for (int v = 0; v < N / 4; ++v) {
        const int e = 4 * v;
        uint4 *q = reinterpret_cast<uint4 *>(dst + e);
        const uint4 o = *q;
        *q = make_uint4(scale_out(final_mod(acc[e], p), o.x, sc, p), scale_out(final_mod(acc[e + 1], p), o.y, sc, p),
                        scale_out(final_mod(acc[e + 2], p), o.z, sc, p), scale_out(final_mod(acc[e + 3], p), o.w, sc, p));
    }
}
// One epilogue thread's row of N residues: full rows with 16-byte accesses
// from the first aligned column, edge rows element by element.  SCALED: the
// launch has a product that updates the caller's C (OutScale mode 1).
template <int N, bool SCALED>
__device__ __forceinline__ void store_tile_row(const LeafProd &pr, int64_t r, int64_t c0,
                                               const uint32_t (&acc)[N], uint32_t p) {
    if (r >= pr.rows) return;
    uint32_t *orow = pr.out + r * pr.ldo;
    const bool all_cols = c0 + N <= pr.cols;
    const bool tri_ok = pr.tri == 0 || (pr.tri == 1 && c0 + N - 1 <= r) || (pr.tri == 2 && c0 >= r);
    if (all_cols && tri_ok) {
        // rows of an odd ldc start at any 4-byte offset
        uint32_t *dst = orow + c0;
        const unsigned mis = (unsigned)((reinterpret_cast<uintptr_t>(dst) >> 2) & 3u);
        if constexpr (SCALED) {
            // the update reads C: 16-byte accesses on aligned rows only
            if (!pr.scale.mode) {
                for (int e = 0; e < N; ++e) dst[e] = final_mod(acc[e], p);
            } else if (mis == 0) {
                store_row_scaled<0, N>(dst, acc, p, pr.scale);
            } else {
#pragma unroll
                for (int e = 0; e < N; ++e) dst[e] = scale_out(final_mod(acc[e], p), dst[e], pr.scale, p);
            }
        } else {
            switch (mis) {
                case 0: store_row<0, N>(dst, acc, p); break;
                case 1: store_row<3, N>(dst, acc, p); break;
                case 2: store_row<2, N>(dst, acc, p); break;
                default: store_row<1, N>(dst, acc, p); break;
            }
        }
    } else {
#pragma unroll
        for (int e = 0; e < N; ++e) {
            const int64_t c = c0 + e;
            const bool keep = c < pr.cols && (pr.tri == 0 || (pr.tri == 1 && c <= r) || (pr.tri == 2 && c >= r));
            if (keep) {
                const uint32_t v = final_mod(acc[e], p);
                if constexpr (SCALED)
                    orow[c] = pr.scale.mode ? scale_out(v, orow[c], pr.scale, p) : v;
                else
                    orow[c] = v;
            }
        }
    }
}

// Instruction descriptor of tcgen05.mma kind::f16: D = f32, A = B = bf16,
// both K-major, shape M×N.
constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

}  // namespace tc
}  // namespace fsk
