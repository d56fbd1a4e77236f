// Tensor-core leaf: out = X·Zᵀ mod p on GB300 5th-generation tensor cores.
//
// The leaf products of Algorithm 2 (arXiv 2001.04109, Section 3: P1, P2, P5
// at the leaves, P3 and P4 at every level) and the classical comparator.
//
// Exactness.  Residues are stored as D signed base-256 digits in bf16 (every
// integer of magnitude ≤ 256 is exact in bf16), so X·Zᵀ = Σ_{i,j}
// 256^(i+j)·X_i·Z_jᵀ.  Each X_i·Z_jᵀ is accumulated by tcgen05.mma
// (kind::f16, bf16 inputs, FP32 accumulators in tensor memory) over a K-chunk
// short enough that |partial sum| ≤ chunk·max|d_i|·max|d_j| ≤ 2^24: every
// partial sum is an integer exactly representable in FP32.  After each chunk
// the epilogue warps read the accumulator (tcgen05.ld), convert it to an
// integer, multiply by 256^(i+j) mod p and add into a per-element running
// residue held in registers (delayed modular reduction: one reduction per
// chunk instead of per product).
//
// Pipeline (one CTA per SM, persistent over a longest-first tile list):
//   warp 8  : TMA producer, 4 stages of a 128×64 X-tile and a 256×64 Z-tile,
//             128-byte swizzle;
//   warp 9  : MMA issuer (one thread), 128×256×16 MMAs into one of two TMEM
//             accumulators (2 × 256 columns), so the next chunk's MMAs run
//             while the epilogue drains the previous one;
//   warps 0-7: epilogue; warp w owns TMEM lanes 32·(w mod 4).. and columns
//             128·(w div 4).., i.e. one output row and 128 running residues per
//             thread, kept in registers across the whole K loop.
// Every mbarrier wait is bounded (about two seconds); a wait that runs out
// sets the error word, makes the CTA stop issuing work, drains what it has
// in flight and frees its tensor memory before returning.
#include <cuda.h>
#include <cuda_runtime.h>

#include "ffsyrk_internal.h"

namespace fsk {
namespace {

constexpr int BM = 128, BN = 256, BK = 64;
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;            // 16 KB
constexpr int B_BYTES = BN * BK * 2;            // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;  // 48 KB
constexpr int EPI_WARPS = 8;
constexpr int PRODUCER_WARP = 8, MMA_WARP = 9;
constexpr int NUM_THREADS = 32 * (EPI_WARPS + 2);  // no other warps: every warp has exactly one role
constexpr int EPI_COLS = BN / (EPI_WARPS / 4);  // columns per epilogue thread (128)
constexpr int LD_COLS = 16;  // TMEM columns per tcgen05.ld (128 residues + 16 loads fit 168 regs)
constexpr int TMEM_COLS = 512;
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;
constexpr unsigned int ERR_WAIT = 1u;

// instruction descriptor: D = f32, A = B = bf16, both K-major, N = 256, M = 128
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

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
// Bounded wait for the phase of `bar` with the given parity.  Returns false
// (after recording the error) if it ran out or another role gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          unsigned int *err) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    uint32_t it = 0;
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if ((++it & 255u) == 0) {
            if (*abort_flag) return false;
            if (gtimer() - t0 > WAIT_LIMIT_NS) {
                *abort_flag = 1;
                if (err) atomicOr(err, ERR_WAIT);
                return false;
            }
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

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(IDESC), "r"(acc)
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

// The (tile, K-span, digit pair, K-chunk) sequence every role walks in the
// same order.  K is cut into spans of SPAN_KB k-blocks; inside a span every
// digit pair (i, j) runs over it in chunks of at most chunk_kb[i][j].  Taking
// all pairs of one span before moving on reuses each operand's span D times
// while it is still in L2.
constexpr int SPAN_KB = 16;  // 1024 k-elements
struct UnitIter {
    int D;
    int i, j;          // digit pair
    int kb0, nkb;      // k-block range of this unit
    int span0, span1;  // current span [span0, span1)
    int kblocks;
    const DigitScheme *ds;
    __device__ void start(const DigitScheme &s, int kbl) {
        ds = &s;
        D = s.D;
        kblocks = kbl;
        i = 0;
        j = 0;
        span0 = 0;
        span1 = kbl < SPAN_KB ? kbl : SPAN_KB;
        kb0 = 0;
        set_len();
    }
    __device__ void set_len() {
        const int c = ds->chunk_kb[i][j];
        nkb = span1 - kb0 < c ? span1 - kb0 : c;
    }
    // advance; false when the tile is done
    __device__ bool next() {
        kb0 += nkb;
        if (kb0 < span1) {
            set_len();
            return true;
        }
        if (++j == D) {
            j = 0;
            if (++i == D) {
                i = 0;
                span0 = span1;
                if (span0 >= kblocks) return false;
                span1 = kblocks - span0 < SPAN_KB ? kblocks : span0 + SPAN_KB;
            }
        }
        kb0 = span0;
        set_len();
        return true;
    }
};

__global__ void __launch_bounds__(NUM_THREADS, 1) k_leaf_tc(const LeafProd *__restrict__ prods,
                                                             const LeafTile *__restrict__ tiles,
                                                             int ntiles,
                                                             const CUtensorMap *__restrict__ tmaps,
                                                             ModP m,
                                                             const __grid_constant__ DigitScheme ds,
                                                             unsigned int *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES];
    __shared__ __align__(8) uint64_t accf_bar[2], acce_bar[2], drain_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;

    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf_bar[b], 1);
            mbar_init(&acce_bar[b], EPI_WARPS);
        }
        mbar_init(&drain_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(&tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        fence_before();
    }
    __syncthreads();
    fence_after();
    const uint32_t tmem_base = tmem_slot;

    if (warp == PRODUCER_WARP) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const LeafTile tl = tiles[t];
                const LeafProd pr = prods[tl.prod];
                const CUtensorMap *tm = tmaps + pr.arena;
                // the descriptor was written by a host copy before this launch
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tm)
                             : "memory");
                UnitIter u;
                u.start(ds, pr.kblocks);
                do {
                    const int ya = (int)(pr.a_row0 + (int64_t)u.i * pr.plane_rows + (int64_t)tl.tm * BM);
                    const int yb = (int)(pr.b_row0 + (int64_t)u.j * pr.plane_rows + (int64_t)tl.tn * BN);
                    for (int kb = u.kb0; kb < u.kb0 + u.nkb; ++kb, ++it) {
                        const int s = it % STAGES;
                        const uint32_t ph = (it / STAGES) & 1u;
                        if (!mbar_wait(&empty_bar[s], ph ^ 1u, &abort_flag, err)) {
                            ok = false;
                            break;
                        }
                        unsigned char *sa = smem + s * STAGE_BYTES;
                        unsigned char *sb = sa + A_BYTES;
                        mbar_expect_tx(&full_bar[s], STAGE_BYTES);
                        tma_load(sa, tm, &full_bar[s], kb * BK, ya);
                        tma_load(sb, tm, &full_bar[s], kb * BK, yb);
                        tma_load(sb + B_BYTES / 2, tm, &full_bar[s], kb * BK, yb + BM);
                    }
                } while (ok && u.next());
            }
            if (!ok) {
                // let the copies already issued land before the CTA exits
                const uint32_t first = it > STAGES ? it - STAGES : 0;
                for (uint32_t q = first; q < it; ++q) mbar_drain(&full_bar[q % STAGES], (q / STAGES) & 1u);
            }
        }
    } else if (warp == MMA_WARP) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            uint32_t it = 0, unit = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const LeafProd pr = prods[tiles[t].prod];
                UnitIter u;
                u.start(ds, pr.kblocks);
                do {
                    const uint32_t b = unit & 1u;
                    if (!mbar_wait(&acce_bar[b], ((unit >> 1) & 1u) ^ 1u, &abort_flag, err)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t tmem_d = tmem_base + b * BN;
                    for (int kb = 0; kb < u.nkb; ++kb, ++it) {
                        const int s = it % STAGES;
                        if (!mbar_wait(&full_bar[s], (it / STAGES) & 1u, &abort_flag, err)) {
                            ok = false;
                            break;
                        }
                        fence_after();
                        const uint32_t sa = su32(smem + s * STAGE_BYTES);
                        const uint32_t sb = sa + A_BYTES;
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk)
                            mma_bf16(tmem_d, sdesc(sa + kk * 32), sdesc(sb + kk * 32),
                                     (kb > 0 || kk > 0) ? 1u : 0u);
                        mma_commit(&empty_bar[s]);
                    }
                    if (!ok) break;
                    mma_commit(&accf_bar[b]);
                    ++unit;
                } while (u.next());
            }
            // every MMA issued so far has completed once this barrier fires
            mma_commit(&drain_bar);
            mbar_drain(&drain_bar, 0);
        }
    } else if (warp < EPI_WARPS) {
        // ---------------- epilogue ----------------
        const uint32_t p = m.p, twop = 2 * m.p, off = ds.offset;
        const int quad = warp & 3, colq = warp >> 2;
        uint32_t unit = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const LeafTile tl = tiles[t];
            const LeafProd pr = prods[tl.prod];
            uint32_t acc[EPI_COLS];
#pragma unroll
            for (int e = 0; e < EPI_COLS; ++e) acc[e] = 0;
            UnitIter u;
            u.start(ds, pr.kblocks);
            do {
                const uint32_t b = unit & 1u;
                // warp-uniform outcome: tcgen05.ld below is .sync.aligned
                const bool got = mbar_wait(&accf_bar[b], (unit >> 1) & 1u, &abort_flag, err);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t w = ds.weight[u.i][u.j].w, wsh = ds.weight[u.i][u.j].w_sh;
                const uint32_t taddr =
                    tmem_base + b * BN + ((uint32_t)(quad * 32) << 16) + colq * EPI_COLS;
#pragma unroll
                for (int cc = 0; cc < EPI_COLS / LD_COLS; ++cc) {
                    uint32_t v[LD_COLS];
                    tmem_ld16(taddr + cc * LD_COLS, v);
                    tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < LD_COLS; ++e) {
                        // exact integer |x| ≤ 2^24 → shifted into [0, 2^26) → ·256^(i+j) mod p
                        const int xi = __float2int_rn(__uint_as_float(v[e]));
                        const uint32_t a = (uint32_t)(xi + (int)off);
                        const uint32_t q = __umulhi(a, wsh);
                        const uint32_t r = a * w - q * p;  // [0, 2p)
                        const uint32_t s = acc[cc * LD_COLS + e] + r;
                        acc[cc * LD_COLS + e] = min(s, s - twop);
                    }
                }
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce_bar[b]);
                ++unit;
            } while (u.next());
            if (!ok) break;
            // store the tile's residues
            const int64_t r = (int64_t)tl.tm * BM + quad * 32 + lane;
            const int64_t c0 = (int64_t)tl.tn * BN + colq * EPI_COLS;
            if (r < pr.rows) {
                uint32_t *orow = pr.out + r * pr.ldo;
                const bool all_cols = c0 + EPI_COLS <= pr.cols;
                const bool tri_ok = pr.tri == 0 || (pr.tri == 1 && c0 + EPI_COLS - 1 <= r) ||
                                    (pr.tri == 2 && c0 >= r);
                const bool aligned = ((reinterpret_cast<uintptr_t>(orow + c0) & 15u) == 0);
                if (all_cols && tri_ok && aligned) {
#pragma unroll
                    for (int e = 0; e < EPI_COLS; e += 4) {
                        uint4 v4;
                        v4.x = acc[e] >= p ? acc[e] - p : acc[e];
                        v4.y = acc[e + 1] >= p ? acc[e + 1] - p : acc[e + 1];
                        v4.z = acc[e + 2] >= p ? acc[e + 2] - p : acc[e + 2];
                        v4.w = acc[e + 3] >= p ? acc[e + 3] - p : acc[e + 3];
                        *reinterpret_cast<uint4 *>(orow + c0 + e) = v4;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < EPI_COLS; ++e) {
                        const int64_t c = c0 + e;
                        const bool keep = c < pr.cols && (pr.tri == 0 || (pr.tri == 1 && c <= r) ||
                                                          (pr.tri == 2 && c >= r));
                        if (keep) orow[c] = acc[e] >= p ? acc[e] - p : acc[e];
                    }
                }
            }
        }
    }
    __syncthreads();
    if (warp == MMA_WARP) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

}  // namespace

int leaf_tc_bm() { return BM; }
int leaf_tc_bn() { return BN; }

cudaError_t launch_leaf_tc(const TcLaunch &L, int num_sms, cudaStream_t st) {
    if (L.ntiles == 0) return cudaSuccess;
    const int smem = STAGES * STAGE_BYTES + 1024;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(k_leaf_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    const int grid = L.ntiles < num_sms ? L.ntiles : num_sms;
    k_leaf_tc<<<grid, NUM_THREADS, smem, st>>>(L.prods, L.tiles, L.ntiles,
                                               reinterpret_cast<const CUtensorMap *>(L.tmaps), L.mp,
                                               L.ds, L.err);
    return cudaGetLastError();
}

}  // namespace fsk
