// Tensor-core leaf on CTA pairs: out = X·Zᵀ mod p with tcgen05.mma.cta_group::2.
//
// Same arithmetic as the one-CTA leaf (exact signed base-256 digits in bf16,
// FP32 accumulation over K-chunks bounded by 2^24, delayed reduction mod p
// in the epilogue), on 256×256 output tiles computed by a cluster of two
// CTAs on two SMs.  CTA r of the pair stages rows [128r, 128r + 128) of the
// X tile and rows [128r, 128r + 128) of the Z tile (the tile's columns); one
// 256×256×16 MMA issued by the even CTA reads both CTAs' shared memory, and
// each CTA's tensor memory receives its own 128 rows × 256 columns.  Per SM
// and per k-block this stages 32 KB instead of the 48 KB a one-CTA 128×256
// tile needs for the same multiply-adds, which relieves shared memory.
//
// Synchronisation across the pair:
//   full[s]   lives in the even CTA; its producer expects both CTAs' bytes,
//             and both CTAs' TMA loads (cta_group::2) complete on it;
//   empty[s]  in both CTAs, signalled by a multicast MMA commit;
//   accf[b]   in both CTAs, signalled by a multicast MMA commit;
//   acce[b]   in the even CTA, 16 arrivals: every epilogue warp of both CTAs.
// Every wait is bounded (mbar_wait); the pair meets at cluster barriers after
// initialising its barriers and before releasing tensor memory.
#include <cuda.h>
#include <cuda_runtime.h>

#include "ffsyrk_internal.h"
#include "tc_common.cuh"

namespace fsk {
namespace {

using namespace tc;

constexpr int BM = 256, BN = 256, BK = 64;  // pair tile
constexpr int ROWS = 128;                    // rows of X and of Z staged per CTA
constexpr int STAGES = 6;
constexpr int A_BYTES = ROWS * BK * 2;              // 16 KB
constexpr int B_BYTES = ROWS * BK * 2;              // 16 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;      // 32 KB per CTA
constexpr int EPI_WARPS = 8;
constexpr int PRODUCER_WARP = 8, MMA_WARP = 9;
constexpr int NUM_THREADS = 32 * (EPI_WARPS + 2);
constexpr int EPI_COLS = BN / (EPI_WARPS / 4);      // 128 columns per epilogue thread
constexpr int LD_COLS = 16;
constexpr int TMEM_COLS = 512;
constexpr uint32_t IDESC = idesc_bf16(BM, BN);

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t mapa_rank(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Arrive on a barrier of the pair (cluster address).  The epilogue's only
// obligation to the MMA issuer is that its tensor-memory reads are complete
// (tcgen05.wait::ld and fence::before_thread_sync precede the arrive), so no
// cluster-scope release of ordinary memory is needed.
__device__ __forceinline__ void arrive_remote(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
// TMA load into this CTA's shared memory, completing on a barrier that may
// live in the peer CTA (cluster address).
__device__ __forceinline__ void tma_load_pair(void *dst, const void *tmap, uint32_t bar_cluster,
                                              int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(su32(dst)),
        "l"(tmap), "r"(bar_cluster), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void mma_pair(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(IDESC), "r"(acc)
        : "memory");
}
// Arrive on the barrier at this offset in every CTA of `mask` once all
// previously issued MMAs of this thread have completed.
__device__ __forceinline__ void commit_pair(uint64_t *bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
        " [%0], %1;" ::"r"(su32(bar)),
        "h"(mask)
        : "memory");
}

// LAZY: as in the one-SM leaf, running sums grow unreduced when no tile has
// more units than ds.lazy_units.
template <bool LAZY, bool SCALED>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NUM_THREADS, 1)
    k_leaf_tc2(const LeafProd *__restrict__ prods, const LeafTile *__restrict__ tiles,
               const LeafSeg *__restrict__ segs, int ntiles, const CUtensorMap *__restrict__ tmaps,
               ModP m,
               const __grid_constant__ DigitScheme ds, unsigned int *err,
               const LeafPiece *__restrict__ pieces, const int32_t *__restrict__ entries,
               uint32_t *part, unsigned int *part_ctr) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES];
    __shared__ __align__(8) uint64_t accf_bar[2], acce_bar[2], drain_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;

    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
    // this pair's items: its own list (tiles and pieces of tiles, K range
    // [sx0, sx1) of the schedule), or every npairs-th tile
    const int q0 = entries ? entries[pair] : pair;
    const int q1 = entries ? entries[pair + 1] : ntiles;
    const int qstep = entries ? 1 : npairs;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf_bar[b], 1);
            mbar_init(&acce_bar[b], 2 * EPI_WARPS);
        }
        mbar_init(&drain_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == MMA_WARP) {
        // both CTAs of the pair allocate the same columns together
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(&tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        fence_before();
    }
    __syncthreads();
    cluster_sync();  // the peer's barriers are initialised before any remote use
    fence_after();
    const uint32_t tmem_base = tmem_slot;

    if (warp == PRODUCER_WARP) {
        // ---------------- TMA producer (both CTAs) ----------------
        if (lane == 0) {
            // the operands may still be being written by the preceding grid
            asm volatile("griddepcontrol.wait;" ::: "memory");
            uint32_t it = 0;
            bool ok = true;
            for (int t = q0; t < q1 && ok; t += qstep) {
                const LeafTile tl = tiles[t];
                const LeafProd pr = prods[tl.prod];
                const int sx0 = pieces ? pieces[t].sx0 : 0, sx1 = pieces ? pieces[t].sx1 : pr.nseg;
                const CUtensorMap *tm = tmaps + pr.arena;
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tm)
                             : "memory");
                for (int sx = sx0; sx < sx1 && ok; ++sx) {
                    const LeafSeg sg = segs[pr.seg0 + sx];
                    const int ya = (int)(pr.a_row0 + (int64_t)(sg.ij >> 4) * pr.plane_rows +
                                         (int64_t)tl.tm * BM + rank * ROWS);
                    const int yb = (int)(pr.b_row0 + (int64_t)(sg.ij & 15) * pr.plane_rows +
                                         (int64_t)tl.tn * BN + rank * ROWS);
                    for (int kb = sg.kb0; kb < sg.kb0 + sg.nkb; ++kb, ++it) {
                        const int s = it % STAGES;
                        const uint32_t ph = (it / STAGES) & 1u;
                        if (!mbar_wait(&empty_bar[s], ph ^ 1u, &abort_flag, err)) {
                            ok = false;
                            break;
                        }
                        unsigned char *sa = smem + s * STAGE_BYTES;
                        unsigned char *sb = sa + A_BYTES;
                        const uint32_t fb = mapa_rank(su32(&full_bar[s]), 0);
                        if (rank == 0) mbar_expect_tx(&full_bar[s], 2 * STAGE_BYTES);
                        tma_load_pair(sa, tm, fb, kb * BK, ya);
                        tma_load_pair(sb, tm, fb, kb * BK, yb);
                    }
                }
            }
            if (!ok && rank == 0) {
                const uint32_t first = it > STAGES ? it - STAGES : 0;
                for (uint32_t q = first; q < it; ++q) mbar_drain(&full_bar[q % STAGES], (q / STAGES) & 1u);
            }
        }
    } else if (warp == MMA_WARP) {
        // ---------------- MMA issuer (even CTA only) ----------------
        if (lane == 0 && rank == 0) {
            uint32_t it = 0, unit = 0;
            bool ok = true;
            for (int t = q0; t < q1 && ok; t += qstep) {
                const LeafProd pr = prods[tiles[t].prod];
                const int sx0 = pieces ? pieces[t].sx0 : 0, sx1 = pieces ? pieces[t].sx1 : pr.nseg;
                bool open = false;  // a unit's accumulator is being filled
                uint32_t b = 0, tmem_d = 0;
                for (int sx = sx0; sx < sx1; ++sx) {
                    const LeafSeg sg = segs[pr.seg0 + sx];
                    if (sg.first) {
                        if (open) {
                            commit_pair(&accf_bar[b], 0x3);
                            ++unit;
                        }
                        b = unit & 1u;
                        if (!mbar_wait(&acce_bar[b], ((unit >> 1) & 1u) ^ 1u, &abort_flag, err)) {
                            ok = false;
                            break;
                        }
                        fence_after();
                        tmem_d = tmem_base + b * BN;
                        open = true;
                    }
                    for (int kb = 0; kb < sg.nkb; ++kb, ++it) {
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
                            mma_pair(tmem_d, sdesc(sa + kk * 32), sdesc(sb + kk * 32),
                                     (sg.first && kb == 0 && kk == 0) ? 0u : 1u);
                        commit_pair(&empty_bar[s], 0x3);
                    }
                    if (!ok) break;
                }
                if (!ok) break;
                if (open) {
                    commit_pair(&accf_bar[b], 0x3);
                    ++unit;
                }
            }
            commit_pair(&drain_bar, 0x1);
            mbar_drain(&drain_bar, 0);
        }
    } else if (warp < EPI_WARPS) {
        // ---------------- epilogue (both CTAs) ----------------
        const uint32_t p = m.p, twop = 2 * m.p, off = ds.offset;
        const int quad = warp & 3, colq = warp >> 2;
        const uint32_t acce_leader[2] = {mapa_rank(su32(&acce_bar[0]), 0),
                                         mapa_rank(su32(&acce_bar[1]), 0)};
        uint32_t unit = 0;
        bool ok = true;
        for (int t = q0; t < q1 && ok; t += qstep) {
            const LeafTile tl = tiles[t];
            const LeafProd pr = prods[tl.prod];
            const int sx0 = pieces ? pieces[t].sx0 : 0, sx1 = pieces ? pieces[t].sx1 : pr.nseg;
            uint32_t acc[EPI_COLS];
#pragma unroll
            for (int e = 0; e < EPI_COLS; ++e) acc[e] = 0;
            int lo = 0, hi = 0;  // 16-column chunks of this warp that hold stored entries
            live_chunks(pr, (int64_t)tl.tm * BM + rank * ROWS + quad * 32, (int64_t)tl.tn * BN + colq * EPI_COLS,
                        EPI_COLS / LD_COLS, lo, hi);
            for (int sx = sx0; sx < sx1; ++sx) {
                const LeafSeg sg = segs[pr.seg0 + sx];
                if (!sg.first) continue;  // one drain per unit
                const uint32_t b = unit & 1u;
                const bool got = mbar_wait(&accf_bar[b], (unit >> 1) & 1u, &abort_flag, err);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    break;
                }
                fence_after();
                const MulConst wt = ds.weight[sg.ij >> 4][sg.ij & 15];
                const uint32_t w = wt.w, wsh = wt.w_sh;
                const uint32_t taddr =
                    tmem_base + b * BN + ((uint32_t)(quad * 32) << 16) + colq * EPI_COLS;
#pragma unroll
                for (int cc = 0; cc < EPI_COLS / LD_COLS; ++cc) {
                    if (cc < lo || cc >= hi) continue;
                    uint32_t v[LD_COLS];
                    tmem_ld16(taddr + cc * LD_COLS, v);
                    tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < LD_COLS; ++e) {
                        // exact integer |x| ≤ 2^24 → shifted into [0, 2^26) → ·weight mod p
                        const int xi = __float2int_rn(__uint_as_float(v[e]));
                        const uint32_t a = (uint32_t)(xi + (int)off);
                        const uint32_t q = __umulhi(a, wsh);
                        const uint32_t r = a * w - q * p;  // [0, 2p)
                        if constexpr (LAZY) {
                            acc[cc * LD_COLS + e] += r;
                        } else {
                            const uint32_t s = acc[cc * LD_COLS + e] + r;
                            acc[cc * LD_COLS + e] = min(s, s - twop);
                        }
                    }
                }
                fence_before();
                __syncwarp();
                if (lane == 0) arrive_remote(acce_leader[b]);
                ++unit;
            }
            if (!ok) break;
            if constexpr (LAZY) {
#pragma unroll
                for (int e = 0; e < EPI_COLS; ++e) acc[e] = reduce_2p(acc[e], p, m.barrett);
            }
            const LeafPiece pc = pieces ? pieces[t] : LeafPiece{0, 0, -1, 0, 1};
            if (pc.slot0 >= 0) {
                // a piece of a shared tile: this CTA publishes the residues of
                // its 128 rows; per warp and CTA rank, the piece that finishes
                // last adds the others' and stores (no waiting on other pairs)
                uint32_t *mine = part + ((int64_t)(2 * (pc.slot0 + pc.j) + rank) * (ROWS * BN)) +
                                 threadIdx.x * EPI_COLS;
#pragma unroll
                for (int e = 0; e < EPI_COLS; e += 4) {
                    uint4 v4;
                    v4.x = acc[e] >= p ? acc[e] - p : acc[e];
                    v4.y = acc[e + 1] >= p ? acc[e + 1] - p : acc[e + 1];
                    v4.z = acc[e + 2] >= p ? acc[e + 2] - p : acc[e + 2];
                    v4.w = acc[e + 3] >= p ? acc[e + 3] - p : acc[e + 3];
                    *reinterpret_cast<uint4 *>(mine + e) = v4;
                }
                __threadfence();
                __syncwarp();
                unsigned int *ctr = &part_ctr[(2 * pc.slot0 + rank) * EPI_WARPS + warp];
                unsigned int prev = 0;
                if (lane == 0) prev = atomicAdd(ctr, 1u);
                prev = __shfl_sync(0xffffffffu, prev, 0);
                if (prev != (unsigned)(pc.npieces - 1)) continue;
                __threadfence();
#pragma unroll 1
                for (int q = 0; q < pc.npieces; ++q) {
                    if (q == pc.j) continue;
                    const uint32_t *other = part +
                                            ((int64_t)(2 * (pc.slot0 + q) + rank) * (ROWS * BN)) +
                                            threadIdx.x * EPI_COLS;
#pragma unroll
                    for (int e = 0; e < EPI_COLS; e += 4) {
                        const uint4 o = __ldcg(reinterpret_cast<const uint4 *>(other + e));
                        // acc < 2p and o < p: one conditional subtract keeps it below 2p
                        const uint32_t s0 = acc[e] + o.x, s1 = acc[e + 1] + o.y,
                                       s2 = acc[e + 2] + o.z, s3 = acc[e + 3] + o.w;
                        acc[e] = min(s0, s0 - twop);
                        acc[e + 1] = min(s1, s1 - twop);
                        acc[e + 2] = min(s2, s2 - twop);
                        acc[e + 3] = min(s3, s3 - twop);
                    }
                }
                if (lane == 0) *ctr = 0;  // ready for the next launch
            }
            store_tile_row<EPI_COLS, SCALED>(pr, (int64_t)tl.tm * BM + rank * ROWS + quad * 32 + lane,
                                     (int64_t)tl.tn * BN + colq * EPI_COLS, acc, p);
        }
    }
    __syncthreads();
    cluster_sync();  // no CTA leaves while its peer may still signal it
    if (warp == MMA_WARP) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

}  // namespace

int leaf_tc2_bm() { return BM; }
int leaf_tc2_bn() { return BN; }

cudaError_t launch_leaf_tc2(const TcLaunch &L, int num_sms, cudaStream_t st) {
    if (L.ntiles == 0) return cudaSuccess;
    const int smem = STAGES * STAGE_BYTES + 1024;
    // the dynamic shared-memory opt-in and the pairs that fit at once, per device
    static DeviceOnce attr_once;
    int max_pairs = 0;
    cudaError_t ea = once_per_device(attr_once, &max_pairs, [smem, num_sms](int *out) {
        cudaError_t e = cudaSuccess;
        for (auto fn : {k_leaf_tc2<true, false>, k_leaf_tc2<false, false>, k_leaf_tc2<true, true>, k_leaf_tc2<false, true>})
            if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * (num_sms / 2), 1, 1);
        cfg.blockDim = dim3(NUM_THREADS, 1, 1);
        cfg.dynamicSmemBytes = smem;
        int clusters = 0;
        e = cudaOccupancyMaxActiveClusters(&clusters, k_leaf_tc2<true, false>, &cfg);
        if (e != cudaSuccess || clusters <= 0) {
            cudaGetLastError();
            clusters = num_sms / 2;
        }
        *out = clusters;
        return cudaSuccess;
    });
    if (ea != cudaSuccess) return ea;
    // with per-pair work lists the grid has exactly one pair per list
    const int pairs = L.entries ? L.nentries : (L.ntiles < max_pairs ? L.ntiles : max_pairs);
    const bool lazy = L.max_units <= L.ds.lazy_units;
    auto kern = L.scaled ? (lazy ? k_leaf_tc2<true, true> : k_leaf_tc2<false, true>)
                         : (lazy ? k_leaf_tc2<true, false> : k_leaf_tc2<false, false>);
    // programmatic dependent launch, as for the one-SM leaf
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(2 * pairs));
    cfg.blockDim = dim3(NUM_THREADS);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, L.prods, L.tiles, L.segs, L.ntiles,
                              reinterpret_cast<const CUtensorMap *>(L.tmaps), L.mp, L.ds, L.err,
                              L.pieces, L.entries, L.part, L.part_ctr);
}

}  // namespace fsk
