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
// Pipeline (one CTA per SM, persistent: tiles are taken from a device work
// queue -- an atomic counter over a longest-first tile list -- by the
// producer warp and handed to the MMA and epilogue warps through a small
// shared-memory ring):
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
#include "tc_common.cuh"

namespace fsk {
namespace {

constexpr int BM = 128, BN = 256, BK = 64;
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;            // 16 KB
constexpr int B_BYTES = BN * BK * 2;            // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;  // 48 KB
// Epilogue warps: EW = 8 (128 running sums per thread) or 16 (64 per thread,
// four warps per scheduler instead of two, for launches of many short tiles,
// whose accumulator drains come every few k-blocks).  Warps 0..EW−1 drain,
// warp EW produces, warp EW + 1 issues MMAs.
// With 8 epilogue warps the CTA has 12 warps, three warpgroups: the third
// (producer, MMA issuer and two idle warps) gives registers to the two
// epilogue warpgroups with setmaxnreg, 168 at launch becoming 56 and 224
// (2·128·224 + 128·56 = 384·168 = 64,512; per scheduler 3·32·168 = 16,128
// ≤ 16,384), so an epilogue thread holds its 128 sums and two 16-column
// accumulator chunks: it loads the next chunk from tensor memory while it
// reduces the current one.  The 16-warp CTA (18 warps) keeps 96 registers.
template <int EW>
struct Roles {
    static constexpr int EPI_WARPS = EW;
    static constexpr int PRODUCER_WARP = EW, MMA_WARP = EW + 1;
    static constexpr bool SPLIT_REGS = EW == 8;
    static constexpr int NUM_THREADS = SPLIT_REGS ? 384 : 32 * (EW + 2);
    static constexpr int EPI_COLS = BN / (EW / 4);     // columns per epilogue thread
    static constexpr int ISSUE_REGS = 56, EPI_REGS = 224;  // SPLIT_REGS: after setmaxnreg
};
constexpr int LD_COLS = 16;  // TMEM columns per tcgen05.ld
constexpr int RING = 4;      // tiles handed from the producer to the MMA and epilogue warps
constexpr int TMEM_COLS = 512;

constexpr uint32_t IDESC = tc::idesc_bf16(BM, BN);
using namespace tc;

// LAZY: no tile of the launch has more units than ds.lazy_units, so the
// running sums may grow unreduced (one add per unit and element) and are
// brought below 2p once, before the store; otherwise every unit's add is
// followed by a conditional subtract that keeps them below 2p.
template <bool LAZY, bool SCALED, int EW>
__global__ void __launch_bounds__(Roles<EW>::NUM_THREADS, 1) k_leaf_tc(const LeafProd *__restrict__ prods,
                                                             const LeafTile *__restrict__ tiles,
                                                             const LeafSeg *__restrict__ segs,
                                                             int ntiles,
                                                             const CUtensorMap *__restrict__ tmaps,
                                                             ModP m,
                                                             const __grid_constant__ DigitScheme ds,
                                                             unsigned int *err,
                                                             unsigned int *tile_ctr,
                                                             const LeafPiece *__restrict__ pieces,
                                                             const int32_t *__restrict__ entries,
                                                             int nentries, uint32_t *part,
                                                             unsigned int *part_ctr) {
    constexpr int EPI_WARPS = Roles<EW>::EPI_WARPS, PRODUCER_WARP = Roles<EW>::PRODUCER_WARP,
                  MMA_WARP = Roles<EW>::MMA_WARP, EPI_COLS = Roles<EW>::EPI_COLS;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES];
    __shared__ __align__(8) uint64_t accf_bar[2], acce_bar[2], drain_bar;
    __shared__ __align__(8) uint64_t ring_full[RING], ring_empty[RING];
    __shared__ int tile_ring[RING];
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
        for (int q = 0; q < RING; ++q) {
            mbar_init(&ring_full[q], 1);
            mbar_init(&ring_empty[q], 1 + EPI_WARPS);
        }
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

    if (warp >= EPI_WARPS) {
    if constexpr (Roles<EW>::SPLIT_REGS)
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(Roles<EW>::ISSUE_REGS));
    if (warp == PRODUCER_WARP) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            // the operands may still be being written by the preceding grid
            asm volatile("griddepcontrol.wait;" ::: "memory");
            uint32_t it = 0, seq = 0;
            bool ok = true;
            for (uint32_t round = 0; ok; ++round) {
                // next entry from the device work queue (or round-robin); its
                // items go to the MMA and epilogue warps through the shared
                // ring, followed by -1 once the queue is empty
                const int e = tile_ctr ? (int)atomicAdd(tile_ctr, 1u) : (int)(blockIdx.x + round * gridDim.x);
                const bool done = e >= nentries;
                const int i0 = done ? 0 : (entries ? entries[e] : e);
                const int i1 = done ? 1 : (entries ? entries[e + 1] : e + 1);
                for (int t = i0; t < i1 && ok; ++t, ++seq) {
                    const int slot = seq % RING;
                    if (!mbar_wait(&ring_empty[slot], ((seq / RING) & 1u) ^ 1u, &abort_flag, err)) {
                        ok = false;
                        break;
                    }
                    tile_ring[slot] = done ? -1 : t;
                    mbar_arrive(&ring_full[slot]);
                    if (done) break;
                    const LeafTile tl = tiles[t];
                    const LeafProd pr = prods[tl.prod];
                    const int sx0 = pieces ? pieces[t].sx0 : 0, sx1 = pieces ? pieces[t].sx1 : pr.nseg;
                    const CUtensorMap *tm = tmaps + pr.arena;
                    // the descriptor was written by a host copy before this launch
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tm)
                                 : "memory");
                    for (int sx = sx0; sx < sx1 && ok; ++sx) {
                        const LeafSeg sg = segs[pr.seg0 + sx];
                        const int ya = (int)(pr.a_row0 + (int64_t)(sg.ij >> 4) * pr.plane_rows + (int64_t)tl.tm * BM);
                        const int yb = (int)(pr.b_row0 + (int64_t)(sg.ij & 15) * pr.plane_rows + (int64_t)tl.tn * BN);
                        for (int kb = sg.kb0; kb < sg.kb0 + sg.nkb; ++kb, ++it) {
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
                    }
                }
                if (done) break;
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
            for (uint32_t seq = 0; ok; ++seq) {
                const int slot = seq % RING;
                if (!mbar_wait(&ring_full[slot], (seq / RING) & 1u, &abort_flag, err)) {
                    ok = false;
                    break;
                }
                const int t = tile_ring[slot];
                mbar_arrive(&ring_empty[slot]);
                if (t < 0) break;
                const LeafProd pr = prods[tiles[t].prod];
                const int sx0 = pieces ? pieces[t].sx0 : 0, sx1 = pieces ? pieces[t].sx1 : pr.nseg;
                bool open = false;  // a unit's accumulator is being filled
                uint32_t b = 0, tmem_d = 0;
                for (int sx = sx0; sx < sx1; ++sx) {
                    const LeafSeg sg = segs[pr.seg0 + sx];
                    if (sg.first) {
                        if (open) {
                            mma_commit(&accf_bar[b]);
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
                            mma_bf16(tmem_d, sdesc(sa + kk * 32), sdesc(sb + kk * 32), IDESC,
                                     (sg.first && kb == 0 && kk == 0) ? 0u : 1u);
                        mma_commit(&empty_bar[s]);
                    }
                    if (!ok) break;
                }
                if (!ok) break;
                if (open) {
                    mma_commit(&accf_bar[b]);
                    ++unit;
                }
            }
            // every MMA issued so far has completed once this barrier fires
            mma_commit(&drain_bar);
            mbar_drain(&drain_bar, 0);
        }
    }  // warps past the MMA issuer (SPLIT_REGS) have no role
    } else {
        // ---------------- epilogue ----------------
        if constexpr (Roles<EW>::SPLIT_REGS)
            asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(Roles<EW>::EPI_REGS));
        const uint32_t p = m.p, twop = 2 * m.p, off = ds.offset;
        const int quad = warp & 3, colq = warp >> 2;
        uint32_t unit = 0;
        bool ok = true;
        for (uint32_t seq = 0; ok; ++seq) {
            const int slot = seq % RING;
            const bool gotr = mbar_wait(&ring_full[slot], (seq / RING) & 1u, &abort_flag, err);
            if (!__all_sync(0xffffffffu, gotr)) break;
            const int t = tile_ring[slot];
            __syncwarp();
            if (lane == 0) mbar_arrive(&ring_empty[slot]);
            if (t < 0) break;
            const LeafTile tl = tiles[t];
            const LeafProd pr = prods[tl.prod];
            uint32_t acc[EPI_COLS];  // running sums of the tile row's residues
#pragma unroll
            for (int e = 0; e < EPI_COLS; ++e) acc[e] = 0;
            int lo = 0, hi = 0;  // 16-column chunks of this warp that hold stored entries
            live_chunks(pr, (int64_t)tl.tm * BM + quad * 32, (int64_t)tl.tn * BN + colq * EPI_COLS,
                        EPI_COLS / LD_COLS, lo, hi);
            const int sx0 = pieces ? pieces[t].sx0 : 0, sx1 = pieces ? pieces[t].sx1 : pr.nseg;
            for (int sx = sx0; sx < sx1; ++sx) {
                const LeafSeg sg = segs[pr.seg0 + sx];
                if (!sg.first) continue;  // one drain per unit
                const uint32_t b = unit & 1u;
                // warp-uniform outcome: tcgen05.ld below is .sync.aligned
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
                // one 16-column chunk: exact integer |x| ≤ 2^24 → shifted into
                // [0, 2^26) → ·weight mod p → added to the running sums
#define FSK_REDUCE_CHUNK(CC, V)                                                  \
    _Pragma("unroll") for (int e = 0; e < LD_COLS; ++e) {                        \
        const int xi = __float2int_rn(__uint_as_float((V)[e]));                  \
        const uint32_t a = (uint32_t)(xi + (int)off);                            \
        const uint32_t q = __umulhi(a, wsh);                                     \
        const uint32_t r = a * w - q * p; /* [0, 2p) */                          \
        if constexpr (LAZY) {                                                    \
            acc[(CC) * LD_COLS + e] += r;                                        \
        } else {                                                                 \
            const uint32_t s = acc[(CC) * LD_COLS + e] + r;                      \
            acc[(CC) * LD_COLS + e] = min(s, s - twop);                          \
        }                                                                        \
    }
                if constexpr (Roles<EW>::SPLIT_REGS) {
                    // two chunk buffers: chunk cc + 1 loads while chunk cc is reduced
                    // (tcgen05.wait::ld waits for every load of the thread, so the
                    // next load is issued after the wait)
                    uint32_t va[LD_COLS], vb[LD_COLS];
#pragma unroll
                    for (int cc = 0; cc < EPI_COLS / LD_COLS; ++cc) {
                        if (cc < lo || cc >= hi) continue;
                        if (cc == lo) {
                            if (cc & 1) tmem_ld16(taddr + cc * LD_COLS, vb);
                            else tmem_ld16(taddr + cc * LD_COLS, va);
                        }
                        if (cc & 1) tmem_wait_ld_tied(vb);
                        else tmem_wait_ld_tied(va);
                        if (cc + 1 < hi) {
                            if (cc & 1) tmem_ld16(taddr + (cc + 1) * LD_COLS, va);
                            else tmem_ld16(taddr + (cc + 1) * LD_COLS, vb);
                        }
                        if (cc & 1) {
                            FSK_REDUCE_CHUNK(cc, vb)
                        } else {
                            FSK_REDUCE_CHUNK(cc, va)
                        }
                    }
                } else {
#pragma unroll
                    for (int cc = 0; cc < EPI_COLS / LD_COLS; ++cc) {
                        if (cc < lo || cc >= hi) continue;
                        uint32_t v[LD_COLS];
                        tmem_ld16(taddr + cc * LD_COLS, v);
                        tmem_wait_ld();
                        FSK_REDUCE_CHUNK(cc, v)
                    }
                }
#undef FSK_REDUCE_CHUNK
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce_bar[b]);
                ++unit;
            }
            if constexpr (LAZY) {
#pragma unroll
                for (int e = 0; e < EPI_COLS; ++e) acc[e] = reduce_2p(acc[e], p, m.barrett);
            }
            if (!ok) break;
            const LeafPiece pc = pieces ? pieces[t] : LeafPiece{0, 0, -1, 0, 1};
            if (pc.slot0 >= 0) {
                // a piece of a shared tile: publish its residues; the piece
                // that finishes last adds the others' and stores the tile
                uint32_t *mine = part + ((int64_t)(pc.slot0 + pc.j) * (BM * BN)) + threadIdx.x * EPI_COLS;
#pragma unroll
                for (int e = 0; e < EPI_COLS; e += 4) {
                    uint4 v4;
                    v4.x = acc[e] >= p ? acc[e] - p : acc[e];
                    v4.y = acc[e + 1] >= p ? acc[e + 1] - p : acc[e + 1];
                    v4.z = acc[e + 2] >= p ? acc[e + 2] - p : acc[e + 2];
                    v4.w = acc[e + 3] >= p ? acc[e + 3] - p : acc[e + 3];
                    *reinterpret_cast<uint4 *>(mine + e) = v4;
                }
                // per warp: its 32 rows × 128 columns are combined by the
                // CTA whose warp finishes them last (no cross-warp barrier)
                __threadfence();
                __syncwarp();
                unsigned int prev = 0;
                if (lane == 0) prev = atomicAdd(&part_ctr[pc.slot0 * EPI_WARPS + warp], 1u);
                prev = __shfl_sync(0xffffffffu, prev, 0);
                if (prev != (unsigned)(pc.npieces - 1)) continue;
                __threadfence();
#pragma unroll 1
                for (int q = 0; q < pc.npieces; ++q) {
                    if (q == pc.j) continue;
                    const uint32_t *other = part + ((int64_t)(pc.slot0 + q) * (BM * BN)) + threadIdx.x * EPI_COLS;
#pragma unroll
                    for (int e = 0; e < EPI_COLS; e += 4) {
                        const uint4 o = __ldcg(reinterpret_cast<const uint4 *>(other + e));
                        // acc < 2p and o < p: the sum stays below 2p after one conditional subtract
                        uint32_t s0 = acc[e] + o.x, s1 = acc[e + 1] + o.y, s2 = acc[e + 2] + o.z,
                                 s3 = acc[e + 3] + o.w;
                        acc[e] = min(s0, s0 - twop);
                        acc[e + 1] = min(s1, s1 - twop);
                        acc[e + 2] = min(s2, s2 - twop);
                        acc[e + 3] = min(s3, s3 - twop);
                    }
                }
                if (lane == 0) part_ctr[pc.slot0 * EPI_WARPS + warp] = 0;  // ready for the next launch
            }
            // store the tile's residues
            store_tile_row<EPI_COLS, SCALED>(pr, (int64_t)tl.tm * BM + quad * 32 + lane,
                                     (int64_t)tl.tn * BN + colq * EPI_COLS, acc, p);
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

// Failure-detection self-test: one thread waits on an mbarrier that nothing
// ever signals, gives up after limit_ns and records the timeout in the error
// word -- the same path every bounded wait of the leaf takes -- and the
// kernel returns normally, so the context stays usable.
__global__ void k_wait_selftest(unsigned int *err, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint64_t t0 = gtimer();
        while (!mbar_try(&bar, 0)) {
            if (gtimer() - t0 > limit_ns) {
                atomicOr(err, ERR_WAIT);
                break;
            }
        }
    }
}

}  // namespace

cudaError_t launch_wait_selftest(unsigned int *err, unsigned long long limit_ns, cudaStream_t st) {
    k_wait_selftest<<<1, 32, 0, st>>>(err, limit_ns);
    return cudaGetLastError();
}

int leaf_tc_bm() { return BM; }
int leaf_tc_bn() { return BN; }

cudaError_t launch_leaf_tc(const TcLaunch &L, int num_sms, cudaStream_t st) {
    if (L.ntiles == 0) return cudaSuccess;
    const int smem = STAGES * STAGE_BYTES + 1024;
    // the dynamic shared-memory opt-in, once per device
    static DeviceOnce attr_once;
    cudaError_t ea = once_per_device(attr_once, nullptr, [smem](int *) {
        cudaError_t e = cudaSuccess;
        for (auto fn : {k_leaf_tc<true, false, 8>, k_leaf_tc<false, false, 8>, k_leaf_tc<true, true, 8>,
                        k_leaf_tc<false, true, 8>, k_leaf_tc<true, false, 16>, k_leaf_tc<false, false, 16>,
                        k_leaf_tc<true, true, 16>, k_leaf_tc<false, true, 16>})
            if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        // the 8-warp instances hand registers between warpgroups with
        // setmaxnreg, whose budget assumes exactly 168 registers per thread
        // at launch (384 · 168): with fewer, setmaxnreg.inc would wait forever
        for (auto fn : {k_leaf_tc<true, false, 8>, k_leaf_tc<false, false, 8>, k_leaf_tc<true, true, 8>,
                        k_leaf_tc<false, true, 8>}) {
            cudaFuncAttributes fa{};
            if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
            if (e == cudaSuccess &&
                fa.numRegs * Roles<8>::NUM_THREADS !=
                    2 * 128 * Roles<8>::EPI_REGS + 128 * Roles<8>::ISSUE_REGS)
                e = cudaErrorInvalidConfiguration;
        }
        return e;
    });
    if (ea != cudaSuccess) return ea;
    const int nwork = L.entries ? L.nentries : L.ntiles;
    const int grid = nwork < num_sms ? nwork : num_sms;
    const bool lazy = L.max_units <= L.ds.lazy_units;
    // frequent accumulator drains (many short tiles, or the short units of
    // Karatsuba's digit-sum products): the 16-warp epilogue, four warps per
    // scheduler, drains a unit in about half the time
    const bool wide_epi = L.epi_warps == 16;
    auto kern = wide_epi ? (L.scaled ? (lazy ? k_leaf_tc<true, true, 16> : k_leaf_tc<false, true, 16>)
                                     : (lazy ? k_leaf_tc<true, false, 16> : k_leaf_tc<false, false, 16>))
                         : (L.scaled ? (lazy ? k_leaf_tc<true, true, 8> : k_leaf_tc<false, true, 8>)
                                     : (lazy ? k_leaf_tc<true, false, 8> : k_leaf_tc<false, false, 8>));
    // programmatic dependent launch: the prologue may overlap the grid that
    // writes the operands (the producer waits for it before its first load)
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(wide_epi ? Roles<16>::NUM_THREADS : Roles<8>::NUM_THREADS);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int nentries = L.entries ? L.nentries : L.ntiles;
    return cudaLaunchKernelEx(&cfg, kern, L.prods, L.tiles, L.segs, L.ntiles,
                              reinterpret_cast<const CUtensorMap *>(L.tmaps), L.mp, L.ds, L.err,
                              L.tile_ctr, L.pieces, L.entries, nentries, L.part, L.part_ctr);
}

}  // namespace fsk
