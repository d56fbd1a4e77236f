// INT8 leaf: out = X·Zᵀ mod p on the warp-level INT8 tensor path
// (mma.sync.m16n8k32, 8-bit operands, int32 accumulators in registers).
//
// The leaf products of Algorithm 2 (arXiv 2001.04109, Section 3) with the
// paper's delayed modular reduction (Section 4.2) carried out on exact
// integer products: a residue's symmetric representative s ∈ [−(p−1)/2,
// (p−1)/2] is stored as the D bytes of its two's complement, s = Σ_{t<D−1}
// u_t·256^t + s_{D−1}·256^{D−1} with unsigned low digits u_t ∈ [0, 255] and
// a signed top digit, so X·Zᵀ = Σ_{i,j} 256^(i+j)·X_i·Z_jᵀ and every digit
// product is an exact mma.sync of u8 or s8 operands.  The pairs of one
// weight class i + j accumulate in one set of int32 registers (a "unit")
// while the sum of their bounds 128·k-blocks·max|d_i|·max|d_j| stays within
// 2^30; each unit is then reduced once: a = acc + c·p ≥ 0 (c·p the least
// multiple of p ≥ 2^30), times 256^(i+j) mod p with Shoup's quotient, added
// to a running residue below 2p.
//
// There is no tcgen05 INT8 MMA on sm_103a (ptxas rejects .kind::i8 for it),
// so this leaf uses the warp-level instruction; its throughput is measured
// by ffsyrk_probe_pipe.
//
// CTA: one 128×128 output tile at a time (persistent CTAs, tiles taken
// round-robin from a longest-first list); warp 8 is the TMA producer (one
// 128-row box of the X plane and one of the Z plane per 128-column k-block,
// 128-byte swizzle, 4 stages), warps 0–7 compute: warp w owns rows
// 64·(w mod 2).. and columns 32·(w div 2).. of the tile, fed by ldmatrix.
// The int32 accumulators live in registers; each thread's running residues
// live in shared memory (64 words per thread, laid out thread-minor), which
// is touched once per unit only.
// Every mbarrier wait is bounded; a wait that runs out records the error and
// the CTA stops.
#include <cuda.h>
#include <cuda_runtime.h>

#include "ffsyrk_internal.h"
#include "tc_common.cuh"

namespace fsk {
namespace {

using namespace tc;

constexpr int BM = 128, BN = 128, BK = 128;  // tile rows, columns, k-block (bytes)
constexpr int STAGES = 4;
constexpr int X_BYTES = BM * BK, Z_BYTES = BN * BK;  // 16 KB each
constexpr int STAGE_BYTES = X_BYTES + Z_BYTES;
constexpr int MMA_WARPS = 8, PRODUCER_WARP = 8;
constexpr int NUM_THREADS = 32 * (MMA_WARPS + 1);
constexpr int WM = 64, WN = 32;              // warp tile
constexpr int MF = WM / 16, NF = WN / 8;     // m16 and n8 fragments per warp
constexpr int RES_WORDS = MF * NF * 4;       // residues per compute thread
constexpr int RES_BYTES = RES_WORDS * MMA_WARPS * 32 * 4;  // 64 KB

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2,
                                        uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

// One m16n8k32 product; SA / SB: operand is signed (the top digit) or unsigned.
template <bool SA, bool SB>
__device__ __forceinline__ void mma_i8(int32_t (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    if constexpr (SA && SB)
        asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                     "{%8,%9}, {%0,%1,%2,%3};"
                     : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
                     : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    else if constexpr (SA && !SB)
        asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                     "{%8,%9}, {%0,%1,%2,%3};"
                     : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
                     : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    else if constexpr (!SA && SB)
        asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.u8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                     "{%8,%9}, {%0,%1,%2,%3};"
                     : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
                     : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    else
        asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                     "{%8,%9}, {%0,%1,%2,%3};"
                     : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
                     : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Address of 16-byte chunk `ch` of row `r` in a 128-byte-swizzled tile
// (TMA SWIZZLE_128B: chunk ch of row r sits at chunk ch ^ (r mod 8)).
__device__ __forceinline__ uint32_t swz(uint32_t base, int r, int ch) {
    return base + (uint32_t)(r * 128 + ((ch ^ (r & 7)) << 4));
}

// The warp's MMAs over one staged k-block (four k32 steps).
template <bool SA, bool SB>
__device__ __forceinline__ void kblock(int32_t (&acc)[MF][NF][4], uint32_t sx, uint32_t sz, int wm, int wn,
                                       int lane) {
    const int q = lane >> 3, l8 = lane & 7;
#pragma unroll
    for (int kk = 0; kk < BK / 32; ++kk) {
        uint32_t a[MF][4], b[NF][2];
#pragma unroll
        for (int mf = 0; mf < MF; ++mf) {
            // matrices: rows 0–7 / 8–15 of the fragment, k-bytes 0–15 / 16–31
            const int r = wm * WM + mf * 16 + l8 + (q & 1) * 8;
            ldsm_x4(swz(sx, r, 2 * kk + (q >> 1)), a[mf][0], a[mf][1], a[mf][2], a[mf][3]);
        }
#pragma unroll
        for (int nf = 0; nf < NF; nf += 2) {
            // matrices: columns of fragments nf, nf + 1; k-bytes 0–15 / 16–31
            const int r = wn * WN + (nf + (q >> 1)) * 8 + l8;
            ldsm_x4(swz(sz, r, 2 * kk + (q & 1)), b[nf][0], b[nf][1], b[nf + 1][0], b[nf + 1][1]);
        }
#pragma unroll
        for (int mf = 0; mf < MF; ++mf)
#pragma unroll
            for (int nf = 0; nf < NF; ++nf) mma_i8<SA, SB>(acc[mf][nf], a[mf], b[nf]);
    }
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
    k_leaf_i8(const LeafProd *__restrict__ prods, const LeafTile *__restrict__ tiles,
              const LeafSeg *__restrict__ segs, int ntiles, const CUtensorMap *__restrict__ tmaps,
              ModP m, const __grid_constant__ DigitScheme ds, unsigned int *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES];
    __shared__ volatile int abort_flag;
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    // each compute thread's running residues (word (f, thread) at f·256 + thread)
    uint32_t *res = reinterpret_cast<uint32_t *>(smem + STAGES * STAGE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], MMA_WARPS);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == PRODUCER_WARP) {
        if (lane == 0) {
            asm volatile("griddepcontrol.wait;" ::: "memory");
            uint32_t it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const LeafTile tl = tiles[t];
                const LeafProd pr = prods[tl.prod];
                const CUtensorMap *tm = tmaps + pr.arena;
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tm) : "memory");
                for (int sx = 0; sx < pr.nseg && ok; ++sx) {
                    const LeafSeg sg = segs[pr.seg0 + sx];
                    const int ya = (int)(pr.a_row0 + (int64_t)(sg.ij >> 4) * pr.plane_rows + (int64_t)tl.tm * BM);
                    const int yb = (int)(pr.b_row0 + (int64_t)(sg.ij & 15) * pr.plane_rows + (int64_t)tl.tn * BN);
                    for (int kb = sg.kb0; kb < sg.kb0 + sg.nkb; ++kb, ++it) {
                        const int s = it % STAGES;
                        if (!mbar_wait(&empty_bar[s], ((it / STAGES) & 1u) ^ 1u, &abort_flag, err)) {
                            ok = false;
                            break;
                        }
                        unsigned char *sa = smem + s * STAGE_BYTES;
                        mbar_expect_tx(&full_bar[s], STAGE_BYTES);
                        tma_load(sa, tm, &full_bar[s], kb * BK, ya);
                        tma_load(sa + X_BYTES, tm, &full_bar[s], kb * BK, yb);
                    }
                }
            }
            if (!ok) {
                const uint32_t first = it > STAGES ? it - STAGES : 0;
                for (uint32_t q = first; q < it; ++q) mbar_drain(&full_bar[q % STAGES], (q / STAGES) & 1u);
            }
        }
    } else {
        const int wm = warp & 1, wn = warp >> 1;
        const int g = lane >> 2, t4 = lane & 3;
        const uint32_t p = m.p, twop = 2 * m.p, off = ds.offset;
        const int top = ds.D - 1;
        uint32_t it = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const LeafTile tl = tiles[t];
            const LeafProd pr = prods[tl.prod];
            int32_t acc[MF][NF][4];
#pragma unroll
            for (int mf = 0; mf < MF; ++mf)
#pragma unroll
                for (int nf = 0; nf < NF; ++nf)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[mf][nf][e] = 0;
            bool first_unit = true;
            for (int sx = 0; sx < pr.nseg && ok; ++sx) {
                const LeafSeg sg = segs[pr.seg0 + sx];
                const int si = sg.ij >> 4, sj = sg.ij & 15;
                const int kind = ((si == top) ? 2 : 0) | ((sj == top) ? 1 : 0);
                for (int kb = 0; kb < sg.nkb; ++kb, ++it) {
                    const int s = it % STAGES;
                    const bool got = mbar_wait(&full_bar[s], (it / STAGES) & 1u, &abort_flag, err);
                    if (!__all_sync(0xffffffffu, got)) {
                        ok = false;
                        break;
                    }
                    const uint32_t sx_ = su32(smem + s * STAGE_BYTES), sz_ = sx_ + X_BYTES;
                    switch (kind) {
                        case 0: kblock<false, false>(acc, sx_, sz_, wm, wn, lane); break;
                        case 1: kblock<false, true>(acc, sx_, sz_, wm, wn, lane); break;
                        case 2: kblock<true, false>(acc, sx_, sz_, wm, wn, lane); break;
                        default: kblock<true, true>(acc, sx_, sz_, wm, wn, lane); break;
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&empty_bar[s]);
                }
                if (!ok) break;
                // the unit ends here when the next segment opens one (or the tile ends)
                const bool last = sx + 1 == pr.nseg || segs[pr.seg0 + sx + 1].first;
                if (last) {
                    const MulConst wt = ds.weight[si][sj];
#pragma unroll
                    for (int mf = 0; mf < MF; ++mf)
#pragma unroll
                        for (int nf = 0; nf < NF; ++nf)
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                // |acc| ≤ 2^30 → a ∈ [0, 2^31 + p) → ·256^(i+j) mod p in [0, 2p)
                                const uint32_t a = (uint32_t)acc[mf][nf][e] + off;
                                const uint32_t qq = __umulhi(a, wt.w_sh);
                                const uint32_t r = a * wt.w - qq * p;
                                uint32_t &slot = res[((mf * NF + nf) * 4 + e) * (MMA_WARPS * 32) + threadIdx.x];
                                const uint32_t sum = first_unit ? r : slot + r;
                                slot = min(sum, sum - twop);
                                acc[mf][nf][e] = 0;
                            }
                    first_unit = false;
                }
            }
            if (!ok) break;
            // store: fragment (mf, nf) holds rows g and g + 8, columns 2·t4 and 2·t4 + 1
            const int64_t rb = (int64_t)tl.tm * BM + wm * WM, cb = (int64_t)tl.tn * BN + wn * WN;
#pragma unroll
            for (int mf = 0; mf < MF; ++mf)
#pragma unroll
                for (int hr = 0; hr < 2; ++hr) {
                    const int64_t r = rb + mf * 16 + g + 8 * hr;
                    if (r >= pr.rows) continue;
                    uint32_t *orow = pr.out + r * pr.ldo;
#pragma unroll
                    for (int nf = 0; nf < NF; ++nf)
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int64_t c = cb + nf * 8 + 2 * t4 + e;
                            const bool keep = c < pr.cols &&
                                              (pr.tri == 0 || (pr.tri == 1 && c <= r) || (pr.tri == 2 && c >= r));
                            if (!keep) continue;
                            const uint32_t v =
                                first_unit ? 0u
                                           : final_mod(res[((mf * NF + nf) * 4 + 2 * hr + e) * (MMA_WARPS * 32) +
                                                           threadIdx.x],
                                                       p);
                            orow[c] = pr.scale.mode ? scale_out(v, orow[c], pr.scale, p) : v;
                        }
                }
        }
    }
    __syncthreads();
}

}  // namespace

int leaf_i8_bm() { return BM; }
int leaf_i8_bn() { return BN; }

cudaError_t launch_leaf_i8(const I8Launch &L, int num_sms, cudaStream_t st) {
    if (L.ntiles == 0) return cudaSuccess;
    const int smem = STAGES * STAGE_BYTES + RES_BYTES + 1024;
    static DeviceOnce attr_once;
    cudaError_t ea = once_per_device(attr_once, nullptr, [smem](int *) {
        return cudaFuncSetAttribute(k_leaf_i8, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    });
    if (ea != cudaSuccess) return ea;
    const int grid = L.ntiles < num_sms ? L.ntiles : num_sms;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(NUM_THREADS);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_leaf_i8, L.prods, L.tiles, L.segs, L.ntiles,
                              reinterpret_cast<const CUtensorMap *>(L.tmaps), L.mp, L.ds, L.err);
}

}  // namespace fsk
