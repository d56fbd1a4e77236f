// CUDA-core leaf: out = X·Zᵀ mod p with 32×32→64-bit multiply-adds.
//
// The plain integer leaf that the tensor-core leaf is measured against.
// Operands are uint32 residues in [0, p) (one "digit plane" per operand in a
// uint32 arena).  Every product is < p² < 2^48, so a uint64 accumulator
// takes 2^15 products before it is reduced, which is far beyond one 32-wide
// k-block: the sum is reduced once per 2^15 k and once at the end.
// 64×64 output tile, 256 threads, 4×4 outputs per thread, 32-wide k-blocks
// staged through shared memory.
#include "ffsyrk_internal.h"

namespace fsk {
namespace {

constexpr int TI = 64;   // output tile
constexpr int TK = 32;   // k-block
constexpr int SLD = TI + 4;

__global__ void __launch_bounds__(256) k_leaf_i64(const LeafProd *__restrict__ prods,
                                                  const LeafTile *__restrict__ tiles,
                                                  const uint32_t *const *__restrict__ arenas,
                                                  const int64_t *__restrict__ arena_kpad,
                                                  ModP m) {
    __shared__ __align__(16) uint32_t xs[TK][SLD];
    __shared__ __align__(16) uint32_t zs[TK][SLD];
    const LeafTile tl = tiles[blockIdx.x];
    const LeafProd pr = prods[tl.prod];
    const uint32_t *base = arenas[pr.arena];
    const int64_t kpad = arena_kpad[pr.arena];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = (int64_t)tl.tm * TI, col0 = (int64_t)tl.tn * TI;
    const uint32_t *xa = base + (pr.a_row0 + row0) * kpad;
    const uint32_t *za = base + (pr.b_row0 + col0) * kpad;
    unsigned long long acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0ull;
    const uint64_t p = m.p;
    const int nkb = (int)(kpad / TK);
    int since = 0;
    for (int kb = 0; kb < nkb; ++kb) {
        // each thread moves 2 × (16 B of X) and 2 × (16 B of Z)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int lr = (tid >> 3) + 32 * q;  // tile row
            const int lk = (tid & 7) * 4;        // k within the block
            uint4 vx = *reinterpret_cast<const uint4 *>(xa + (int64_t)lr * kpad + kb * TK + lk);
            uint4 vz = *reinterpret_cast<const uint4 *>(za + (int64_t)lr * kpad + kb * TK + lk);
            xs[lk + 0][lr] = vx.x;
            xs[lk + 1][lr] = vx.y;
            xs[lk + 2][lr] = vx.z;
            xs[lk + 3][lr] = vx.w;
            zs[lk + 0][lr] = vz.x;
            zs[lk + 1][lr] = vz.y;
            zs[lk + 2][lr] = vz.z;
            zs[lk + 3][lr] = vz.w;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < TK; ++kk) {
            uint4 a = *reinterpret_cast<const uint4 *>(&xs[kk][ty * 4]);
            uint4 b = *reinterpret_cast<const uint4 *>(&zs[kk][tx * 4]);
            const uint32_t av[4] = {a.x, a.y, a.z, a.w};
            const uint32_t bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += (unsigned long long)av[i] * bv[j];
        }
        __syncthreads();
        since += TK;
        if (since >= 32768) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] %= p;
            since = 0;
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t r = row0 + ty * 4 + i;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t c = col0 + tx * 4 + j;
            if (r >= pr.rows || c >= pr.cols) continue;
            const bool keep = pr.tri == 0 || (pr.tri == 1 && c <= r) || (pr.tri == 2 && c >= r);
            if (!keep) continue;
            uint32_t *o = pr.out + r * pr.ldo + c;
            const uint32_t v = (uint32_t)(acc[i][j] % p);
            *o = pr.scale.mode ? scale_out(v, *o, pr.scale, p) : v;
        }
    }
}

}  // namespace

int leaf_i64_tile() { return TI; }

cudaError_t launch_leaf_i64_arrays(const LeafProd *prods_dev, const LeafTile *tiles_dev,
                                   int ntiles, const uint32_t *const *arenas_dev,
                                   const int64_t *kpad_dev, ModP mp, cudaStream_t st) {
    if (ntiles == 0) return cudaSuccess;
    k_leaf_i64<<<ntiles, 256, 0, st>>>(prods_dev, tiles_dev, arenas_dev, kpad_dev, mp);
    return cudaGetLastError();
}

}  // namespace fsk
