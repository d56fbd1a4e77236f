// Diagonal and block-diagonal scaling on the GPU (arXiv 2001.04109,
// Section 5: Algorithm 4 "nrsyf", Algorithm 5 "syrkd", Algorithm 6 "syrkbd"
// for odd p).
//
// A·B·Aᵀ with B symmetric block diagonal becomes Ā·Āᵀ for Ā = A·W: every
// 2×2 block of B is made congruent to a diagonal one (B = T·Diag(d̄)·Tᵀ),
// Diag(d̄) = Δ·Δᵀ is factored without a field extension (square roots of the
// squares, Algorithm 4 on consecutive pairs of non-squares, one added zero
// column when their number is odd), and W = [T 0]·Δ.  Each column of W has
// at most four nonzero entries.  The planning runs in three small kernels:
//
//  * k_scale_cols   (one thread per column): T and d̄ of the column's block,
//                   its Legendre symbol, and W's column for a square d̄;
//  * k_scale_rank   (one CTA): the non-square columns listed in column order;
//  * k_scale_pairs  (one thread per pair): Algorithm 4 on consecutive
//                   non-squares, W's two columns.
//
// k_col_mix then writes Ā = A·W into the plan's scratch, and the ordinary
// symmetric product of Ā follows.  The arithmetic is exact in F_p; the
// choices (which root, which pairing, the order of each column's terms) are
// those of the host planner ffsyrkbd_factor, so both give the same W.
#include <algorithm>

#include "ffsyrk_internal.h"

namespace fsk {
namespace {

// x mod p for any x < 2^64 (Barrett with minv = ⌊(2^64 − 1)/p⌋: the quotient
// estimate is low by at most one, so one correction suffices)
__device__ __forceinline__ uint32_t fred64(uint64_t x, const ScaleConst &f) {
    const uint64_t q = __umul64hi(x, f.minv);
    uint64_t r = x - q * f.p;
    return (uint32_t)(r >= f.p ? r - f.p : r);
}
__device__ __forceinline__ uint32_t fmul(uint32_t a, uint32_t b, const ScaleConst &f) {
    return fred64((uint64_t)a * b, f);
}
__device__ __forceinline__ uint32_t fadd(uint32_t a, uint32_t b, uint32_t p) {
    const uint32_t r = a + b;
    return r >= p ? r - p : r;
}
__device__ __forceinline__ uint32_t fneg(uint32_t a, uint32_t p) { return a ? p - a : 0u; }
__device__ uint32_t fpow(uint32_t a, uint32_t e, const ScaleConst &f) {
    uint32_t r = 1, b = a;
    while (e) {
        if (e & 1) r = fmul(r, b, f);
        b = fmul(b, b, f);
        e >>= 1;
    }
    return r;
}
__device__ __forceinline__ uint32_t finv(uint32_t a, const ScaleConst &f) {
    return fpow(a, f.p - 2, f);
}
// The start of Tonelli–Shanks for a ≠ 0, from one exponentiation:
// x = a^((q−1)/2), t = a^q = x²·a, r = a^((q+1)/2) = x·a (p − 1 = q·2^s).
// Euler's criterion is a^((p−1)/2) = t^(2^(s−1)): a is a square exactly when
// s − 1 squarings take t to 1.
struct TsStart {
    uint32_t t, r;
};
__device__ __forceinline__ TsStart ts_start(uint32_t a, const ScaleConst &f) {
    const uint32_t x = fpow(a, (f.q - 1) / 2, f);
    return TsStart{fmul(fmul(x, x, f), a, f), fmul(x, a, f)};
}
__device__ __forceinline__ bool ts_is_square(uint32_t t, const ScaleConst &f) {
    uint32_t e = t;
    for (uint32_t i = 1; i < f.s; ++i) e = fmul(e, e, f);
    return e == 1;
}
// Tonelli–Shanks from (t, r) of a square: the same steps, and so the same
// root, as the host planner.  Every loop is bounded by the 2-adic valuation
// s of p − 1; a non-square (never produced by the planner) sets *bad.
__device__ uint32_t ts_finish(TsStart st, const ScaleConst &f, bool *bad) {
    uint32_t M = f.s, c = f.zq, t = st.t, r = st.r;
    for (int guard = 0; t != 1; ++guard) {
        uint32_t i = 0, t2 = t;
        while (t2 != 1 && i < M) {
            t2 = fmul(t2, t2, f);
            ++i;
        }
        if (i >= M || guard > 64) {
            *bad = true;
            return 0;
        }
        uint32_t b = c;
        for (uint32_t e = 0; e + i + 1 < M; ++e) b = fmul(b, b, f);
        M = i;
        c = fmul(b, b, f);
        t = fmul(t, c, f);
        r = fmul(r, b, f);
    }
    return r;
}
__device__ __forceinline__ uint32_t fsqrt(uint32_t a, const ScaleConst &f, bool *bad) {
    return a == 0 ? 0u : ts_finish(ts_start(a, f), f, bad);
}

// One column of W under construction: up to four (source column, weight).
struct WCol {
    int src[4];
    uint32_t w[4];
    __device__ void clear() {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            src[t] = -1;
            w[t] = 0;
        }
    }
    // weight·A_s joins the column: equal sources merge, zero weights and the
    // zero column s ≥ k add nothing (the host planner's rule)
    __device__ void add(int64_t s, uint32_t weight, int64_t k, uint32_t p, bool *bad) {
        if (s >= k || weight == 0) return;
        for (int t = 0; t < 4; ++t)
            if (src[t] == (int)s) {
                w[t] = fadd(w[t], weight, p);
                return;
            }
        for (int t = 0; t < 4; ++t)
            if (src[t] < 0) {
                src[t] = (int)s;
                w[t] = weight;
                return;
            }
        *bad = true;
    }
    // W's column c: the sources, and each weight with its Shoup quotient
    // ⌊w·2^32/p⌋ for the column mix
    __device__ void store(const ScalePlan &sp, int64_t c, uint32_t p) const {
        sp.src[c] = make_int4(src[0], src[1], src[2], src[3]);
        uint32_t sh[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) sh[t] = (uint32_t)(((uint64_t)w[t] << 32) / p);
        sp.w[2 * c] = make_uint4(w[0], sh[0], w[1], sh[1]);
        sp.w[2 * c + 1] = make_uint4(w[2], sh[2], w[3], sh[3]);
    }
};

// coef·(column col of A·T) into column `out`: T's column col is
// ta[col]·e_col + tb[col]·e_mate (mate −1: none)
__device__ __forceinline__ void add_t(WCol &out, int64_t col, uint32_t coef, const ScalePlan &sp,
                                      int64_t k, const ScaleConst &f, bool *bad) {
    if (col >= k) return;
    out.add(col, fmul(coef, sp.ta[col], f), k, f.p, bad);
    const int32_t m = sp.mate[col];
    if (m >= 0) out.add(m, fmul(coef, sp.tb[col], f), k, f.p, bad);
}

// Per column c < kk: clear W's column; for c < k find the 2×2 block of B
// holding c (e[c] or e[c−1] nonzero mod p; the host has checked that blocks
// do not overlap), its congruence T and diagonal d̄ (the paper's antidiagonal
// identity for x = γ = 0, one elimination step otherwise), flag non-squares,
// and write W's column √d̄_c·T_c for a square d̄_c.
__global__ void __launch_bounds__(256) k_scale_cols(const uint32_t *__restrict__ d,
                                                    const uint32_t *__restrict__ e, int has_e,
                                                    int64_t k, int64_t kk, ScaleConst f,
                                                    ScalePlan sp, unsigned int *err) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= kk) return;
    WCol col;
    col.clear();
    if (c >= k) {
        col.store(sp, c, f.p);
        return;
    }
    const uint32_t p = f.p;
    const bool first = has_e && c + 1 < k && fred64(e[c], f) != 0;
    const bool second = has_e && c >= 1 && fred64(e[c - 1], f) != 0;
    uint32_t dbar = fred64(d[c], f), ta = 1, tb = 0;
    int32_t mate = -1;
    if (first || second) {
        const int64_t j = first ? c : c - 1;  // the block is (j, j+1)
        const uint32_t x = fred64(d[j], f), g = fred64(d[j + 1], f), beta = fred64(e[j], f);
        mate = (int32_t)(first ? c + 1 : c - 1);
        if (x == 0 && g == 0) {
            // [[0, β], [β, 0]] = T·Diag(β/2, −β/2)·Tᵀ, T = [[1, 1], [1, −1]]
            const uint32_t h = fmul(beta, f.inv2, f);
            ta = first ? 1u : p - 1;
            tb = 1;
            dbar = first ? h : fneg(h, p);
        } else if (g != 0) {
            // T = [[1, β/γ], [0, 1]], d̄ = (x − β²/γ, γ)
            const uint32_t r = fmul(beta, finv(g, f), f);
            if (first) {
                tb = 0;
                dbar = fadd(x, fneg(fmul(beta, r, f), p), p);
            } else {
                tb = r;
                dbar = g;
            }
        } else {
            // T = [[1, 0], [β/x, 1]], d̄ = (x, −β²/x)
            const uint32_t r = fmul(beta, finv(x, f), f);
            if (first) {
                tb = r;
                dbar = x;
            } else {
                tb = 0;
                dbar = fneg(fmul(beta, r, f), p);
            }
        }
    }
    sp.dbar[c] = dbar;
    sp.ta[c] = ta;
    sp.tb[c] = tb;
    sp.mate[c] = mate;
    // one exponentiation gives both the Legendre symbol and the start of the
    // square root
    const TsStart st = dbar ? ts_start(dbar, f) : TsStart{1u, 0u};
    const bool ns = dbar != 0 && !ts_is_square(st.t, f);
    sp.flag[c] = ns ? 1u : 0u;
    if (!ns) {
        bool bad = false;
        const uint32_t u = dbar ? ts_finish(st, f, &bad) : 0u;
        // √d̄_c·T_c, in the host planner's term order (column c, then mate)
        col.add(c, fmul(u, ta, f), k, p, &bad);
        if (mate >= 0) col.add(mate, fmul(u, tb, f), k, p, &bad);
        if (bad) atomicOr(err, 2u);
    }
    col.store(sp, c, f.p);
}

// One CTA: ns[r] = the r-th column with a non-square d̄, in column order;
// ns_count = their number.  Columns go in chunks of 8 per thread.
constexpr int RANK_THREADS = 1024;
constexpr int RANK_PER_THREAD = 8;
__global__ void __launch_bounds__(RANK_THREADS) k_scale_rank(int64_t k, ScalePlan sp) {
    __shared__ int warp_tot[RANK_THREADS / 32];
    __shared__ int64_t base_s;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) base_s = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < k; c0 += (int64_t)RANK_THREADS * RANK_PER_THREAD) {
        const int64_t my0 = c0 + (int64_t)tid * RANK_PER_THREAD;
        int cnt = 0;
        for (int t = 0; t < RANK_PER_THREAD; ++t)
            if (my0 + t < k && sp.flag[my0 + t]) ++cnt;
        // exclusive prefix over the CTA
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int v = warp_tot[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            warp_tot[lane] = v;  // inclusive over warps
        }
        __syncthreads();
        const int64_t base = base_s;
        int64_t r = base + (wid ? warp_tot[wid - 1] : 0) + (incl - cnt);
        for (int t = 0; t < RANK_PER_THREAD; ++t)
            if (my0 + t < k && sp.flag[my0 + t]) sp.ns[r++] = (int32_t)(my0 + t);
        __syncthreads();
        if (tid == 0) base_s = base + warp_tot[RANK_THREADS / 32 - 1];
        __syncthreads();
    }
    if (tid == 0) *sp.ns_count = base_s;
}

// Pair q: non-squares ns[2q] = i and ns[2q+1] = j (or the added zero column
// j = k, given d̄_i again, when the count is odd).  Algorithm 4 gives
// [[a, b], [c, dd]] with a² + b² = d̄_i, c² + dd² = d̄_j, ac + bd = 0; column i
// of W is a·T_i + c·T_j, column j is dd·T_j + b·T_i.
__global__ void __launch_bounds__(128) k_scale_pairs(int64_t k, int64_t kk, ScaleConst f,
                                                     ScalePlan sp, unsigned int *err) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t cnt = *sp.ns_count;
    if (2 * q >= cnt) return;
    const int64_t i = sp.ns[2 * q];
    const int64_t j = 2 * q + 1 < cnt ? sp.ns[2 * q + 1] : k;
    if (j >= kk) {  // an odd count the host did not plan a column for
        atomicOr(err, 2u);
        return;
    }
    const uint32_t p = f.p;
    bool bad = false;
    const uint32_t alpha = sp.dbar[i];
    const uint32_t beta = j < k ? sp.dbar[j] : alpha;
    // Algorithm 3 for the non-square α: a² = α/s, b = a·√(s − 1), s the
    // least non-square; then dd = a·√(β/α), c = −b·dd/a.  Written as two
    // independent chains, a → 1/a and 1/α → √(β/α), which the SM overlaps.
    const uint32_t a = fsqrt(fmul(alpha, f.s_inv, f), f, &bad);
    const uint32_t alpha_inv = finv(alpha, f);
    const uint32_t ainv = finv(a, f);
    const uint32_t root = fsqrt(fmul(beta, alpha_inv, f), f, &bad);
    const uint32_t b = fmul(a, f.c_sos, f);
    const uint32_t dd = fmul(a, root, f);
    const uint32_t c = fneg(fmul(fmul(b, dd, f), ainv, f), p);
    WCol ci, cj;
    ci.clear();
    cj.clear();
    add_t(ci, i, a, sp, k, f, &bad);
    add_t(ci, j, c, sp, k, f, &bad);
    add_t(cj, j, dd, sp, k, f, &bad);
    add_t(cj, i, b, sp, k, f, &bad);
    ci.store(sp, i, p);
    cj.store(sp, j, p);
    if (bad) atomicOr(err, 2u);
}

// Ā = A·W: column c of Ā is Σ_t w_{c,t}·A_{src_{c,t}} over at most four
// columns of A (the used terms first, src −1 after them), with A's entries
// any uint32: Shoup's product x·w mod p needs no reduction of x < 2^32.  One
// thread per column of a 256-column block, each looping over many rows (grid
// y strides the rows, four rows per step with their loads issued first), so
// W's column is loaded once per thread and only its used terms are computed.
__global__ void __launch_bounds__(256) k_col_mix(const uint32_t *__restrict__ A, int64_t lda,
                                                 int64_t n, int64_t kk,
                                                 const int4 *__restrict__ src,
                                                 const uint4 *__restrict__ w, uint32_t *B,
                                                 int64_t ldb, ModP m) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= kk) return;
    const int4 s4 = src[c];
    const uint4 w01 = w[2 * c], w23 = w[2 * c + 1];
    const int sc[4] = {s4.x, s4.y, s4.z, s4.w};
    const MulConst wc[4] = {{w01.x, w01.y}, {w01.z, w01.w}, {w23.x, w23.y}, {w23.z, w23.w}};
    const int nt = (sc[0] >= 0) + (sc[1] >= 0) + (sc[2] >= 0) + (sc[3] >= 0);
    const uint32_t p = m.p;
    const int64_t gy = gridDim.y;
    for (int64_t r0 = blockIdx.y; r0 < n; r0 += 4 * gy) {
        uint32_t y[4] = {0u, 0u, 0u, 0u};
        for (int t = 0; t < nt; ++t) {
            uint32_t x[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t r = r0 + q * gy;
                x[q] = r < n ? __ldg(A + r * lda + sc[t]) : 0u;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t qq = __umulhi(x[q], wc[t].w_sh);
                uint32_t v = x[q] * wc[t].w - qq * p;  // in [0, 2p)
                v = v >= p ? v - p : v;
                y[q] = fadd(y[q], v, p);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t r = r0 + q * gy;
            if (r < n) B[r * ldb + c] = y[q];
        }
    }
}

}  // namespace

cudaError_t launch_scale_plan(const uint32_t *d_dev, const uint32_t *e_dev, bool has_e, int64_t k,
                              int64_t kk, const ScaleConst &f, const ScalePlan &sp,
                              unsigned int *err, cudaStream_t st) {
    if (kk == 0) return cudaSuccess;
    k_scale_cols<<<(unsigned)((kk + 255) / 256), 256, 0, st>>>(d_dev, e_dev, has_e ? 1 : 0, k, kk,
                                                               f, sp, err);
    if (k > 0) {
        k_scale_rank<<<1, RANK_THREADS, 0, st>>>(k, sp);
        const int64_t pairs = (k + 2) / 2;
        k_scale_pairs<<<(unsigned)((pairs + 127) / 128), 128, 0, st>>>(k, kk, f, sp, err);
    }
    return cudaGetLastError();
}

cudaError_t launch_col_mix(const uint32_t *A, int64_t lda, int64_t n, int64_t kk, const int4 *src,
                           const uint4 *w, uint32_t *B, int64_t ldb, ModP mp, cudaStream_t st) {
    if (n == 0 || kk == 0) return cudaSuccess;
    // about 16 blocks of 256 threads per SM in all, each thread on n/grid.y rows
    const int64_t gx = (kk + 255) / 256;
    const int64_t gy = std::max<int64_t>(1, std::min<int64_t>(n, (152 * 16 + gx - 1) / gx));
    dim3 grid((unsigned)gx, (unsigned)gy);
    k_col_mix<<<grid, 256, 0, st>>>(A, lda, n, kk, src, w, B, ldb, mp);
    return cudaGetLastError();
}

}  // namespace fsk
